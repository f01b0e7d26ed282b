"""Brute-force tools for tiny inputs (independent of the oracle's algorithms).

lp_vertex: optimum of a linear objective over {lo <= x <= hi, G x + h <= 0} by
enumerating every vertex (n active constraints out of the 2n box faces and the
rows), solving each n x n system in FP64 and keeping the feasible points.
knapsack_greedy: the fractional knapsack greedy of the paper's knapsack
equivalence (sort items by value/weight ratio, take whole items, then a fraction).
"""
import itertools

import numpy as np


def lp_vertex(obj, c0, G, h, lo, hi, sense="min", tol=1e-9):
    obj = np.asarray(obj, np.float64)
    n = obj.size
    G = np.atleast_2d(np.asarray(G, np.float64)) if G is not None and len(G) else np.zeros((0, n))
    h = np.atleast_1d(np.asarray(h, np.float64)) if h is not None and len(h) else np.zeros(0)
    # constraints a.x <= b
    A = [(-np.eye(n)[i], -lo[i]) for i in range(n)] + [(np.eye(n)[i], hi[i]) for i in range(n)]
    A += [(G[k], -h[k]) for k in range(G.shape[0])]
    best = None
    for sub in itertools.combinations(range(len(A)), n):
        M = np.array([A[s][0] for s in sub])
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, np.array([A[s][1] for s in sub]))
        ok = all(a @ x <= bb + tol * (1 + abs(bb)) for a, bb in A)
        if not ok:
            continue
        v = obj @ x + c0
        if best is None or (v < best if sense == "min" else v > best):
            best = v
    return best


def knapsack_greedy(a, c0, g, h, lo, hi):
    """min a.x + c0 s.t. g.x + h <= 0, lo <= x <= hi via the fractional knapsack greedy.

    Change of variables x = lo + (hi-lo) y, y in [0,1]^n turns the problem into
    max r.y s.t. s.y <= cap with r = -(hi-lo) a, s = (hi-lo) g, cap = -(g.lo + h).
    Negative weights are removed by the textbook flip y_j = 1 - y'_j; then items are
    taken whole in decreasing value/weight order and the last one fractionally."""
    a, g, lo, hi = (np.asarray(v, np.float64) for v in (a, g, lo, hi))
    w = hi - lo
    r = -w * a
    s = w * g
    cap = -(g @ lo + h)
    const = 0.0
    flip = s < 0
    # flipped item: value -r, weight -s, and its full weight/value are pre-committed
    cap = cap - s[flip].sum()
    const += r[flip].sum()
    rr = np.where(flip, -r, r)
    ss = np.where(flip, -s, s)
    if cap < 0:
        return np.inf
    yp = np.zeros(a.size)
    # zero-weight items with positive value are free
    free = (ss == 0) & (rr > 0)
    yp[free] = 1.0
    cand = [j for j in range(a.size) if ss[j] > 0 and rr[j] > 0]
    cand.sort(key=lambda j: -rr[j] / ss[j])
    for j in cand:
        take = min(1.0, cap / ss[j])
        yp[j] = take
        cap -= ss[j] * take
        if take < 1.0:
            break
    y = np.where(flip, 1.0 - yp, yp)
    x = lo + w * y
    return a @ x + c0
