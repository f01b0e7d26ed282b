"""The oracle's clipping solvers against brute force and the mathematics.

Pins: Lemma A.1 (box extremes at vertices), Theorem 1 (one-row complete clipping
is the exact LP optimum; equals the fractional-knapsack greedy), Theorem 2
(one-row relaxed clipping is component-wise tight; with several rows, the tightest row per
coordinate), weak duality and monotone
ascent for Algorithm 1 with several rows, its exactness when the rows' supports are disjoint (a
separable dual), the a-priori infeasibility test, the
order-dependency example of the Appendix (Algorithm 3 vs Algorithm 2), the constraint
importance order (hyperplane distances by least squares), and the batch round's relaxed
modes (parallel, sequential, sequential in importance order) on a hand-derived example and
against sampled feasible points."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from tests._brute import knapsack_greedy, lp_vertex


def rand_box(rng, n):
    lo = rng.uniform(-1.0, 0.5, n)
    hi = lo + rng.uniform(0.05, 2.0, n)
    return lo, hi


def cutting_row(rng, lo, hi, spread=0.8):
    g = rng.normal(size=lo.size)
    xh, ep = (lo + hi) / 2, (hi - lo) / 2
    h = -(g @ xh) + rng.uniform(-spread, spread) * (np.abs(g) @ ep)
    return g, h


def test_concretize_equals_vertex_extremes():
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = int(rng.integers(1, 7))
        lo, hi = rand_box(rng, n)
        a, c = rng.normal(size=n), rng.normal()
        vals = [a @ np.where(np.array(bits), hi, lo) + c for bits in itertools.product([0, 1], repeat=n)]
        vmin, vmax = O.concretize(a, c, lo, hi)
        assert vmin == pytest.approx(min(vals), abs=1e-12)
        assert vmax == pytest.approx(max(vals), abs=1e-12)


def test_one_row_complete_clip_is_lp_and_knapsack():
    rng = np.random.default_rng(2)
    for _ in range(200):
        n = int(rng.integers(1, 6))
        lo, hi = rand_box(rng, n)
        g, h = cutting_row(rng, lo, hi)
        a, c = rng.normal(size=n), rng.normal()
        lp = lp_vertex(a, c, [g], [h], lo, hi)
        ks = knapsack_greedy(a, c, g, h, lo, hi)
        v, beta, _ = O.complete_clip(a, c, [g], [h], lo, hi, sweeps=1)
        assert beta[0] >= 0.0
        assert v == pytest.approx(lp, abs=1e-9 * (1 + abs(lp)))
        assert ks == pytest.approx(lp, abs=1e-9 * (1 + abs(lp)))


def test_one_row_relaxed_clip_is_componentwise_tight():
    rng = np.random.default_rng(3)
    for _ in range(100):
        n = int(rng.integers(1, 6))
        lo, hi = rand_box(rng, n)
        g, h = cutting_row(rng, lo, hi)
        lo2, hi2, inf = O.relaxed_clip([g], [h], lo, hi)
        assert not inf
        for i in range(n):
            e = np.eye(n)[i]
            assert lo2[i] == pytest.approx(lp_vertex(e, 0.0, [g], [h], lo, hi, "min"), abs=1e-9)
            assert hi2[i] == pytest.approx(lp_vertex(e, 0.0, [g], [h], lo, hi, "max"), abs=1e-9)


def test_multi_row_relaxed_clip_is_the_tightest_row_on_the_same_box():
    """Algorithm 2 clips the box with every row against the same (unclipped) box and keeps the
    tightest end per coordinate: each end is the best of the rows' one-row LP optima (Theorem 2),
    computed here by vertex enumeration for each row alone."""
    rng = np.random.default_rng(9)
    for _ in range(60):
        n = int(rng.integers(1, 5))
        R = int(rng.integers(2, 4))
        lo, hi = rand_box(rng, n)
        rows = [cutting_row(rng, lo, hi, spread=0.5) for _ in range(R)]
        G = [g for g, _ in rows]
        h = [hh for _, hh in rows]
        lo2, hi2, inf = O.relaxed_clip(G, h, lo, hi)
        want_lo = np.array([max(lp_vertex(np.eye(n)[i], 0.0, [g], [hh], lo, hi, "min") for g, hh in rows)
                            for i in range(n)])
        want_hi = np.array([min(lp_vertex(np.eye(n)[i], 0.0, [g], [hh], lo, hi, "max") for g, hh in rows)
                            for i in range(n)])
        gap = np.max(want_lo - want_hi)
        if abs(gap) <= 1e-9:
            continue  # an interval closing to a point: the decision is a tie
        # the rows' intervals fail to meet in some coordinate exactly when the batch is infeasible
        assert inf == (gap > 0), (gap, inf)
        if not inf:
            assert np.allclose(lo2, want_lo, rtol=0, atol=1e-9)
            assert np.allclose(hi2, want_hi, rtol=0, atol=1e-9)


def test_multi_row_weak_duality_and_monotone_ascent():
    rng = np.random.default_rng(4)
    for _ in range(80):
        n = int(rng.integers(2, 5))
        R = int(rng.integers(2, 4))
        lo, hi = rand_box(rng, n)
        # rows through a common interior point keep the system feasible
        x0 = lo + (hi - lo) * rng.uniform(0.3, 0.7, n)
        G = rng.normal(size=(R, n))
        h = -(G @ x0) - rng.uniform(0.0, 0.3, R) * (np.abs(G) @ ((hi - lo) / 2))
        a, c = rng.normal(size=n), rng.normal()
        lp = lp_vertex(a, c, G, h, lo, hi)
        base, _ = O.concretize(a, c, lo, hi)
        prev = base
        for s in range(1, 6):
            v, beta, _ = O.complete_clip(a, c, G, h, lo, hi, sweeps=s)
            assert np.all(beta >= 0.0)
            assert v <= lp + 1e-9 * (1 + abs(lp))          # weak duality
            assert v >= prev - 1e-12 * (1 + abs(prev))      # ascent never decreases the dual
            assert O.dual_value(a, c, G, h, lo, hi, beta) == pytest.approx(v, abs=1e-12 * (1 + abs(v)))
            prev = v


def test_multi_row_disjoint_supports_is_exact_lp():
    """Rows on disjoint sets of coordinates make the dual separable: D(beta) is a constant plus one
    concave 1-D dual per row, and each row step of Algorithm 1 maximises its own exactly (Theorem 1),
    whatever the other multipliers. So one sweep reaches the dual optimum, and by LP duality the value
    is the exact LP optimum over the box and all rows (vertex enumeration)."""
    rng = np.random.default_rng(8)
    for _ in range(80):
        R = int(rng.integers(2, 4))
        sizes = rng.integers(1, 3, size=R)
        while sizes.sum() > 4:
            sizes[int(np.argmax(sizes))] -= 1
        n = int(sizes.sum()) + int(rng.integers(0, 2))  # plus at most one coordinate in no row
        lo, hi = rand_box(rng, n)
        xh, ep = (lo + hi) / 2, (hi - lo) / 2
        perm = rng.permutation(n)
        G = np.zeros((R, n))
        h = np.zeros(R)
        start = 0
        for p in range(R):
            idx = perm[start:start + sizes[p]]
            start += sizes[p]
            G[p, idx] = rng.normal(size=idx.size)
            h[p] = -(G[p] @ xh) + rng.uniform(-0.6, 0.6) * (np.abs(G[p]) @ ep)  # cuts its own coordinates
        a, c = rng.normal(size=n), rng.normal()
        lp = lp_vertex(a, c, G, h, lo, hi)
        for sweeps in (1, 3):
            v, beta, _ = O.complete_clip(a, c, G, h, lo, hi, sweeps=sweeps)
            assert np.all(beta >= 0.0)
            assert v == pytest.approx(lp, abs=1e-9 * (1 + abs(lp))), (sweeps, v, lp)


def test_infeasibility_precheck_matches_lp():
    rng = np.random.default_rng(5)
    for _ in range(100):
        n = int(rng.integers(1, 5))
        lo, hi = rand_box(rng, n)
        g, h = cutting_row(rng, lo, hi, spread=2.0)
        f, vmin, vmax, _ = O.row_check(g, h, lo, hi)
        lp = lp_vertex(g, h, None, None, lo, hi)  # min over the box of g.x + h
        assert vmin == pytest.approx(lp, abs=1e-12)
        assert (f == 1) == (lp > 0)
        if f == 1:
            lo2, hi2, inf = O.relaxed_clip([g], [h], lo, hi)
            assert inf


def test_clipped_box_contains_feasible_samples():
    rng = np.random.default_rng(6)
    for _ in range(30):
        n = int(rng.integers(2, 8))
        R = int(rng.integers(1, 4))
        lo, hi = rand_box(rng, n)
        G = np.stack([cutting_row(rng, lo, hi)[0] for _ in range(R)])
        h = np.array([cutting_row(rng, lo, hi)[1] for _ in range(R)])
        for seq in (False, True):
            lo2, hi2, inf = O.relaxed_clip(G, h, lo, hi, sequential=seq)
            assert np.all(lo2 >= lo) and np.all(hi2 <= hi)
            X = lo + (hi - lo) * rng.uniform(size=(4000, n))
            feas = np.all(X @ G.T + h <= 0, axis=1)
            if inf:
                assert not feas.any()
            else:
                assert np.all(X[feas] >= lo2 - 1e-12) and np.all(X[feas] <= hi2 + 1e-12)
        lop, hip, _ = O.relaxed_clip(G, h, lo, hi)
        los, his, infs = O.relaxed_clip(G, h, lo, hi, sequential=True)
        if not infs:
            assert np.all(los >= lop - 1e-12) and np.all(his <= hip + 1e-12)


def test_order_dependency_example():
    # Appendix, order dependency: sequential clipping depends on the row order when one
    # row's clip uses a bound that the other row tightens.  Instance on the box [0,2]^2:
    # F1: x1 + x2 <= 2 (clips x1 <= 2 - lo2), F2: -x2 + 1 <= 0 (lo2 = 1).
    lo, hi = np.array([0.0, 0.0]), np.array([2.0, 2.0])
    G = np.array([[1.0, 1.0], [0.0, -1.0]])
    h = np.array([-2.0, 1.0])
    a_lo, a_hi, _ = O.relaxed_clip(G, h, lo, hi, sequential=True)          # F1 then F2
    b_lo, b_hi, _ = O.relaxed_clip(G[::-1], h[::-1], lo, hi, sequential=True)  # F2 then F1
    p_lo, p_hi, _ = O.relaxed_clip(G, h, lo, hi, sequential=False)
    assert np.array_equal(a_hi, [2.0, 2.0]) and np.array_equal(a_lo, [0.0, 1.0])
    assert np.array_equal(b_hi, [1.0, 2.0]) and np.array_equal(b_lo, [0.0, 1.0])
    # the exact feasible range of x1 is [0, 1]: F2-then-F1 reaches it, F1-then-F2 does not
    assert lp_vertex([1.0, 0.0], 0.0, G, h, lo, hi, "max") == pytest.approx(1.0)
    # the parallel box is order-independent and contains both sequential boxes
    assert np.all(p_lo <= a_lo) and np.all(p_hi >= a_hi)
    assert np.all(p_lo <= b_lo) and np.all(p_hi >= b_hi)


def test_row_order_is_ascending_hyperplane_distance():
    # Constraint importance heuristic (Appendix, details of heuristics): rows ascend in the
    # distance of their hyperplane from the box centre.  The distance is measured here as the
    # length of the least-norm correction that moves the centre onto the hyperplane
    # (np.linalg.lstsq), not by the closed form the oracle uses.
    rng = np.random.default_rng(11)
    for _ in range(20):
        n = int(rng.integers(2, 9))
        R = int(rng.integers(1, 7))
        lo, hi = rand_box(rng, n)
        xh = (lo + hi) / 2
        G = rng.normal(size=(R, n))
        h = rng.normal(size=R) * 2.0
        if R >= 3:
            G[2], h[2] = G[0], h[0]          # an exact tie: stays after row 0
        perm = O.row_order(G, h, lo, hi)
        dist = []
        for k in range(R):
            y, *_ = np.linalg.lstsq(G[k][None, :], np.array([-h[k] - G[k] @ xh]), rcond=None)
            dist.append(np.linalg.norm(y))
        d = np.array(dist)[perm]
        assert sorted(perm.tolist()) == list(range(R))
        assert np.all(np.diff(d) >= -1e-12 * (1 + d[1:]))
        if R >= 3:
            assert perm.tolist().index(0) < perm.tolist().index(2)
    # a zero row has no hyperplane: it goes last
    G = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    perm = O.row_order(G, [1.0, -5.0, -0.5], [0.0, 0.0], [1.0, 1.0])
    assert perm.tolist() == [2, 1, 0]


def _two_input_round(relaxed):
    # A 2-input ReLU net and two extra rows on the box [0,2] x [0,3]:
    #   F1: x1 + x2 - 2 <= 0,   F2: -x2 + 1.4 <= 0.
    # Theorem 2 by hand.  Parallel (Algorithm 2, both rows on the input box): F1 gives
    # hi1 = 2 - lo2 = 2, hi2 = 2 - lo1 = 2; F2 gives lo2 = 1.4: box [0,2] x [1.4,2].
    # Sequential in row order (F1 then F2): F1 -> [0,2] x [0,2], F2 -> [0,2] x [1.4,2].
    # Sequential in the constraint-importance order: the centre (1, 1.5) lies at
    # |1 + 1.5 - 2| / sqrt(2) = 0.354 from F1 and |-1.5 + 1.4| = 0.1 from F2, so F2 first:
    # [0,2] x [1.4,3], then F1: hi1 = 2 - 1.4 = 0.6, hi2 = 2 - 0 = 2 -> [0,0.6] x [1.4,2].
    from paper_2512_11087_gb300 import workloads as WL
    net = O.Net(WL.he_mlp([2, 4, 1], seed=0))
    lo, hi = np.array([0.0, 0.0]), np.array([2.0, 3.0])
    cache = O.make_cache(O.root_crown(net, lo, hi))
    G = np.array([[1.0, 1.0], [0.0, -1.0]])
    h = np.array([-2.0, 1.4])
    out = O.bound_batch(net, cache, lo[None], hi[None], row_off=np.array([0, 2], np.int32), G=G, h=h,
                        C=np.ones((1, 1)), t=np.zeros(1), relaxed=relaxed, sweeps=0)
    return out["lo_clip"][0], out["hi_clip"][0], out["infeasible"][0]


@pytest.mark.parametrize("relaxed,want_lo,want_hi", [
    (1, [0.0, 1.4], [2.0, 2.0]),
    (2, [0.0, 1.4], [2.0, 2.0]),
    (3, [0.0, 1.4], [0.6, 2.0]),
])
def test_round_relaxed_modes_on_hand_example(relaxed, want_lo, want_hi):
    lo, hi, inf = _two_input_round(relaxed)
    assert not inf
    # the box is stored in FP32, rounded outward: within one FP32 step outside the exact value
    for got, want, up in [(lo, want_lo, False), (hi, want_hi, True)]:
        for g, w in zip(got, want):
            step = float(np.spacing(np.float32(w)))
            if up:
                assert w <= g <= w + step
            else:
                assert w - step <= g <= w


def test_round_sequential_modes_tighter_than_parallel_and_sound():
    # Algorithm 3 clips each row against the box the earlier rows left, so its box lies
    # inside Algorithm 2's; both contain every feasible point (sampled).
    from paper_2512_11087_gb300 import workloads as WL
    rng = np.random.default_rng(12)
    net = O.Net(WL.he_mlp([4, 8, 8, 2], seed=3))
    lo0, hi0 = np.full(4, -1.0), np.full(4, 1.0)
    cache = O.make_cache(O.root_crown(net, lo0, hi0))
    B = 12
    lo, hi = np.tile(lo0, (B, 1)), np.tile(hi0, (B, 1))
    row_off, G, h = WL.random_cut_rows(lo, hi, B, 1, 4, seed=5)
    boxes = {}
    for mode in (1, 2, 3):
        o = O.bound_batch(net, cache, lo, hi, row_off=row_off, G=G, h=h, C=np.ones((1, 2)), t=np.zeros(1),
                          relaxed=mode, sweeps=0)
        boxes[mode] = (o["lo_clip"], o["hi_clip"], o["infeasible"])
    X = rng.uniform(-1, 1, size=(20000, 4))
    for b in range(B):
        rows = slice(row_off[b], row_off[b + 1])
        feas = np.all(X @ G[rows].T + h[rows] <= 0, axis=1)
        for mode in (1, 2, 3):
            l, u, inf = boxes[mode][0][b], boxes[mode][1][b], boxes[mode][2][b]
            if inf:
                assert not feas.any()
                continue
            assert np.all(X[feas] >= l - 1e-12) and np.all(X[feas] <= u + 1e-12)
        if not boxes[1][2][b]:
            for mode in (2, 3):
                if not boxes[mode][2][b]:
                    assert np.all(boxes[mode][0][b] >= boxes[1][0][b]) and np.all(boxes[mode][1][b] <= boxes[1][1][b])
