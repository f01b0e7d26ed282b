"""The oracle's activation-BaB loop (Algorithm 5) on tiny networks.

Pins: (1) soundness against brute force -- the exact minimum of the spec over the input box, by
enumerating every activation pattern of a 2-input net and solving each pattern's LP on its linear
region by vertex enumeration: a "verified" answer needs a positive minimum, a negative minimum must
leave the answer "unknown"; (2) the bookkeeping identities of every iteration (each parent gives
two children or is stuck; each child is verified, infeasible, depth-limited or pushed; the list
shrinks by the picked parents and grows by the pushed children); (3) the stack discipline (the
untouched bottom of the list, children carrying their parent's codes plus one); (4) a root that
verifies ends the loop before the first iteration."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_11087_gb300 import workloads as WL
from tests._brute import lp_vertex
from tests._cases import Case


def _exact_min(layers, C, t, lo, hi):
    """min over the box of C_0 y(x) + t_0 by activation patterns (2-D input)."""
    Ws = [np.asarray(l["W"], np.float64) for l in layers]
    bs = [np.asarray(l["b"], np.float64) for l in layers]
    hidden = [w.shape[0] for w in Ws[:-1]]
    best = np.inf
    for pat in itertools.product([0, 1], repeat=sum(hidden)):
        A, c = np.eye(lo.size), np.zeros(lo.size)   # zhat = A x + c
        G, h = [], []
        k = 0
        for i, n in enumerate(hidden):
            zA, zc = Ws[i] @ A, Ws[i] @ c + bs[i]
            s = np.array(pat[k:k + n], float)
            k += n
            for j in range(n):   # active: z_j >= 0 -> -z_j <= 0; inactive: z_j <= 0
                sg = -1.0 if s[j] else 1.0
                G.append(sg * zA[j]); h.append(sg * zc[j])
            A, c = s[:, None] * zA, s * zc
        yA, yc = Ws[-1] @ A, Ws[-1] @ c + bs[-1]
        v = lp_vertex(C[0] @ yA, float(C[0] @ yc + t[0]), np.array(G), np.array(h), lo, hi)
        if v is not None:
            best = min(best, v)
    return best


def _tiny(seed, t0):
    layers = WL.he_mlp([2, 4, 4, 2], seed=seed)
    C = np.array([[1.0, -1.0]])
    t = np.array([t0])
    case = Case(None, 1, 0, 0, 0.5, seed=seed, layers=layers, m_spec=(C, t), clip01=False)
    return case, layers, C, t


def _run(case, C, t, **kw):
    args = dict(batch=4, top_k=-1, capacity=4096, max_depth=8, max_iters=200, sweeps=4)
    args.update(kw)
    return O.activation_bab(case.net, case.cache, case.lo0[None], case.hi0[None], C, t, **args)


def _check_bookkeeping(rec):
    before = 0
    for k, s in enumerate(rec["iters"]):
        if k > 0:
            assert s["children"] == 2 * (s["picked"] - s["stuck"])
        assert s["children"] == s["verified"] + s["infeasible"] + s["depth_limited"] + s["pushed"]
        assert s["remaining"] == before - s["picked"] + s["pushed"]
        assert len(rec["lists"][k]) == s["remaining"]
        before = s["remaining"]


@pytest.mark.parametrize("seed", [3, 4, 5, 6])
def test_loop_is_sound_against_the_exact_minimum(seed):
    case, layers, C, _ = _tiny(seed, 0.0)
    exact0 = _exact_min(layers, C, np.zeros(1), case.lo0.astype(np.float64), case.hi0.astype(np.float64))
    seen = set()
    for shift in (0.05, 0.3, -0.05):      # the threshold moves the true minimum to +-shift
        t = np.array([-exact0 + shift])
        rec = _run(case, C, t)
        _check_bookkeeping(rec)
        seen.add(rec["status"])
        if rec["status"] == "verified":
            assert exact0 + t[0] > 0
        if exact0 + t[0] < 0:
            assert rec["status"] == "unknown"
    assert "unknown" in seen


def test_loop_verifies_a_clear_property_and_counts_domains():
    case, layers, C, _ = _tiny(7, 0.0)
    exact0 = _exact_min(layers, C, np.zeros(1), case.lo0.astype(np.float64), case.hi0.astype(np.float64))
    t = np.array([-exact0 + 0.3])
    rec = _run(case, C, t, sweeps=6)
    _check_bookkeeping(rec)
    assert rec["status"] == "verified"
    visited = sum(s["children"] for s in rec["iters"])
    assert visited >= 1 + 2 * (len(rec["iters"]) - 1)


def test_stack_discipline():
    case, layers, C, _ = _tiny(8, 0.0)
    exact0 = _exact_min(layers, C, np.zeros(1), case.lo0.astype(np.float64), case.hi0.astype(np.float64))
    rec = _run(case, C, np.array([-exact0 + 0.02]), batch=2, max_iters=6)
    _check_bookkeeping(rec)
    for k in range(1, len(rec["lists"])):
        prev, cur, s = rec["lists"][k - 1], rec["lists"][k], rec["iters"][k]
        keep = len(prev) - s["picked"]
        assert cur[:keep] == prev[:keep]                  # the bottom of the stack is untouched
        parents = prev[keep:]
        for codes in cur[keep:]:                          # every pushed child: a parent's codes + one
            assert any(codes[:-1] == p for p in parents) and len(codes) >= 1


def test_root_that_verifies_ends_before_the_first_iteration():
    case, layers, C, _ = _tiny(9, 1e3)
    rec = _run(case, C, np.array([1e3]))
    assert len(rec["iters"]) == 1 and rec["iters"][0]["verified"] == 1 and rec["status"] == "verified"
