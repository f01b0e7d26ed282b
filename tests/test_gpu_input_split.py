"""The input-BaB split step (Algorithm 4; cv_input_split) through the C-ABI against the oracle on
the same inputs: every output bit-exact (boxes, rows, offsets, parents: copies and FP32 decisions
taken in the oracle's order).  Then one whole input-BaB iteration: a round with final planes out,
the split, and a round on the children with their inherited rows, against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402
from tests.test_gpu_parity import compare  # noqa: E402

pytestmark = pytest.mark.gpu


def _gpu_split(lo, hi, A, c, lower, ver, inf):
    from paper_2512_11087_gb300 import engine as E
    d = lambda x, t=torch.float32: torch.as_tensor(np.ascontiguousarray(x)).to("cuda", t)
    out = E.input_split(d(lo), d(hi), d(A), d(c), d(lower), d(ver, torch.uint8), d(inf, torch.uint8))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check_equal(g, o):
    for k in ("lo", "hi", "row_off", "G", "h", "parent"):
        assert g[k].shape == o[k].shape, (k, g[k].shape, o[k].shape)
        assert np.array_equal(g[k].view(np.uint8), np.ascontiguousarray(o[k]).view(np.uint8)), k


def _parents(rng, B, n0, m, p_ver=0.2, p_inf=0.1, one_row=0.3):
    lo = rng.uniform(-1, 0.5, size=(B, n0)).astype(np.float32)
    hi = (lo + rng.uniform(0.0, 1.5, size=(B, n0))).astype(np.float32)
    A = rng.normal(size=(B, m, n0)).astype(np.float32)
    c = rng.normal(size=(B, m)).astype(np.float32)
    lower = rng.normal(size=(B, m)).astype(np.float32)
    single = rng.uniform(size=B) < one_row          # parents with exactly one unproven row
    lower[single] = np.abs(lower[single]) + 0.1
    lower[single, rng.integers(0, m, size=int(single.sum()))] = -0.5
    ver = (rng.uniform(size=B) < p_ver).astype(np.uint8)
    inf = (rng.uniform(size=B) < p_inf).astype(np.uint8)
    return lo, hi, A, c, lower, ver, inf


@pytest.mark.parametrize("B,n0,m,seed", [(200, 37, 5, 1), (64, 784, 9, 2), (4099, 12, 3, 3), (1, 1, 1, 4)])
def test_split_bit_exact(B, n0, m, seed):
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    args = _parents(rng, B, n0, m)
    _check_equal(_gpu_split(*args), O.input_split(*args))


def test_split_edge_cases():
    from oracle import oracle as O
    rng = np.random.default_rng(5)
    lo, hi, A, c, lower, ver, inf = _parents(rng, 30, 8, 2, p_ver=0.0, p_inf=0.0)
    # zero planes (widest axis), equal widths (lowest index), equal scores, a flat box
    A[0] = 0.0
    hi[1] = lo[1] + 1.0
    A[1] = 1.0
    lower[1] = -1.0
    hi[2] = lo[2]
    cases = [(lo, hi, A, c, lower, ver, inf),
             (lo, hi, A, c, lower, np.ones(30, np.uint8), inf),           # every parent dropped
             (lo, hi, A, c, np.full_like(lower, 2.0), ver, inf)]          # every row proven, none flagged
    for args in cases:
        _check_equal(_gpu_split(*args), O.input_split(*args))


def test_split_of_no_parents():
    g = _gpu_split(np.zeros((0, 4)), np.zeros((0, 4)), np.zeros((0, 2, 4)), np.zeros((0, 2)), np.zeros((0, 2)),
                   np.zeros(0), np.zeros(0))
    assert g["row_off"].tolist() == [0] and g["lo"].shape == (0, 4)


def test_one_input_bab_iteration():
    # round (final planes out) -> split -> round on the children with their inherited rows;
    # one spec row so that kept parents pass their plane on
    from oracle import oracle as O
    from paper_2512_11087_gb300 import engine as E
    from paper_2512_11087_gb300 import workloads as WL
    case = Case([6, 24, 24, 3], 48, 0, 0, 0.15, seed=9, sweeps=3, centre="pm1", clip01=False)
    # 48 sub-boxes of the root box (a fifth of its radius), spec row e_0 - e_2: some parents are
    # proven, the others have one unproven row whose plane cuts their children
    rng = np.random.default_rng(19)
    lo0, hi0 = case.lo0.astype(np.float64), case.hi0.astype(np.float64)
    r = 0.5 * (hi0 - lo0)
    cen = lo0 + r + rng.uniform(-0.9, 0.9, size=(48, 6)) * r
    case.lo, case.hi = (cen - 0.2 * r).astype(np.float32), (cen + 0.2 * r).astype(np.float32)
    C, t = WL.margin_spec(3, y=0)
    case.C, case.t, case.m = C[1:2], t[1:2], 1
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    d = E.to_dev
    rnd = E.Round(net, case.B, case.m, sweeps=case.sweeps, want_final=True)
    out = rnd.run(d(case.lo), d(case.hi), d(case.C), d(case.t))
    torch.cuda.synchronize()
    par = {k: v.cpu().numpy().copy() for k, v in out.items()}
    # the split, on the GPU round's own outputs, against the oracle's split of the same arrays
    sp = _gpu_split(par["lo_clip"], par["hi_clip"], par["final_A"], par["final_c"], par["lower"],
                    par["verified"], par["infeasible"])
    _check_equal(sp, O.input_split(par["lo_clip"], par["hi_clip"], par["final_A"], par["final_c"], par["lower"],
                                   par["verified"], par["infeasible"]))
    n = sp["lo"].shape[0]
    assert n > 0 and sp["row_off"][-1] == n          # one unproven row: every child has its plane
    # the children's round (relaxed clipping with the inherited planes) against the oracle
    kid = Case([6, 24, 24, 3], n, 0, 0, 0.15, seed=9, sweeps=3, centre="pm1", clip01=False)
    kid.C, kid.t, kid.m = case.C, case.t, 1
    kid.lo, kid.hi = sp["lo"], sp["hi"]
    kid.row_off, kid.G, kid.h, kid.max_rows = sp["row_off"], sp["G"], sp["h"], 1
    from tests.test_gpu_parity import gpu_round
    g = gpu_round(kid)
    o = kid.oracle()
    compare(kid, g, o)
    # clipping with the inherited plane tightens some child box
    assert np.any(g["lo_clip"] > sp["lo"]) or np.any(g["hi_clip"] < sp["hi"])
    net.close()
