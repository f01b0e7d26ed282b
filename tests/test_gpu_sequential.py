"""Sequential relaxed clipping (Algorithm 3) on the GPU, in row order and in the
constraint-importance order of the Appendix's heuristics, against the oracle through the C-ABI,
at the bar of test_gpu_parity (boxes contain the oracle's and are at most two FP32 ulps wider,
flags exact, bounds within 1e-5 of their scale and never tighter)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case  # noqa: E402
from tests.test_gpu_parity import compare, gpu_round  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    ("mlp32_many_rows", dict(dims=[32, 40, 40, 6], B=40, kmin=0, kmax=2, eps=0.1, sweeps=6, cut_rows=(0, 6))),
    ("mlp5x50_rows_and_splits", dict(dims=[5] + [50] * 6 + [5], B=128, kmin=0, kmax=8, eps=0.05, centre="pm1",
                                     clip01=False, out_rows=1, sweeps=0)),
    ("mlp784_ragged", dict(dims=[784, 70, 70, 10], B=37, kmin=1, kmax=4, eps=0.02, sweeps=10)),
    ("mlp24_up_to_20_rows", dict(dims=[24, 32, 32, 6], B=24, kmin=0, kmax=3, eps=0.1, sweeps=3, cut_rows=(4, 20))),
    ("mlp4_cutting_rows", dict(dims=[4, 16, 16, 3], B=40, kmin=0, kmax=2, eps=0.3, sweeps=4, cut_rows=(2, 6), seed=8)),
]


@pytest.mark.parametrize("relaxed", [2, 3])
@pytest.mark.parametrize("name,kw", CASES)
def test_sequential_round_parity(name, kw, relaxed):
    case = Case(relaxed=relaxed, **kw)
    g = gpu_round(case)
    o = case.oracle()
    compare(case, g, o)


@pytest.mark.parametrize("relaxed", [2, 3])
def test_sequential_tighter_than_parallel(relaxed):
    # Algorithm 3 clips each row against the box the earlier rows left: its box lies inside
    # Algorithm 2's (both GPU, both checked against the oracle above).
    # (Four inputs: there Theorem 2 cuts often; on the oracle this case's total box width is
    # 72.1 parallel, 71.4 sequential and 72.0 in the importance order.)
    kw = dict(dims=[4, 16, 16, 3], B=40, kmin=0, kmax=2, eps=0.3, sweeps=0, cut_rows=(2, 6), seed=7)
    gp = gpu_round(Case(relaxed=1, **kw))
    gs = gpu_round(Case(relaxed=relaxed, **kw))
    ok = (gp["infeasible"] == 0) & (gs["infeasible"] == 0)
    assert np.all(gs["lo_clip"][ok] >= gp["lo_clip"][ok]) and np.all(gs["hi_clip"][ok] <= gp["hi_clip"][ok])
    assert np.all(gs["infeasible"] >= gp["infeasible"])
    tighter = (gs["hi_clip"][ok] - gs["lo_clip"][ok]).sum() < (gp["hi_clip"][ok] - gp["lo_clip"][ok]).sum()
    assert tighter


def test_sequential_jointly_infeasible_rows():
    # Two rows each feasible on the box but not together (x_0 >= c and x_0 <= c - d), and a
    # subdomain where the second row only becomes infeasible on the box the first one left.
    case = Case([6, 10, 10, 3], 3, 0, 0, 0.3, sweeps=2, seed=5, relaxed=2)
    lo, hi = case.lo[0].astype(np.float64), case.hi[0].astype(np.float64)
    c = 0.5 * (lo[0] + hi[0])
    G = np.zeros((5, case.n0))
    h = np.zeros(5)
    G[0, 0], h[0] = -1.0, c                 # x_0 >= c
    G[1, 0], h[1] = 1.0, -(c - 0.01)        # x_0 <= c - 0.01
    G[2, 0], h[2] = -1.0, c                 # subdomain 1: x_0 >= c ...
    G[3, :2], h[3] = [1.0, 1.0], -(c + lo[1] - 0.02)  # ... and x_0 + x_1 <= c + lo_1 - 0.02
    G[4, 1], h[4] = 1.0, -hi[1]             # subdomain 2: redundant (x_1 <= hi_1)
    case.row_off = np.array([0, 2, 4, 5], np.int32)
    case.G, case.h = G.astype(np.float32), h.astype(np.float32)
    case.max_rows = 2
    for relaxed in (2, 3):
        case.relaxed = relaxed
        g = gpu_round(case)
        o = case.oracle()
        assert o["infeasible"].tolist() == [1, 1, 0]
        compare(case, g, o)


def test_relaxed_mode_out_of_range_is_refused():
    case = Case([8, 10, 3], 2, 1, 2, 0.1)
    case.relaxed = 4
    with pytest.raises(RuntimeError, match="bad options"):
        gpu_round(case)
