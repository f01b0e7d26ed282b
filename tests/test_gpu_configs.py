"""Parity on the shapes of two further workload families, against the FP64 oracle through the
C-ABI, at batch sizes the oracle finishes in seconds:

* the BaB stress shape (784 -> 512x8 -> 10, 0-24 split constraints per subdomain, relaxed +
  complete clipping with 10 sweeps), on the split-precision and the FP32 path;
* a CIFAR-style CNN (three convolutions, two dense layers) with uneven 1-16 splits per subdomain,
  bounded once directly and once by replaying a captured CUDA graph of the same round."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402
from tests.test_gpu_parity import compare, gpu_round  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stress_case():
    case = Case([784] + [512] * 8 + [10], 8, 0, 24, 0.02, sweeps=10, seed=5)
    return case, case.oracle()


@pytest.mark.parametrize("precision", [1, 0])
def test_stress_shape_parity(stress_case, precision):
    case, o = stress_case
    assert case.max_splits > 8  # exercises the wide complete-clipping launch
    g = gpu_round(case, precision=precision)
    st = compare(case, g, o)
    print("stress shape", precision, st)


def test_cnn_uneven_rows_graph_replay_parity():
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    layers = WL.he_cnn((3, 16, 16), [(8, 4, 2, 1), (16, 4, 2, 1), (16, 3, 1, 1)], [40, 10], seed=6)
    case = Case(None, 32, 1, 16, 2.0 / 255.0, layers=layers, sweeps=5, seed=6)
    counts = np.diff(case.split_off)
    assert counts.min() >= 1 and counts.max() > 8
    o = case.oracle()
    direct = gpu_round(case)
    compare(case, direct, o)
    # the same round captured in a graph and replayed
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, sweeps=case.sweeps)
    d = E.to_dev
    rnd.capture(d(case.lo), d(case.hi), d(case.C), d(case.t), split_off=d(case.split_off),
                split_ids=d(case.split_ids))
    out = rnd.replay()
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    for k in direct:
        assert np.array_equal(direct[k], g[k]), k
    assert capi.cv_device_status(net.handle) == 0
    capi.cv_graph_destroy(rnd.graph)
    net.close()
