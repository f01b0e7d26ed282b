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


@pytest.mark.parametrize("precision", [0, 1])
def test_cnn3x32_full_size_sampled(precision):
    """The CIFAR-style CNN of the benchmark table at its full size: 3x32x32 input, 2048 subdomains with
    1-16 splits, relaxed + complete clipping (10 sweeps) on 80 seeded target slots per subdomain, on
    the FP32 and the split-BF16 tensor-core path (the dense conv layers have up to 4096 outputs: eight
    passes).  The GPU bounds all 2048 subdomains (rows too large to stage in shared memory: the wide
    complete-clipping launch takes every subdomain); the oracle bounds 8 of them, evenly spaced."""
    from paper_2512_11087_gb300 import workloads as WL
    cfg = WL.CONFIGS["cnn3x32"]
    layers = WL.he_cnn(cfg["in_shape"], cfg["convs"], cfg["fcs"], seed=0)
    case = Case(None, cfg["B"], cfg["kmin"], cfg["kmax"], cfg["eps"], layers=layers, sweeps=cfg["sweeps"], seed=0,
                targets=80)
    g = gpu_round(case, precision=precision)
    sample = (np.arange(8) * case.B) // 8 + 3
    sub = Case.__new__(Case)
    sub.__dict__.update(case.__dict__)
    sub.B = sample.size
    sub.lo, sub.hi = case.lo[sample], case.hi[sample]
    so, ids = np.zeros(sample.size + 1, np.int32), []
    to, tids = np.zeros(sample.size + 1, np.int32), []
    for i, b in enumerate(sample):
        seg = case.split_ids[case.split_off[b]:case.split_off[b + 1]]
        ids.append(seg)
        so[i + 1] = so[i] + seg.size
        tseg = case.tgt_ids[case.tgt_off[b]:case.tgt_off[b + 1]]
        tids.append(tseg)
        to[i + 1] = to[i] + tseg.size
    sub.split_off, sub.split_ids = so, np.concatenate(ids).astype(np.int32)
    sub.tgt_off, sub.tgt_ids = to, np.concatenate(tids).astype(np.int32)
    o = sub.oracle(nthreads=0)
    gs = {k: v[sample] for k, v in g.items()}
    st = compare(sub, gs, o)
    print("cnn3x32 sampled parity", st)


@pytest.mark.parametrize("precision", [0, 1])
def test_alpha_gradient_config4_full_size_sampled(precision):
    """Configuration 4's shape at full batch: 784->1024x4->10, 1024 subdomains, slopes per (subdomain,
    spec row, neuron).  The GPU computes all 1024 bounds and gradients (FP32 CUDA-core contractions,
    or the split-BF16 tensor cores with 1024-wide layers in two K passes); 4 subdomains are checked
    against the oracle's FP64 reverse sweep at the bar of tests/test_gpu_alpha.py."""
    from oracle import oracle as O
    from paper_2512_11087_gb300 import engine as E
    from tests.test_gpu_alpha import _full_bounds, _setup, _state
    s = _setup([784, 1024, 1024, 1024, 1024, 10], 1024, 9, eps=0.02)
    st = _state(s, precision)
    lower, grad = st.bound_and_grad(E.to_dev(s["alpha"]))
    torch.cuda.synchronize()
    sample = [0, 341, 682, 1023]
    lower = lower.cpu().numpy()[sample]
    grad = grad[sample].cpu().numpy()
    sub = {k: (v[sample] if isinstance(v, np.ndarray) and v.ndim >= 2 and v.shape[0] == s["B"] else v)
           for k, v in s.items()}
    o = O.bound_batch(s["onet"], s["cache"] | dict(root_l=s["rl"].astype(np.float64),
                                                   root_u=s["ru"].astype(np.float64)),
                      sub["lo"], sub["hi"], l_in=sub["l"], u_in=sub["u"], C=s["C"], t=s["t"],
                      alpha=sub["alpha"].astype(np.float64), relaxed=0, sweeps=0)
    worst = 0.0
    for i in range(len(sample)):
        hl, hu, hs = _full_bounds(sub, i)
        f, g = O.alpha_grad(s["onet"], hl, hu, hs, sub["lo"][i], sub["hi"][i], s["C"], s["t"],
                            sub["alpha"][i].astype(np.float64))
        sc = o["lower_scale"][i]
        assert np.all(lower[i] <= f + 1e-12 * sc)
        assert np.all(np.abs(lower[i] - f) <= 1e-5 * sc)
        for r in range(s["m"]):
            gmax = np.max(np.abs(g[r]))
            if gmax == 0:
                assert np.all(grad[i, r] == 0)
                continue
            err = np.max(np.abs(grad[i, r] - g[r])) / gmax
            worst = max(worst, err)
            assert err <= 1e-4, (i, r, err)
    print("config-4 sampled gradient error / row max", worst)
    s["net"].close()
