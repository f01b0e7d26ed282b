"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Both sides receive the same seeded inputs and the same root cache (the oracle's planes as
FP32 values), so every step is compared on identical data.  Tolerance (the arithmetic of the
kernels, see the file headers of csrc/): a bound may differ from the oracle by at most
1e-5 of its magnitude scale (the sum of the absolute values of the terms that form it, as
the oracle reports it) and must never be tighter than the oracle's, beyond the oracle's
own FP64 rounding (1e-12 of the scale).  Boxes: the GPU machine contains the oracle box and is
at most two FP32 ulps wider.  Integer outputs (infeasible flags, masks) match exactly except
where the oracle's deciding value lies within the tolerance band of the threshold, where the
GPU must take the conservative decision; such cases are counted and must be rare."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5
SOUND = 1e-12
LAST_CC_STATS = []  # decision counters of the last gpu_round (complete clipping)


def gpu_round(case: Case, precision=0, want_weight=False, **kw):
    from paper_2512_11087_gb300 import engine as E
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, max_rows=case.max_rows, relaxed=case.relaxed,
                  sweeps=case.sweeps, precision=precision, alpha_mode=case.alpha_mode, enforce_splits=case.enforce,
                  want_weight=want_weight)
    rnd.enable_timer()
    d = E.to_dev
    out = rnd.run(d(case.lo), d(case.hi), d(case.C), d(case.t), split_off=d(case.split_off),
                  split_ids=d(case.split_ids), row_off=d(case.row_off), G=d(case.G), h=d(case.h),
                  tgt_off=d(case.tgt_off), tgt_ids=d(case.tgt_ids), **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    # complete clipping's decisions with two or more rows: every one certified
    st = rnd.cc_stats()
    LAST_CC_STATS[:] = st
    print("cc row steps, certified, several candidates, widened, uncertified, over the limit:", st)
    assert st[4] == 0, st
    from paper_2512_11087_gb300 import capi
    assert capi.cv_device_status(net.handle) == 0
    net.close()
    return res


def compare(case, g, o, sound_bounds=True, report=None):
    """Element-wise comparison; returns a dict of statistics."""
    st = {}
    U = case.U
    inf_g, inf_o = g["infeasible"].astype(bool), o["infeasible"].astype(bool)
    assert np.array_equal(inf_g, inf_o), (np.nonzero(inf_g != inf_o))
    fe = ~inf_o
    # boxes
    lo_o, hi_o = o["lo_clip"], o["hi_clip"]
    assert np.all(g["lo_clip"] <= lo_o) and np.all(g["hi_clip"] >= hi_o)
    ulp = np.spacing(np.maximum(np.abs(lo_o), np.abs(hi_o)).astype(np.float32)).astype(np.float64)
    st["box_max_ulps"] = float(max(np.max((lo_o - g["lo_clip"]) / ulp), np.max((g["hi_clip"] - hi_o) / ulp)))
    assert st["box_max_ulps"] <= 2.0
    # intermediate bounds
    if U:
        for k, sc in (("l", "l_scale"), ("u", "u_scale")):
            gv, ov, s = g[k][:, :U][fe], o[k][:, :U][fe], o[sc][:, :U][fe]
            err = np.abs(gv - ov) / s
            st[f"{k}_max_rel"] = float(err.max()) if err.size else 0.0
            assert st[f"{k}_max_rel"] <= TOL
            if sound_bounds:
                viol = (gv - ov) / s if k == "l" else (ov - gv) / s
                assert viol.size == 0 or viol.max() <= SOUND, (k, viol.max())
        # masks: exact except in the tolerance band, where only the conservative (unstable) call is allowed
        mg, mo = g["mask"][:, :U], o["mask"][:, :U]
        diff = (mg != mo)
        st["mask_mismatch"] = int(diff.sum())
        if diff.any():
            bi, ci = np.nonzero(diff)
            for b, c in zip(bi, ci):
                assert mg[b, c] == 0, "GPU took a non-conservative stability decision"
                band = TOL * max(o["l_scale"][b, c], o["u_scale"][b, c])
                assert min(abs(o["l"][b, c]), abs(o["u"][b, c])) <= band
        assert st["mask_mismatch"] <= max(2, mg.size // 10000)
    # spec bounds
    lg, lo_, ls = g["lower"][fe], o["lower"][fe], o["lower_scale"][fe]
    err = np.abs(lg - lo_) / ls
    st["lower_max_rel"] = float(err.max()) if err.size else 0.0
    st["lower_med_rel"] = float(np.median(err)) if err.size else 0.0
    st["lower_max_rel_to_value"] = float(np.max(np.abs(lg - lo_) / np.maximum(np.abs(lo_), 1e-30))) if err.size else 0.0
    assert st["lower_max_rel"] <= TOL, st
    if sound_bounds:
        assert np.all(lg <= lo_ + SOUND * ls)
    assert np.all(np.isinf(g["lower"][inf_o]))
    # verified: exact except rows within the band of 0
    vg, vo = g["verified"].astype(bool), o["verified"].astype(bool)
    for b in np.nonzero(vg != vo)[0]:
        assert not vg[b] and vo[b]
        assert np.min(np.abs(o["lower"][b]) / o["lower_scale"][b]) <= TOL
    if report is not None:
        report.update(st)
    print(st)
    return st


def test_paper_toy_example_on_gpu():
    import json, os
    from fractions import Fraction
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_2d.json")))
    layers = [dict(kind=0, W=np.array(gold["W1"], np.float32), b=np.array(gold["b1"], np.float32),
                   in_shape=(2,), out_shape=(2,)),
              dict(kind=0, W=np.array([gold["w2"]], np.float32), b=np.array(gold["b2"], np.float32),
                   in_shape=(2,), out_shape=(1,))]
    case = Case(None, 1, 0, 0, 0.0, layers=layers, m_spec=(np.array([[1.0]], np.float32), np.zeros(1, np.float32)),
                alpha_mode=1, enforce=0)
    case.lo = np.array([gold["box_lo"]], np.float32)
    case.hi = np.array([gold["box_hi"]], np.float32)
    case.lo0, case.hi0 = case.lo[0], case.hi[0]
    from oracle import oracle as O
    root = O.root_crown(case.net, case.lo0, case.hi0, alpha_mode=1)
    case.cache = O.make_cache(root)
    case.U = 2
    case.split_off, case.split_ids, case.max_splits = np.array([0, 1], np.int32), np.array([-1], np.int32), 1
    # relaxed clipping: bound -2, box [-1,1] x [5/7,1]
    case.relaxed, case.sweeps = 1, 0
    g = gpu_round(case)
    o = case.oracle()
    tol = TOL * o["lower_scale"][0, 0]
    assert o["lower"][0, 0] == pytest.approx(-2.0, abs=1e-6)
    assert -2.0 - tol <= g["lower"][0, 0] <= -2.0
    assert g["hi_clip"][0, 0] >= 1.0 and g["hi_clip"][0, 0] - 1.0 < 1e-6
    assert g["lo_clip"][0, 1] <= 5 / 7 and 5 / 7 - g["lo_clip"][0, 1] < 1e-6
    compare(case, g, o)
    # complete clipping on the original box: zbar_2 = -3 under z1 <= 0 and the output bound 0.
    # The split neuron is clamped to its side (standard activation BaB); its clipped upper bound is
    # exactly 0 in the walk-through, a tie no padded FP32 bound can certify.
    case.relaxed, case.sweeps, case.enforce = 0, 1, 1
    g = gpu_round(case)
    o = case.oracle()
    assert np.array_equal(o["u"][0], [0.0, -3.0]) and o["lower"][0, 0] == 0.0
    assert g["u"][0, 0] == 0.0
    assert -3.0 <= g["u"][0, 1] <= -3.0 + TOL * o["u_scale"][0, 1]
    assert -TOL * o["lower_scale"][0, 0] <= g["lower"][0, 0] <= 0.0
    compare(case, g, o)


@pytest.mark.parametrize("name,kw", [
    ("mlp5x50_relaxed", dict(dims=[5] + [50] * 6 + [5], B=256, kmin=0, kmax=8, eps=0.05, centre="pm1",
                             clip01=False, out_rows=1, sweeps=0)),
    ("mlp5x50_complete", dict(dims=[5] + [50] * 6 + [5], B=64, kmin=1, kmax=8, eps=0.05, centre="pm1",
                              clip01=False, out_rows=0, sweeps=10)),
    ("mlp24_complete", dict(dims=[24, 32, 32, 32, 6], B=48, kmin=1, kmax=4, eps=0.1, sweeps=10)),
    ("mlp784_ragged", dict(dims=[784, 70, 70, 10], B=37, kmin=1, kmax=4, eps=0.02, sweeps=10)),
    ("mlp784_targets", dict(dims=[784, 64, 64, 10], B=20, kmin=1, kmax=4, eps=0.02, sweeps=3, targets=7)),
    ("mlp100_no_splits", dict(dims=[100, 40, 40, 7], B=9, kmin=0, kmax=0, eps=0.05, sweeps=5)),
    ("mlp32_many_rows", dict(dims=[32, 40, 40, 6], B=40, kmin=0, kmax=2, eps=0.1, sweeps=6, cut_rows=(0, 6))),
    ("mlp32_up_to_26_rows", dict(dims=[32, 40, 40, 6], B=24, kmin=0, kmax=2, eps=0.1, sweeps=4, cut_rows=(6, 24))),
])
def test_round_parity(name, kw):
    case = Case(**kw)
    g = gpu_round(case)
    o = case.oracle()
    compare(case, g, o)


@pytest.mark.parametrize("name,kw", [
    ("mlp5x50_relaxed", dict(dims=[5] + [50] * 6 + [5], B=256, kmin=0, kmax=8, eps=0.05, centre="pm1",
                             clip01=False, out_rows=1, sweeps=0)),
    ("mlp24_complete", dict(dims=[24, 32, 32, 32, 6], B=48, kmin=1, kmax=4, eps=0.1, sweeps=10)),
    ("mlp784_ragged", dict(dims=[784, 70, 70, 10], B=37, kmin=1, kmax=4, eps=0.02, sweeps=10)),
    ("mlp784_targets", dict(dims=[784, 64, 64, 10], B=20, kmin=1, kmax=4, eps=0.02, sweeps=3, targets=7)),
    ("mlp100_wide", dict(dims=[100, 300, 500, 7], B=11, kmin=1, kmax=3, eps=0.05, sweeps=3)),
])
def test_round_parity_tensor_core(name, kw):
    """The split-BF16 tensor-core back-substitution (CV_PREC_BF16X8) against the same oracle, at
    the same bar; K in (0, 512] covers one and two exact accumulator sets and ragged tiles."""
    from paper_2512_11087_gb300 import capi
    case = Case(**kw)
    g = gpu_round(case, precision=capi.CV_PREC_BF16X8)
    o = case.oracle()
    compare(case, g, o)


@pytest.mark.parametrize("name,kw", [
    ("k600_three_chunks", dict(dims=[20, 600, 5], B=12, kmin=1, kmax=2, eps=0.1, sweeps=2)),
    ("k1024_two_passes", dict(dims=[64, 1024, 1024, 10], B=10, kmin=1, kmax=3, eps=0.05, sweeps=2)),
    ("k1300_three_passes", dict(dims=[30, 1300, 200, 7], B=9, kmin=0, kmax=3, eps=0.05, sweeps=3)),
])
def test_round_parity_tensor_core_wide_layers(name, kw):
    """Layers with more than 512 outputs on the tensor cores: K in passes of two exact accumulator
    sets, the chunk sums of all but the last pass carried in shared memory (one, two and three passes;
    a last pass with one chunk)."""
    from paper_2512_11087_gb300 import capi
    case = Case(**kw)
    g = gpu_round(case, precision=capi.CV_PREC_BF16X8)
    o = case.oracle()
    compare(case, g, o)


@pytest.mark.parametrize("precision", [0, 1])
def test_round_parity_alpha_given(precision):
    case = Case([30, 40, 40, 5], 16, 0, 3, 0.1, sweeps=0, seed=4)
    rng = np.random.default_rng(9)
    alpha = rng.uniform(0, 1, size=(case.B, case.m, case.net.H)).astype(np.float32)
    from paper_2512_11087_gb300 import engine as E
    g = gpu_round(case, precision=precision, alpha=E.to_dev(alpha))
    o = case.oracle(alpha=alpha.astype(np.float64))
    compare(case, g, o)


def test_infeasible_and_edge_cases():
    # (1) a split on a root-stable neuron against its sign; (2) an extra row that no point of the
    # box satisfies; (3) a subdomain without rows.  Both sides must flag exactly (1) and (2).
    case = Case([12, 20, 20, 4], 6, 1, 2, 0.3, sweeps=4, seed=3, out_rows=1)
    stable = np.nonzero(case.cache["root_l"] >= 0)[0]
    assert stable.size > 0
    so, si = case.split_off.copy(), case.split_ids.copy()
    si[so[0]] = -(int(stable[0]) + 1)          # z <= 0 on a neuron that is always active
    case.split_ids = si
    case.h = case.h.copy()
    case.h[1] = 1e6                            # row 1 (subdomain 1): g.x + 1e6 <= 0 is empty
    so2 = so.copy()
    case.split_off = so2
    g = gpu_round(case)
    o = case.oracle()
    assert o["infeasible"][0] == 1 and o["infeasible"][1] == 1
    assert np.all(np.isinf(g["lower"][:2])) and np.all(g["verified"][:2] == 1)
    compare(case, g, o, sound_bounds=False)


def test_cache_build_parity():
    """a1 on the GPU (cv_cache_build) against the oracle's root CROWN: bounds within 1e-5 of the
    back-substitution magnitude scale, never tighter, same unstable set (outside the band)."""
    from oracle import oracle as O
    from paper_2512_11087_gb300 import engine as E, workloads as WL
    for dims, eps, seed in [([24, 32, 32, 32, 6], 0.1, 0), ([784, 256, 256, 256, 256, 256, 256, 10], 0.02, 0),
                            ([5] + [50] * 6 + [5], 0.05, 1)]:
        layers = WL.he_mlp(dims, seed=seed)
        lo0, hi0 = WL.box(dims[0], eps, seed=seed, centre="unit" if dims[0] > 5 else "pm1", clip01=dims[0] > 5)
        net = E.Net(layers)
        U = net.build_cache(lo0, hi0)
        gc = net.read_cache()
        root = O.root_crown(O.Net(layers), lo0, hi0)
        bs = root["bscale"]
        el = (root["l"] - gc["root_l"]) / bs
        eu = (gc["root_u"] - root["u"]) / bs
        print(dims[0], len(dims), "max rel l %.2e u %.2e" % (el.max(), eu.max()))
        assert el.min() >= -1e-12 and eu.min() >= -1e-12
        assert el.max() <= TOL and eu.max() <= TOL
        unst_o = (root["l"] < 0) & (root["u"] > 0)
        unst_g = np.zeros_like(unst_o)
        unst_g[gc["ids"]] = True
        diff = np.nonzero(unst_o != unst_g)[0]
        for g_ in diff:  # only conservative calls inside the band
            assert unst_g[g_] and min(abs(root["l"][g_]), abs(root["u"][g_])) <= TOL * bs[g_]
        assert U == unst_g.sum()
        # the cached planes are valid: sampled points satisfy them
        rng = np.random.default_rng(0)
        X = lo0 + (hi0 - lo0) * rng.uniform(size=(2000, dims[0]))
        _, pre = O.Net(layers).forward(X)
        Z = np.concatenate(pre, axis=1)[:, gc["ids"]]
        assert np.all(Z >= X @ gc["lA"].T.astype(np.float64) + gc["lc"] - 1e-9)
        assert np.all(Z <= X @ gc["uA"].T.astype(np.float64) + gc["uc"] + 1e-9)
        net.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_call(precision):
    """A captured round (cv_graph_capture / cv_graph_launch) reads its buffers at replay time and
    gives the same outputs as a direct cv_bound_batch call (both precisions: the tensor-core path
    encodes its TMA descriptors on the host during capture)."""
    from paper_2512_11087_gb300 import engine as E
    case = Case([24, 32, 32, 32, 6], 32, 1, 4, 0.1, sweeps=5, seed=2)
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, sweeps=case.sweeps, precision=precision)
    d = E.to_dev
    lo, hi = d(case.lo), d(case.hi)
    args = (d(case.C), d(case.t))
    so, si = d(case.split_off), d(case.split_ids)
    direct = {k: v.clone() for k, v in rnd.run(lo, hi, *args, split_off=so, split_ids=si).items()}
    # capture on scratch data, then write the real inputs and replay
    lo_s, hi_s = lo.clone(), hi.clone()
    lo.zero_(); hi.fill_(1.0)
    rnd.capture(lo, hi, *args, split_off=so, split_ids=si)
    lo.copy_(lo_s); hi.copy_(hi_s)
    for k in rnd.out:
        rnd.out[k].zero_()
    out = rnd.replay()
    torch.cuda.synchronize()
    for k in direct:
        assert torch.equal(direct[k], out[k]), k
    from paper_2512_11087_gb300 import capi
    capi.cv_graph_destroy(rnd.graph)
    net.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_cnn_round_parity(precision):
    """A small CIFAR-shaped CNN (two strided 4x4 convolutions, a 3x3 one, two dense layers): the
    conv layers are expanded to matrices independently on both sides; on both paths (the first
    layer has 864 outputs: two tensor-core passes)."""
    from paper_2512_11087_gb300 import workloads as WL
    layers = WL.he_cnn((3, 12, 12), [(6, 4, 2, 1), (8, 4, 2, 1), (8, 3, 1, 1)], [20, 10], seed=4)
    case = Case(None, 24, 1, 6, 2.0 / 255.0, layers=layers, sweeps=4, seed=4)
    g = gpu_round(case, precision=precision)
    o = case.oracle()
    compare(case, g, o)


@pytest.mark.parametrize("precision", [1, 0])
def test_bench_workload_full_size_sampled(precision):
    """The benchmark's launch configuration: 784->256x6->10, 4096 subdomains with 1-4 splits,
    relaxed + complete clipping with 10 sweeps, split-precision tensor-core path (the bench's
    default) and the plain FP32 path.  The GPU bounds all subdomains; the oracle bounds a sample."""
    from paper_2512_11087_gb300 import workloads as WL
    cfg = WL.CONFIGS["mlp784x256"]
    case = Case(cfg["dims"], cfg["B"], cfg["kmin"], cfg["kmax"], cfg["eps"], sweeps=cfg["sweeps"], seed=0)
    g = gpu_round(case, precision=precision)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([rng.choice(case.B, 254, replace=False), [0, case.B - 1]]))
    sub = Case.__new__(Case)
    sub.__dict__.update(case.__dict__)
    sub.B = sample.size
    sub.lo, sub.hi = case.lo[sample], case.hi[sample]
    so = np.zeros(sample.size + 1, np.int32)
    ids = []
    for i, b in enumerate(sample):
        seg = case.split_ids[case.split_off[b]:case.split_off[b + 1]]
        ids.append(seg)
        so[i + 1] = so[i] + seg.size
    sub.split_off, sub.split_ids = so, np.concatenate(ids).astype(np.int32)
    o = sub.oracle(nthreads=0)
    gs = {k: v[sample] for k, v in g.items()}
    st = compare(sub, gs, o)
    print("full-size sampled parity", st)


def test_round_summary_of_a_round():
    # cv_round_summary against its definition on the round's own outputs, and its counts against the oracle's
    from paper_2512_11087_gb300 import engine as E, workloads as WL
    C, t = WL.margin_spec(4)
    # the threshold puts the verified / unverified cut between two of the oracle's bounds 3e-3 apart
    case = Case([16, 32, 32, 4], 300, 1, 3, 0.12, seed=41, sweeps=2, out_rows=1, m_spec=(C, t + 3.691))
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, max_rows=case.max_rows, sweeps=case.sweeps)
    d = E.to_dev
    out = rnd.run(d(case.lo), d(case.hi), d(case.C), d(case.t), split_off=d(case.split_off),
                  split_ids=d(case.split_ids), row_off=d(case.row_off), G=d(case.G), h=d(case.h))
    s = E.reduce_round_summary(*E.round_summary(out))
    g = {k: v.cpu().numpy() for k, v in out.items()}
    feas = g["infeasible"] == 0
    lm = g["lower"].min(axis=1)
    assert s["infeasible"] == int((~feas).sum()) and s["verified"] == int((feas & (g["verified"] == 1)).sum())
    assert s["lower_min"] == (float(lm[feas].min()) if feas.any() else float("inf"))
    unv = feas & (g["verified"] == 0)
    assert s["lower_min_unverified"] == (float(lm[unv].min()) if unv.any() else float("inf"))
    o = case.oracle()
    ofeas = o["infeasible"] == 0
    assert s["infeasible"] == int((~ofeas).sum()) and s["verified"] == int((ofeas & (o["verified"] == 1)).sum())
    assert 0 < s["infeasible"] and 0 < s["verified"] < case.B - s["infeasible"]
    net.close()


@pytest.mark.parametrize("n0,extra", [(200, 1), (600, 1), (200, 4), (600, 4)])
def test_complete_clipping_exact_ties_over_the_candidate_limit(n0, extra):
    """Every breakpoint of a row step exactly tied.

    The first hidden neuron's plane is all ones and the first row is g = -1 (sum x >= the box
    centre's sum, less a slack), so on that row's first step every element's breakpoint is exactly
    1: every element is a candidate of the certification, more than its list holds. The over-limit
    search bisects on the candidates' stored ordinals. Their ties fit the list (n0 = 200) or exceed
    it (n0 = 600: the counts recomputed from the rows). With 1 random row besides, the main launch
    runs; with 4, the wide launch. Against the oracle's FP64 Algorithm 1; the search must have run."""
    from paper_2512_11087_gb300 import workloads as WL
    dims = [n0, 4, 3]
    layers = WL.he_mlp(dims, seed=41)
    lo0, hi0 = WL.box(n0, 0.05, seed=41, centre="unit", clip01=True)
    xh = 0.5 * (lo0.astype(np.float64) + hi0.astype(np.float64))
    ep = 0.5 * (hi0.astype(np.float64) - lo0.astype(np.float64))
    layers[0]["W"][0, :] = 1.0
    layers[0]["b"][0] = np.float32(-xh.sum())
    case = Case(dims, 2, 0, 0, 0.05, seed=41, layers=layers, sweeps=3, relaxed=0)
    assert np.array_equal(case.lo0, lo0) and np.array_equal(case.hi0, hi0)
    off, Gr, hr = WL.random_cut_rows(case.lo, case.hi, case.B, extra, extra, seed=43)
    G = np.empty((case.B * (extra + 1), n0), np.float32)
    h = np.empty(case.B * (extra + 1), np.float32)
    for b in range(case.B):
        G[b * (extra + 1)] = -1.0
        h[b * (extra + 1)] = np.float32(xh.sum() - 0.3 * ep.sum())
        G[b * (extra + 1) + 1:(b + 1) * (extra + 1)] = Gr[off[b]:off[b + 1]]
        h[b * (extra + 1) + 1:(b + 1) * (extra + 1)] = hr[off[b]:off[b + 1]]
    case.row_off = np.arange(0, case.B * (extra + 1) + 1, extra + 1, dtype=np.int32)
    case.G, case.h, case.max_rows = G, h, extra + 1
    g = gpu_round(case)
    o = case.oracle()
    compare(case, g, o)
    assert LAST_CC_STATS[5] > 0, LAST_CC_STATS  # the over-limit search ran
