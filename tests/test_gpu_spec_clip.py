"""Complete clipping of the spec rows' final planes (cv_spec_clip) through the C-ABI.

Parity: the oracle runs its own round with final planes (FP64 CROWN, its clipped box) and applies
its FP64 Algorithm 1 (complete_clip) to every spec row it leaves unproven, over that plane, box and
the subdomain's active rows; the GPU's round followed by cv_spec_clip must lie within 1e-5 of the
oracle's scale and never above it (beyond the oracle's own rounding).  Rows the GPU had already
proven stay bit for bit, and verified follows the new bounds.  No oracle input comes from the GPU.
Soundness: on a small network the new bounds hold at sampled feasible points."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5
SOUND = 1e-12


def _run(case):
    from paper_2512_11087_gb300 import engine as E
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, max_rows=case.max_rows, sweeps=case.sweeps,
                  want_final=True)
    d = E.to_dev
    args = (d(case.lo), d(case.hi), d(case.C), d(case.t))
    kw = dict(split_off=d(case.split_off), split_ids=d(case.split_ids), row_off=d(case.row_off), G=d(case.G),
              h=d(case.h))
    out = rnd.run(*args, **kw)
    torch.cuda.synchronize()
    before = {k: v.cpu().numpy().copy() for k, v in out.items()}
    rnd.spec_clip(*args, **kw)
    torch.cuda.synchronize()
    after = {k: v.cpu().numpy().copy() for k, v in out.items()}
    from paper_2512_11087_gb300 import capi
    assert capi.cv_device_status(net.handle) == 0
    net.close()
    return before, after


def _active_rows(case, b):
    """The subdomain's rows (splits as cached FP32 planes, then extra rows) that the pre-check keeps on
    the input box, in order."""
    from oracle import oracle as O
    c = case.cache
    slot = {int(g): i for i, g in enumerate(c["ids"])}
    G, h = [], []
    for code in case.split_ids[case.split_off[b]:case.split_off[b + 1]]:
        g = abs(int(code)) - 1
        if g not in slot:
            continue
        s = slot[g]
        if code > 0:
            G.append(-f32(c["uA"][s]).astype(np.float64)); h.append(-float(f32(c["uc"][s])))
        else:
            G.append(f32(c["lA"][s]).astype(np.float64)); h.append(float(f32(c["lc"][s])))
    if case.row_off is not None:
        for r in range(case.row_off[b], case.row_off[b + 1]):
            G.append(case.G[r].astype(np.float64)); h.append(float(case.h[r]))
    keep = [k for k in range(len(h)) if O.row_check(G[k], h[k], case.lo[b], case.hi[b])[0] == 0]
    return np.array([G[k] for k in keep]).reshape(len(keep), case.n0), np.array([h[k] for k in keep])


@pytest.mark.parametrize("kw", [
    dict(dims=[32, 40, 40, 6], B=40, kmin=1, kmax=3, eps=0.1, sweeps=6, cut_rows=(0, 4), seed=11),
    dict(dims=[24, 32, 32, 5], B=24, kmin=0, kmax=2, eps=0.1, sweeps=4, cut_rows=(5, 12), seed=12),
])
def test_spec_clip_parity(kw):
    from oracle import oracle as O
    case = Case(**kw)
    g0, g1 = _run(case)
    o = case.oracle(want_final=True)
    raised = 0
    assert np.array_equal(g0["infeasible"], o["infeasible"])
    for b in range(case.B):
        if g0["infeasible"][b]:
            assert np.array_equal(g1["lower"][b].view(np.uint32), g0["lower"][b].view(np.uint32))
            continue
        G, h = _active_rows(case, b)
        for r in range(case.m):
            l0, l1 = float(g0["lower"][b, r]), float(g1["lower"][b, r])
            if l0 > 0 or h.size == 0:
                assert np.float32(l1).view(np.uint32) == np.float32(l0).view(np.uint32)
                continue
            # the oracle's own plane and box
            v, _, sc = O.complete_clip(o["final_A"][b, r], float(o["final_c"][b, r]), G, h, o["lo_clip"][b],
                                       o["hi_clip"][b], case.sweeps)
            want = max(float(o["lower"][b, r]), v)
            sc = max(sc, float(o["lower_scale"][b, r]))
            assert l1 >= l0
            assert l1 <= want + SOUND * sc, (b, r, l1, want)
            assert abs(l1 - want) <= TOL * sc, (b, r, l1, want, sc)
            raised += l1 > l0
    assert raised > 0
    ver = g1["infeasible"].astype(bool) | np.all(g1["lower"] > 0, axis=1)
    assert np.array_equal(g1["verified"].astype(bool), ver)


def test_spec_clip_is_sound_at_feasible_points():
    from oracle import oracle as O
    case = Case([4, 16, 16, 3], 16, 2, 4, 0.5, sweeps=10, seed=13, centre="pm1", clip01=False)
    g0, g1 = _run(case)
    rng = np.random.default_rng(14)
    net = O.Net(case.layers)
    for b in range(case.B):
        X = rng.uniform(case.lo[b], case.hi[b], size=(20000, 4))
        G, h = _active_rows(case, b)
        feas = np.all(X @ G.T + h <= 0, axis=1) if h.size else np.ones(len(X), bool)
        if g1["infeasible"][b] or not feas.any():
            continue
        z = X[feas].astype(np.float64)
        for i, (W, bb) in enumerate(zip(net.Ws, net.bs)):
            z = z @ W.T + bb
            if i < len(net.Ws) - 1:
                z = np.maximum(z, 0.0)
        F = z @ case.C.T.astype(np.float64) - case.t
        assert np.all(g1["lower"][b] <= F.min(axis=0) + 1e-6)
