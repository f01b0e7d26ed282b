"""The slope gradient (cv_alpha_grad) and Adam step (cv_alpha_adam) against the FP64 oracle.

Both sides get the same network, box, per-subdomain bounds (FP32 values) and slopes.  The bound
f must match the oracle within 1e-5 of its magnitude scale and never be tighter; the gradient is
FP32 without a pad and must match the oracle's FP64 reverse sweep within 1e-4 of the largest
gradient of its spec row; a directional finite difference of the GPU bound itself agrees with
the GPU gradient; Adam matches the oracle's step; 20 Adam steps raise the bounds."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2512_11087_gb300 import workloads as WL  # noqa: E402
from tests._cases import f32, rd32, ru32  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(dims, B, seed, eps=0.1):
    from paper_2512_11087_gb300 import engine as E
    layers = WL.he_mlp(dims, seed=seed)
    onet = O.Net(layers)
    lo0, hi0 = WL.box(dims[0], eps, seed=seed, clip01=True)
    root = O.root_crown(onet, lo0, hi0)
    cache = O.make_cache(root)
    rl, ru = rd32(root["l"]), ru32(root["u"])
    net = E.Net(layers)
    net.set_cache(f32(lo0), f32(hi0), rl, ru, cache["ids"], f32(cache["lA"]), f32(cache["lc"]), f32(cache["uA"]),
                  f32(cache["uc"]))
    rng = np.random.default_rng(seed)
    ids = cache["ids"]
    U = ids.size
    # per-subdomain bounds: root bounds of the cached neurons, tightened at random
    l = np.tile(rl[ids], (B, 1)).astype(np.float64)
    u = np.tile(ru[ids], (B, 1)).astype(np.float64)
    shrink = rng.uniform(0.0, 0.6, size=(B, U))
    side = rng.uniform(size=(B, U)) < 0.5
    l = np.where(side, l + shrink * (u - l) * 0.5, l)
    u = np.where(~side, u - shrink * (u - l) * 0.5, u)
    l, u = rd32(l), ru32(u)
    mask = np.where(l >= 0, 1, np.where(u <= 0, -1, 0)).astype(np.int8)
    C, t = WL.margin_spec(dims[-1], y=0)
    m = C.shape[0]
    alpha = rng.uniform(0, 1, size=(B, m, onet.H)).astype(np.float32)
    lo, hi = WL.tile_box(lo0, hi0, B)
    return dict(net=net, onet=onet, root=root, ids=ids, rl=rl, ru=ru, l=l, u=u, mask=mask, C=C, t=t, alpha=alpha,
                lo=lo, hi=hi, B=B, m=m, cache=cache)


def _full_bounds(s, b):
    hl = s["rl"].astype(np.float64).copy()
    hu = s["ru"].astype(np.float64).copy()
    hs = np.where(hl >= 0, 1, np.where(hu <= 0, -1, 0)).astype(np.int8)
    hl[s["ids"]] = s["l"][b]
    hu[s["ids"]] = s["u"][b]
    hs[s["ids"]] = s["mask"][b]
    return hl, hu, hs


def _state(s, precision=0):
    from paper_2512_11087_gb300 import engine as E
    d = E.to_dev
    return E.AlphaState(s["net"], d(s["lo"]), d(s["hi"]), d(s["l"]), d(s["u"]), d(s["mask"]), d(s["C"]), d(s["t"]),
                        precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dims,B,seed", [([30, 40, 40, 40, 5], 6, 1), ([784, 96, 96, 10], 5, 2),
                                         ([5] + [50] * 6 + [5], 4, 3), ([40, 600, 300, 6], 5, 4)])
def test_alpha_gradient_parity(dims, B, seed, precision):
    """FP32 CUDA-core contractions and the split-BF16 tensor-core forward and reverse sweep (the
    last network has a 600-wide layer: several K passes both ways)."""
    from paper_2512_11087_gb300 import engine as E
    s = _setup(dims, B, seed, eps=0.05 if dims[0] > 5 else 0.1)
    st = _state(s, precision)
    rng = np.random.default_rng(seed + 10)
    gf = rng.uniform(0.5, 1.5, size=(B, s["m"])).astype(np.float32)
    lower, grad = st.bound_and_grad(E.to_dev(s["alpha"]), E.to_dev(gf))
    lower, grad = lower.cpu().numpy(), grad.cpu().numpy()
    # scales of the bounds from the oracle's round with the same bounds and slopes (no clipping)
    o = O.bound_batch(s["onet"], s["cache"] | dict(root_l=s["rl"].astype(np.float64), root_u=s["ru"].astype(np.float64)),
                      s["lo"], s["hi"], l_in=s["l"], u_in=s["u"], C=s["C"], t=s["t"],
                      alpha=s["alpha"].astype(np.float64), relaxed=0, sweeps=0)
    worst = 0.0
    for b in range(B):
        hl, hu, hs = _full_bounds(s, b)
        f, g = O.alpha_grad(s["onet"], hl, hu, hs, s["lo"][b], s["hi"][b], s["C"], s["t"],
                            s["alpha"][b].astype(np.float64), gf[b].astype(np.float64))
        np.testing.assert_allclose(f, o["lower"][b], rtol=0, atol=1e-9 * np.max(o["lower_scale"][b]))
        sc = o["lower_scale"][b]
        assert np.all(lower[b] <= f + 1e-12 * sc)
        assert np.all(np.abs(lower[b] - f) <= 1e-5 * sc)
        for r in range(s["m"]):
            gmax = np.max(np.abs(g[r]))
            if gmax == 0:
                assert np.all(grad[b, r] == 0)
                continue
            err = np.max(np.abs(grad[b, r] - g[r])) / gmax
            worst = max(worst, err)
            assert err <= 1e-4, (b, r, err)
    print("max gradient error / row max", worst)
    s["net"].close()


def test_alpha_autograd_and_finite_difference():
    from paper_2512_11087_gb300 import engine as E
    s = _setup([30, 40, 40, 40, 5], 3, 5)
    st = _state(s)
    alpha = E.to_dev(s["alpha"]).requires_grad_(True)
    lower = E.AlphaBound.apply(alpha, st)
    gen = torch.Generator(device=alpha.device).manual_seed(11)
    w = torch.rand(lower.shape, generator=gen, device=alpha.device)
    (lower * w).sum().backward()
    _, g1 = st.bound_and_grad(alpha.detach())
    assert torch.allclose(alpha.grad, g1 * w.unsqueeze(-1))
    # directional derivative of the GPU bound along a random direction (f is affine in each slope
    # while no relaxation choice flips; a small step keeps the choices, and slopes near 0 or 1 are
    # left out of the direction so that the clamp to [0, 1] does not cut the step)
    h = 1e-3
    inner = (alpha.detach() > 0.01) & (alpha.detach() < 0.99)
    v = torch.randn(alpha.shape, generator=gen, device=alpha.device) * (alpha.grad != 0) * inner
    fp, _ = st.bound_and_grad((alpha.detach() + h * v).clamp(0, 1))
    fm, _ = st.bound_and_grad((alpha.detach() - h * v).clamp(0, 1))
    fd = ((fp - fm) * w).sum().item() / (2 * h)
    an = (alpha.grad * v).sum().item()
    assert fd == pytest.approx(an, rel=2e-2, abs=1e-3 * max(1.0, abs(an)))
    s["net"].close()


def test_adam_step_matches_oracle_and_optimisation_improves():
    from paper_2512_11087_gb300 import capi, engine as E
    rng = np.random.default_rng(3)
    n = 4096
    a0 = rng.uniform(0, 1, n)
    g = rng.normal(size=n)
    m1, m2 = np.zeros(n), np.zeros(n)
    ao = a0.copy()
    O.adam_step(ao, m1, m2, g, t=1, lr=0.1)
    O.adam_step(ao, m1, m2, 0.5 * g, t=2, lr=0.098)
    ag = E.to_dev(a0.astype(np.float32)); gm1 = torch.zeros_like(ag); gm2 = torch.zeros_like(ag)
    capi.cv_alpha_adam(ag, gm1, gm2, E.to_dev(g.astype(np.float32)), 1, 0.1)
    capi.cv_alpha_adam(ag, gm1, gm2, E.to_dev((0.5 * g).astype(np.float32)), 2, 0.098)
    assert np.allclose(ag.cpu().numpy(), ao, atol=2e-6)
    # 20 steps on a 784 -> 1024x4 -> 10 shaped problem (reduced batch): the bound goes up
    s = _setup([784, 1024, 1024, 1024, 1024, 10], 4, 7, eps=0.02)
    st = _state(s)
    alpha0 = torch.where(E.to_dev(s["u"]).new_ones(1).bool(), E.to_dev(s["alpha"]), E.to_dev(s["alpha"]))
    _, hist = E.optimize_alpha(st, alpha0, steps=20)
    first, last = hist[0].cpu().numpy(), hist[-1].cpu().numpy()
    print("mean bound before / after 20 Adam steps:", first.mean(), last.mean())
    assert last.mean() > first.mean()
    s["net"].close()


def _split_setup(dims, B, seed, eps=0.05):
    """A batch whose subdomains hold 1-3 splits each, enforced on the split neurons' bounds, with
    random split multipliers beta >= 0."""
    s = _setup(dims, B, seed, eps=eps)
    so, si = WL.draw_splits(s["ids"], B, 1, 3, seed=seed + 5)
    H = s["onet"].H
    bsign = np.zeros((B, H), np.int8)
    slot = {int(g): c for c, g in enumerate(s["ids"])}
    for b in range(B):
        for code in si[so[b]:so[b + 1]]:
            g = abs(int(code)) - 1
            bsign[b, g] = 1 if code > 0 else -1
            c = slot[g]
            if code > 0: s["l"][b, c] = max(s["l"][b, c], 0.0)
            else: s["u"][b, c] = min(s["u"][b, c], 0.0)
    s["mask"] = np.where(s["l"] >= 0, 1, np.where(s["u"] <= 0, -1, 0)).astype(np.int8)
    rng = np.random.default_rng(seed + 6)
    s["beta"] = (rng.uniform(0, 0.5, size=(B, s["m"], H)) * (bsign[:, None, :] != 0)).astype(np.float32)
    s["bsign"], s["so"], s["si"] = bsign, so, si
    return s


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dims,B,seed", [([30, 40, 40, 40, 5], 6, 21), ([784, 96, 96, 10], 5, 22)])
def test_split_multiplier_bound_and_gradient_parity(dims, B, seed, precision):
    """Split multipliers (beta-CROWN form of the split constraints): the bound and d/d beta against the
    oracle's FP64 back-substitution and reverse sweep; the split signs from the CSR exactly."""
    from paper_2512_11087_gb300 import engine as E
    s = _split_setup(dims, B, seed)
    d = E.to_dev
    sign = E.split_signs(s["net"], d(s["so"]), d(s["si"]), B)
    torch.cuda.synchronize()
    assert np.array_equal(sign.cpu().numpy(), s["bsign"])
    st = E.AlphaState(s["net"], d(s["lo"]), d(s["hi"]), d(s["l"]), d(s["u"]), d(s["mask"]), d(s["C"]), d(s["t"]),
                      precision=precision, split_sign=sign)
    lower, grad, gb = st.bound_and_grad(d(s["alpha"]), beta=d(s["beta"]))
    lower, grad, gb = lower.cpu().numpy(), grad.cpu().numpy(), gb.cpu().numpy()
    worst = 0.0
    for b in range(B):
        hl, hu, hs = _full_bounds(s, b)
        # the magnitude scale of the bounds with the multipliers, over the root magnitudes (as the
        # round's lower_scale)
        zm = np.maximum(np.abs(s["rl"]), np.abs(s["ru"])).astype(np.float64)
        f, g, gbo, sc = O.alpha_grad(s["onet"], hl, hu, hs, s["lo"][b], s["hi"][b], s["C"], s["t"],
                                     s["alpha"][b].astype(np.float64), beta=s["beta"][b].astype(np.float64),
                                     bsign=s["bsign"][b], zmag=zm, want_scale=True)
        assert np.all(lower[b] <= f + 1e-12 * sc)
        assert np.all(np.abs(lower[b] - f) <= 1e-5 * sc), (b, lower[b] - f, sc)
        assert np.all(gb[b][:, s["bsign"][b] == 0] == 0)
        for r in range(s["m"]):
            gmax = np.max(np.abs(gbo[r]))
            if gmax == 0:
                continue
            err = np.max(np.abs(gb[b, r] - gbo[r])) / gmax
            worst = max(worst, err)
            assert err <= 1e-4, (b, r, err)
    print("max d/d beta error / row max", worst)
    s["net"].close()


@pytest.mark.parametrize("precision", [0, 1])
def test_split_multipliers_raise_the_bound_and_stay_sound(precision):
    from paper_2512_11087_gb300 import engine as E
    s = _split_setup([30, 40, 40, 40, 5], 8, 23)
    d = E.to_dev
    sign = E.split_signs(s["net"], d(s["so"]), d(s["si"]), s["B"])
    st = E.AlphaState(s["net"], d(s["lo"]), d(s["hi"]), d(s["l"]), d(s["u"]), d(s["mask"]), d(s["C"]), d(s["t"]),
                      precision=precision, split_sign=sign)
    a0 = d(s["alpha"])
    b0 = torch.zeros(s["B"], s["m"], s["onet"].H, dtype=torch.float32, device="cuda")
    al, bt, hist = E.optimize_alpha(st, a0, steps=15, beta=b0, beta_lr=0.05)
    torch.cuda.synchronize()
    first, last = hist[0].cpu().numpy(), hist[-1].cpu().numpy()
    assert np.mean(last) > np.mean(first)
    bt = bt.cpu().numpy()
    assert np.all(bt >= 0) and np.any(bt > 0)
    al = al.cpu().numpy()
    for b in range(s["B"]):
        hl, hu, hs = _full_bounds(s, b)
        f = O.alpha_grad(s["onet"], hl, hu, hs, s["lo"][b], s["hi"][b], s["C"], s["t"], al[b].astype(np.float64),
                         beta=bt[b].astype(np.float64), bsign=s["bsign"][b])[0]
        assert np.all(last[b] <= f + 1e-9 * (1 + np.abs(f)))
    s["net"].close()
