"""The oracle's alpha gradient against FP64 central finite differences, and Adam."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_11087_gb300 import workloads as WL


def test_alpha_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = [6, 12, 12, 12, 4]
    net = O.Net(WL.he_mlp(dims, seed=3))
    lo = rng.uniform(-1, 0, 6); hi = lo + 0.9
    root = O.root_crown(net, lo, hi)
    hl, hu = root["l"], root["u"]
    hs = np.where(hl >= 0, 1, np.where(hu <= 0, -1, 0)).astype(np.int8)
    assert (hs == 0).sum() > 5
    C, t = WL.margin_spec(4, y=0)
    m, H = C.shape[0], net.H
    alpha = rng.uniform(0.2, 0.8, size=(m, H))
    gf = rng.uniform(0.5, 1.5, m)
    f, g = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, gf)
    h = 1e-6
    checked = 0
    for r in range(m):
        for j in rng.choice(H, 12, replace=False):
            ap, am = alpha.copy(), alpha.copy()
            ap[r, j] += h; am[r, j] -= h
            fp, _ = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, ap, gf)
            fm, _ = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, am, gf)
            fd = gf[r] * (fp[r] - fm[r]) / (2 * h)
            assert g[r, j] == pytest.approx(fd, rel=1e-5, abs=1e-7)
            checked += abs(g[r, j]) > 0
    assert checked > 3
    # stable neurons never carry a slope gradient
    assert np.all(g[:, hs != 0] == 0.0)


def test_alpha_gradient_consistent_with_batch_bound():
    rng = np.random.default_rng(1)
    dims = [5, 10, 10, 3]
    net = O.Net(WL.he_mlp(dims, seed=4))
    lo = rng.uniform(-1, 0, 5).astype(np.float32).astype(np.float64)
    hi = (lo + 0.8).astype(np.float32).astype(np.float64)
    root = O.root_crown(net, lo, hi)
    cache = O.make_cache(root)
    C, t = WL.margin_spec(3, y=0)
    alpha = rng.uniform(0, 1, size=(1, C.shape[0], net.H))
    out = O.bound_batch(net, cache, lo[None], hi[None], C=C, t=t, alpha=alpha, relaxed=0, sweeps=0)
    hs = np.where(root["l"] >= 0, 1, np.where(root["u"] <= 0, -1, 0)).astype(np.int8)
    f, _ = O.alpha_grad(net, root["l"], root["u"], hs, lo, hi, C, t, alpha[0])
    assert np.allclose(f, out["lower"][0], rtol=1e-12, atol=1e-12)
    # the magnitude scale it reports is the round's lower_scale (root magnitudes)
    zm = np.maximum(np.abs(cache["root_l"]), np.abs(cache["root_u"]))
    _, _, sc = O.alpha_grad(net, root["l"], root["u"], hs, lo, hi, C, t, alpha[0], zmag=zm, want_scale=True)
    assert np.allclose(sc, out["lower_scale"][0], rtol=1e-12, atol=0)


def test_adam_first_step_and_clamp():
    # Adam's first bias-corrected step is lr * g / (|g| + eps'): a move of lr along sign(g)
    rng = np.random.default_rng(2)
    g = rng.normal(size=50)
    a = np.full(50, 0.5)
    m1, m2 = np.zeros(50), np.zeros(50)
    O.adam_step(a, m1, m2, g, t=1, lr=0.1, eps=1e-12)
    assert np.allclose(a, 0.5 + 0.1 * np.sign(g), atol=1e-9)
    # a step past the box is clamped to [0, 1]
    a = np.array([0.95, 0.05]); m1, m2 = np.zeros(2), np.zeros(2)
    O.adam_step(a, m1, m2, np.array([1.0, -1.0]), t=1, lr=0.1)
    assert np.array_equal(a, [1.0, 0.0])
    # ascent on a concave 1-D objective converges to its maximiser inside [0,1]
    a = np.array([0.1]); m1, m2 = np.zeros(1), np.zeros(1)
    for it in range(1, 400):
        O.adam_step(a, m1, m2, -2.0 * (a - 0.7), t=it, lr=0.05)
    assert a[0] == pytest.approx(0.7, abs=2e-3)


# ---------------------------------------------------------------- split multipliers (beta)
# A split z_g >= 0 (bsign +1) or z_g <= 0 (-1) holds -bsign_g z_g <= 0 on the subdomain, so adding
# beta_g (-bsign_g z_g), beta_g >= 0, to the CROWN bound keeps it a lower bound there.

def _split_case(seed, dims, nsplit):
    rng = np.random.default_rng(seed)
    net = O.Net(WL.he_mlp(dims, seed=seed))
    lo = rng.uniform(-1, 0, dims[0]); hi = lo + 1.0
    root = O.root_crown(net, lo, hi)
    hl, hu = root["l"].copy(), root["u"].copy()
    un = np.nonzero((hl < 0) & (hu > 0))[0]
    pick = rng.choice(un, nsplit, replace=False)
    bsign = np.zeros(net.H, np.int8)
    for g in pick:
        bsign[g] = 1 if rng.uniform() < 0.5 else -1
        if bsign[g] > 0: hl[g] = 0.0      # the split enforced on the neuron's own bounds
        else: hu[g] = 0.0
    hs = np.where(hl >= 0, 1, np.where(hu <= 0, -1, 0)).astype(np.int8)
    C, t = WL.margin_spec(dims[-1], y=0)
    return rng, net, lo, hi, hl, hu, hs, bsign, C, t


def _true_min(net, lo, hi, bsign, C, t, n=200000, seed=0):
    """least spec value over sampled points of the subdomain (box and split signs)"""
    rng = np.random.default_rng(seed)
    x = lo + (hi - lo) * rng.uniform(size=(n, lo.size))
    ok = np.ones(n, bool)
    z = x
    g0 = 0
    for W, b in zip(net.Ws[:-1], net.bs[:-1]):
        pre = z @ W.T + b
        sl = bsign[g0:g0 + W.shape[0]]
        ok &= np.all((pre * sl[None, :]) >= 0, axis=1)
        z = np.maximum(pre, 0)
        g0 += W.shape[0]
    y = z @ net.Ws[-1].T + net.bs[-1]
    v = y @ C.T + t
    return v[ok].min(axis=0), int(ok.sum())


def test_beta_gradient_matches_finite_differences_and_zero_beta_is_crown():
    rng, net, lo, hi, hl, hu, hs, bsign, C, t = _split_case(11, [6, 12, 12, 12, 4], 4)
    m, H = C.shape[0], net.H
    alpha = rng.uniform(0.2, 0.8, size=(m, H))
    f0, g0 = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha)
    fz, gz, gbz = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, beta=np.zeros((m, H)), bsign=bsign)
    assert np.array_equal(f0, fz) and np.array_equal(g0, gz)
    beta = rng.uniform(0.0, 0.5, size=(m, H)) * (bsign != 0)
    gf = rng.uniform(0.5, 1.5, m)
    f, g, gb = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, gf, beta=beta, bsign=bsign)
    assert np.all(gb[:, bsign == 0] == 0.0)
    h = 1e-6
    checked = 0
    for r in range(m):
        for j in np.nonzero(bsign)[0]:
            bp, bm = beta.copy(), beta.copy()
            bp[r, j] += h; bm[r, j] -= h
            fp = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, gf, beta=bp, bsign=bsign)[0]
            fm = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, gf, beta=bm, bsign=bsign)[0]
            fd = gf[r] * (fp[r] - fm[r]) / (2 * h)
            assert gb[r, j] == pytest.approx(fd, rel=1e-5, abs=1e-7)
            checked += abs(gb[r, j]) > 0
    assert checked > 4


@pytest.mark.parametrize("seed", [12, 13])
def test_beta_bound_stays_below_the_sampled_minimum(seed):
    rng, net, lo, hi, hl, hu, hs, bsign, C, t = _split_case(seed, [4, 10, 10, 3], 3)
    m, H = C.shape[0], net.H
    vmin, nok = _true_min(net, lo, hi, bsign, C, t, seed=seed)
    assert nok > 100
    alpha = np.ones((m, H))
    for scale in (0.1, 1.0, 10.0):
        beta = rng.uniform(0, scale, size=(m, H)) * (bsign != 0)
        f = O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, beta=beta, bsign=bsign)[0]
        assert np.all(f <= vmin + 1e-9)


@pytest.mark.parametrize("seed", [15, 21, 28])
def test_optimal_beta_on_an_affine_region_is_the_exact_lp(seed):
    """One hidden layer whose neurons are all stable but one split neuron: the network is affine on
    the subdomain, so the best beta closes the gap to the LP over the box and the split halfspace
    (LP duality with one constraint), computed here by vertex enumeration."""
    from tests._brute import lp_vertex
    rng = np.random.default_rng(seed)
    n0, n1 = 3, 6
    W1 = rng.normal(size=(n1, n0)); b1 = np.where(rng.uniform(size=n1) < 0.5, 6.0, -6.0); b1[0] = 0.0
    W2 = rng.normal(size=(1, n1)); b2 = np.zeros(1)
    layers = [dict(kind=WL.LAYER_DENSE, W=W1.astype(np.float32), b=b1.astype(np.float32), in_shape=(n0,),
                   out_shape=(n1,)),
              dict(kind=WL.LAYER_DENSE, W=W2.astype(np.float32), b=b2.astype(np.float32), in_shape=(n1,),
                   out_shape=(1,))]
    net = O.Net(layers)
    W1, b1, W2 = net.Ws[0], net.bs[0], net.Ws[1]
    lo, hi = -np.ones(n0), np.ones(n0)
    root = O.root_crown(net, lo, hi)
    hl, hu = root["l"].copy(), root["u"].copy()
    assert hl[0] < 0 < hu[0] and np.all((hl[1:] >= 0) | (hu[1:] <= 0))
    bsign = np.zeros(n1, np.int8); bsign[0] = 1
    hl[0] = 0.0                                    # split z_0 >= 0, enforced
    hs = np.where(hl >= 0, 1, np.where(hu <= 0, -1, 0)).astype(np.int8)
    C, t = np.ones((1, 1)), np.zeros(1)
    alpha = np.ones((1, n1))
    # the exact minimum of the affine network over {box, z_0 >= 0}
    d = (hs > 0).astype(float)
    obj = (W2 * d) @ W1
    c0 = float(((W2 * d) @ b1 + net.bs[1])[0])
    exact = lp_vertex(obj[0], c0, -W1[:1], -b1[:1], lo, hi)
    f_of = lambda bb: O.alpha_grad(net, hl, hu, hs, lo, hi, C, t, alpha, beta=np.array([[bb] + [0.0] * (n1 - 1)]),
                                   bsign=bsign)[0][0]
    # f is concave in beta: ternary search on a bracket that holds the maximiser
    a, b = 0.0, 1.0
    while f_of(2 * b) > f_of(b):
        b *= 2
    b *= 2
    for _ in range(200):
        m1, m2 = a + (b - a) / 3, b - (b - a) / 3
        if f_of(m1) < f_of(m2): a = m1
        else: b = m2
    best = f_of(0.5 * (a + b))
    assert f_of(0.0) < exact - 1e-3           # the split constraint matters here
    assert best <= exact + 1e-9
    assert best == pytest.approx(exact, abs=1e-9 * (1 + abs(exact)))


def test_adam_range_clamps_below_only():
    x = np.array([0.05, 3.0]); m1, m2 = np.zeros(2), np.zeros(2)
    O.adam_step_range(x, m1, m2, np.array([-1.0, 1.0]), t=1, lr=0.1, lo=0.0, hi=np.inf)
    assert x[0] == 0.0 and x[1] == pytest.approx(3.1)
