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
