"""The oracle's bound propagation and batch pipeline against closed forms and sampling.

Pins: an affine network (no hidden layer, or every neuron stable) makes CROWN exact,
so its bound equals the exact LP optimum by vertex enumeration (Lemma A.1 composed
with the back-substitution algebra); sampled points never violate any bound (the
ReLU relaxation Lemma); clipping never loosens anything; feasible points of a
subdomain stay inside its clipped box and bounds."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_11087_gb300 import workloads as WL
from tests._brute import lp_vertex


def small_net(dims, seed, bias_scale=0.0):
    layers = WL.he_mlp(dims, seed=seed)
    if bias_scale:
        rng = np.random.default_rng(seed + 7)
        for ly in layers:
            ly["b"] = (rng.normal(size=ly["b"].shape) * bias_scale).astype(np.float32)
    return layers


def test_affine_network_bound_is_exact_lp():
    rng = np.random.default_rng(0)
    for seed in range(5):
        n0 = int(rng.integers(2, 5))
        layers = small_net([n0, 3], seed, bias_scale=0.5)
        net = O.Net(layers)
        lo = rng.uniform(-1, 0, n0).astype(np.float32).astype(np.float64)
        hi = (lo + rng.uniform(0.1, 1, n0)).astype(np.float32).astype(np.float64)
        C, t = WL.margin_spec(3, y=0)
        cache = O.make_cache(O.root_crown(net, lo, hi))
        out = O.bound_batch(net, cache, lo[None], hi[None], C=C, t=t, relaxed=0, sweeps=0)
        W, b = net.Ws[0], net.bs[0]
        for r in range(C.shape[0]):
            a = C[r] @ W
            exact = lp_vertex(a, C[r] @ b + t[r], None, None, lo, hi)
            assert out["lower"][0, r] == pytest.approx(exact, abs=1e-12)


def test_all_stable_network_is_exact():
    # non-negative hidden weights with a positive bias keep every hidden neuron stably
    # active; a few neurons get a large negative bias and are stably inactive.  The
    # network is affine on the box and CROWN must return the exact minimum.
    rng = np.random.default_rng(1)
    dims = [3, 6, 5, 4]
    layers = small_net(dims, 11)
    for ly in layers[:-1]:
        ly["W"] = np.abs(ly["W"])
        ly["b"] = np.full(ly["b"].shape, 5.0, np.float32)
        ly["b"][:2] = -1000.0
    net = O.Net(layers)
    lo = rng.uniform(-0.1, 0, 3).astype(np.float32).astype(np.float64)
    hi = (lo + 0.05).astype(np.float32).astype(np.float64)
    root = O.root_crown(net, lo, hi)
    assert np.all((root["l"] >= 0) | (root["u"] <= 0))
    assert (root["u"] <= 0).sum() == 4 and (root["l"] >= 0).sum() == 7
    cache = O.make_cache(root)
    assert cache["ids"].size == 0
    C, t = WL.margin_spec(4, y=1)
    out = O.bound_batch(net, cache, lo[None], hi[None], C=C, t=t, relaxed=0, sweeps=0)
    # exact affine composition with the inactive neurons removed
    M, v = np.eye(3), np.zeros(3)
    for i, (W, b) in enumerate(zip(net.Ws, net.bs)):
        M, v = W @ M, W @ v + b
        if i < net.L - 1:
            M[:2] = 0.0
            v[:2] = 0.0
    for r in range(C.shape[0]):
        exact = lp_vertex(C[r] @ M, C[r] @ v + t[r], None, None, lo, hi)
        assert out["lower"][0, r] == pytest.approx(exact, rel=1e-12, abs=1e-10)


def test_root_bounds_and_planes_are_sound_by_sampling():
    rng = np.random.default_rng(2)
    dims = [6, 20, 20, 20, 5]
    net = O.Net(small_net(dims, 3, bias_scale=0.3))
    lo = rng.uniform(-1, 0, 6); hi = lo + 0.6
    r = O.root_crown(net, lo, hi)
    X = lo + (hi - lo) * rng.uniform(size=(20000, 6))
    X = np.vstack([X] + [np.where(np.array(b), hi, lo)[None] for b in itertools.product([0, 1], repeat=6)])
    _, pre = net.forward(X)
    Z = np.concatenate(pre, axis=1)
    assert np.all(Z >= r["l"] - 1e-9) and np.all(Z <= r["u"] + 1e-9)
    assert np.all(Z >= X @ r["lA"].T + r["lc"] - 1e-9)
    assert np.all(Z <= X @ r["uA"].T + r["uc"] + 1e-9)
    # and not vacuous: some neurons unstable, bounds finite
    assert np.all(np.isfinite(r["l"])) and (r["l"] < 0).any() and (r["u"] > 0).any()


def _pattern_ok(pre_all, split_ids):
    ok = np.ones(pre_all.shape[0], bool)
    for code in split_ids:
        g = abs(int(code)) - 1
        ok &= (pre_all[:, g] >= 0) if code > 0 else (pre_all[:, g] <= 0)
    return ok


@pytest.mark.parametrize("sweeps", [0, 3])
def test_batch_soundness_by_sampling(sweeps):
    rng = np.random.default_rng(3)
    dims = [5, 16, 16, 16, 4]
    net = O.Net(small_net(dims, 5, bias_scale=0.2))
    lo0 = rng.uniform(-1, 0, 5); hi0 = lo0 + 0.8
    root = O.root_crown(net, lo0, hi0)
    cache = O.make_cache(root)
    B = 12
    so, si = WL.draw_splits(cache["ids"], B, 1, 4, seed=4)
    lo, hi = WL.tile_box(lo0.astype(np.float32), hi0.astype(np.float32), B)
    lo, hi = lo.astype(np.float64), hi.astype(np.float64)
    C, t = WL.margin_spec(4, y=0)
    out = O.bound_batch(net, cache, lo, hi, split_off=so, split_ids=si, C=C, t=t,
                        relaxed=1, sweeps=sweeps)
    X = lo0 + (hi0 - lo0) * rng.uniform(size=(40000, 5))
    Y, pre = net.forward(X)
    Z = np.concatenate(pre, axis=1)
    F = Y @ C.T + t
    ids = cache["ids"]
    checked = 0
    for b in range(B):
        ok = _pattern_ok(Z, si[so[b]:so[b + 1]])
        if out["infeasible"][b]:
            assert not ok.any()
            continue
        Xb, Zb, Fb = X[ok], Z[ok], F[ok]
        checked += ok.sum()
        assert np.all(Xb >= out["lo_clip"][b] - 1e-12) and np.all(Xb <= out["hi_clip"][b] + 1e-12)
        assert np.all(Zb[:, ids] >= out["l"][b] - 1e-9) and np.all(Zb[:, ids] <= out["u"][b] + 1e-9)
        assert np.all(Fb >= out["lower"][b] - 1e-9)
        # clipping never loosens: inside the root bounds, inside the input box
        assert np.all(out["l"][b] >= root["l"][ids] - 1e-12) and np.all(out["u"][b] <= root["u"][ids] + 1e-12)
        assert np.all(out["lo_clip"][b] >= lo[b]) and np.all(out["hi_clip"][b] <= hi[b])
    assert checked > 100


def test_clipping_only_tightens_the_final_bound():
    rng = np.random.default_rng(4)
    dims = [8, 24, 24, 3]
    net = O.Net(small_net(dims, 9, bias_scale=0.2))
    lo0 = rng.uniform(-1, 0, 8); hi0 = lo0 + 0.5
    cache = O.make_cache(O.root_crown(net, lo0, hi0))
    B = 16
    so, si = WL.draw_splits(cache["ids"], B, 1, 3, seed=8)
    lo, hi = WL.tile_box(lo0.astype(np.float32), hi0.astype(np.float32), B)
    C, t = WL.margin_spec(3, y=2)
    kw = dict(split_off=so, split_ids=si, C=C, t=t)
    plain = O.bound_batch(net, cache, lo, hi, relaxed=0, sweeps=0, **kw)
    rel = O.bound_batch(net, cache, lo, hi, relaxed=1, sweeps=0, **kw)
    comp = O.bound_batch(net, cache, lo, hi, relaxed=1, sweeps=4, **kw)
    fe = ~(plain["infeasible"].astype(bool) | rel["infeasible"].astype(bool) | comp["infeasible"].astype(bool))
    assert fe.any()
    assert np.all(rel["lower"][fe] >= plain["lower"][fe] - 1e-9)
    assert np.all(comp["lower"][fe] >= rel["lower"][fe] - 1e-9)
    assert np.all(comp["l"][fe] >= rel["l"][fe] - 1e-12) and np.all(comp["u"][fe] <= rel["u"][fe] + 1e-12)


def test_no_constraints_reduces_to_crown_with_root_bounds():
    # without splits or rows, one round leaves the root bounds and the box unchanged
    rng = np.random.default_rng(5)
    dims = [4, 10, 10, 3]
    net = O.Net(small_net(dims, 2, bias_scale=0.3))
    lo0 = rng.uniform(-1, 0, 4); hi0 = lo0 + 0.7
    root = O.root_crown(net, lo0, hi0)
    cache = O.make_cache(root)
    C, t = WL.margin_spec(3, y=0)
    out = O.bound_batch(net, cache, lo0[None], hi0[None], C=C, t=t, relaxed=1, sweeps=5)
    assert np.array_equal(out["l"][0], root["l"][cache["ids"]])
    assert np.array_equal(out["u"][0], root["u"][cache["ids"]])
    assert np.array_equal(out["lo_clip"][0], lo0.astype(np.float32)) or np.allclose(out["lo_clip"][0], lo0)
