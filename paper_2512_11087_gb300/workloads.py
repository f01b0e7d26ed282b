"""Seeded synthetic inputs shaped like the paper's branch-and-bound workloads.

This module holds none of the method's arithmetic: it only draws weights, boxes,
split lists, constraint counts and target lists from seeded generators.  Both the
CUDA path and the FP64 oracle receive the arrays it returns.  Anything that
depends on bounds (which neurons are unstable, the final-layer plane used as an
output constraint) is passed IN by the caller, computed by whichever side the
caller trusts.

Recipe (one line per workload; sizes follow the paper's benchmark families):
  * weights: He-normal W ~ N(0, 2/fan_in), zero biases, numpy PCG64 seed 0;
  * boxes: centre x0 ~ U[0,1]^n (image-like) or U[-1,1]^n (control-like),
    L-inf radius eps, optionally intersected with [0,1];
  * splits: drawn uniformly without replacement among the given candidate neuron
    ids, sides uniform (seed 1); per-subdomain counts uniform in [kmin, kmax];
  * extra rows (input-BaB output constraints): the given plane shifted by a
    uniform offset so that it cuts the box (seed 2);
  * random cutting rows (several active rows per subdomain): Gaussian directions,
    each shifted so that the box centre satisfies it with slack (seed 4).
"""
from __future__ import annotations

import numpy as np

LAYER_DENSE = 0
LAYER_CONV2D = 1


def he_mlp(dims, seed=0):
    """Dense ReLU MLP with He-normal weights and zero biases.

    dims = [n0, n1, ..., nL].  Returns a list of layer dicts (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = []
    for i in range(1, len(dims)):
        fan_in = dims[i - 1]
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(dims[i], fan_in)).astype(np.float32)
        b = np.zeros(dims[i], dtype=np.float32)
        layers.append(dict(kind=LAYER_DENSE, W=W, b=b, in_shape=(fan_in,), out_shape=(dims[i],)))
    return layers


def he_cnn(in_shape, convs, fcs, seed=0):
    """ReLU CNN: convs = [(out_c, k, stride, pad), ...], then dense layers fcs = [n, ...].

    Conv weights [out_c, in_c, k, k] He-normal with fan_in = in_c*k*k, zero bias."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = []
    c, h, w = in_shape
    for (oc, k, s, p) in convs:
        fan_in = c * k * k
        Wt = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(oc, c, k, k)).astype(np.float32)
        ho = (h + 2 * p - k) // s + 1
        wo = (w + 2 * p - k) // s + 1
        layers.append(dict(kind=LAYER_CONV2D, W=Wt, b=np.zeros(oc, np.float32),
                           in_shape=(c, h, w), out_shape=(oc, ho, wo), stride=s, pad=p))
        c, h, w = oc, ho, wo
    n = c * h * w
    for m in fcs:
        W = rng.normal(0.0, np.sqrt(2.0 / n), size=(m, n)).astype(np.float32)
        layers.append(dict(kind=LAYER_DENSE, W=W, b=np.zeros(m, np.float32),
                           in_shape=(n,), out_shape=(m,)))
        n = m
    return layers


def layer_dims(layers):
    """[n0, n1, ..., nL] (flattened sizes)."""
    d = [int(np.prod(layers[0]["in_shape"]))]
    for ly in layers:
        d.append(int(np.prod(ly["out_shape"])))
    return d


def box(n, eps, seed=0, centre="unit", clip01=False):
    """An L-inf box of radius eps around a random centre (float32 lo, hi)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    if centre == "unit":
        x0 = rng.uniform(0.0, 1.0, size=n)
    else:
        x0 = rng.uniform(-1.0, 1.0, size=n)
    lo = x0 - eps
    hi = x0 + eps
    if clip01:
        lo = np.maximum(lo, 0.0)
        hi = np.minimum(hi, 1.0)
    return lo.astype(np.float32), hi.astype(np.float32)


def tile_box(lo, hi, B):
    """The same box for B subdomains (activation BaB keeps the root box)."""
    return (np.ascontiguousarray(np.broadcast_to(lo, (B, lo.size))).astype(np.float32),
            np.ascontiguousarray(np.broadcast_to(hi, (B, hi.size))).astype(np.float32))


def margin_spec(n_out, y=0):
    """m = n_out-1 margin rows e_y - e_k and zero thresholds (Appendix, spec matrix)."""
    rows = []
    for k in range(n_out):
        if k == y:
            continue
        r = np.zeros(n_out, np.float32)
        r[y] = 1.0
        r[k] = -1.0
        rows.append(r)
    return np.stack(rows).astype(np.float32), np.zeros(len(rows), np.float32)


def draw_counts(B, kmin, kmax, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(kmin, kmax + 1, size=B)


def draw_splits(candidates, B, kmin, kmax, seed=1):
    """CSR split lists: per subdomain k ~ U{kmin..kmax} distinct candidates, sides uniform.

    candidates: int array of global hidden-neuron ids.  Entries are signed codes
    +(id+1) for z >= 0 (active) and -(id+1) for z <= 0 (inactive)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cand = np.asarray(candidates, dtype=np.int64)
    counts = rng.integers(kmin, kmax + 1, size=B)
    counts = np.minimum(counts, cand.size)
    off = np.zeros(B + 1, np.int32)
    off[1:] = np.cumsum(counts)
    ids = np.empty(int(off[-1]), np.int32)
    for b in range(B):
        pick = rng.choice(cand.size, size=int(counts[b]), replace=False)
        side = rng.integers(0, 2, size=int(counts[b]))
        codes = cand[pick] + 1
        ids[off[b]:off[b + 1]] = np.where(side == 1, codes, -codes)
    return off, ids


def shifted_plane_rows(a, c, lo, hi, B, seed=2, spread=0.5):
    """One extra row per subdomain: the plane a.x + c, shifted so it cuts the box.

    The shift puts the plane's zero level at xhat + s*eps-weighted offset with
    s ~ U(-spread, spread) (so the row is neither infeasible nor redundant)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.asarray(a, np.float64)
    G = np.empty((B, a.size), np.float32)
    h = np.empty(B, np.float32)
    for b in range(B):
        xh = 0.5 * (lo[b].astype(np.float64) + hi[b].astype(np.float64))
        ep = 0.5 * (hi[b].astype(np.float64) - lo[b].astype(np.float64))
        s = rng.uniform(-spread, spread)
        G[b] = a.astype(np.float32)
        h[b] = np.float32(-(a @ xh) + s * (np.abs(a) @ ep))
    off = np.arange(B + 1, dtype=np.int32)
    return off, G, h


def random_cut_rows(lo, hi, B, kmin, kmax, seed=4, spread=0.6):
    """kmin..kmax extra rows g.x + h <= 0 per subdomain (CSR), Gaussian directions, each shifted so
    that the box centre satisfies it with slack s*|g|.eps, s ~ U(0.05, spread): every row cuts the
    box (neither redundant nor infeasible on its own) and the centre stays feasible."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = lo.shape[1]
    counts = rng.integers(kmin, kmax + 1, size=B)
    off = np.zeros(B + 1, np.int32)
    off[1:] = np.cumsum(counts)
    G = np.empty((int(off[-1]), n), np.float32)
    h = np.empty(int(off[-1]), np.float32)
    for b in range(B):
        xh = 0.5 * (lo[b].astype(np.float64) + hi[b].astype(np.float64))
        ep = 0.5 * (hi[b].astype(np.float64) - lo[b].astype(np.float64))
        for r in range(off[b], off[b + 1]):
            g = rng.normal(size=n).astype(np.float32)
            s = rng.uniform(0.05, spread)
            G[r] = g
            h[r] = np.float32(-(g.astype(np.float64) @ xh) - s * (np.abs(g.astype(np.float64)) @ ep))
    return off, G, h


def random_targets(U, B, k, seed=3):
    """CSR lists of k distinct cache slots per subdomain (complete-clipping targets)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(k, U)
    off = np.arange(B + 1, dtype=np.int32) * k
    ids = np.empty(B * k, np.int32)
    for b in range(B):
        ids[b * k:(b + 1) * k] = np.sort(rng.choice(U, size=k, replace=False))
    return off, ids


# Workload shapes (the paper's BaB workload families; sizes per round).
CONFIGS = {
    # control-like small MLP, relaxed clipping, one output constraint per subdomain
    "mlp5x50": dict(dims=[5] + [50] * 6 + [5], centre="pm1", eps=0.05, clip01=False,
                    B=256, kmin=0, kmax=8, out_rows=1, sweeps=0, relaxed=1),
    # MNIST-MLP-like: 784 -> 256x6 -> 10, complete clipping 10 sweeps
    "mlp784x256": dict(dims=[784] + [256] * 6 + [10], centre="unit", eps=0.02, clip01=True,
                       B=4096, kmin=1, kmax=4, out_rows=0, sweeps=10, relaxed=1),
    # alpha optimisation: 784 -> 1024x4 -> 10
    "mlp784x1024": dict(dims=[784] + [1024] * 4 + [10], centre="unit", eps=0.02, clip01=True,
                        B=1024, kmin=0, kmax=12, out_rows=0, sweeps=0, relaxed=1),
    # CIFAR-style CNN on 3x32x32: conv 16 4x4 s2 p1, conv 32 4x4 s2 p1, conv 32 3x3 s1 p1, FC 100, FC 10;
    # 2048 subdomains with 1-16 splits; complete clipping on the top-20 targets per hidden layer
    "cnn3x32": dict(in_shape=(3, 32, 32), convs=[(16, 4, 2, 1), (32, 4, 2, 1), (32, 3, 1, 1)], fcs=[100, 10],
                    centre="unit", eps=2.0 / 255.0, clip01=True, B=2048, kmin=1, kmax=16, out_rows=0, sweeps=10,
                    relaxed=1, topk=20),
    # BaB stress: 784 -> 512x8 -> 10, 65536 subdomains
    "mlp784x512x8": dict(dims=[784] + [512] * 8 + [10], centre="unit", eps=0.02, clip01=True,
                         B=65536, kmin=0, kmax=24, out_rows=0, sweeps=10, relaxed=1),
}
