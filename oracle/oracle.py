"""ctypes wrapper around the FP64 C oracle (cv_oracle.c) plus the conv-to-dense expansion.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg.  It imports nothing from the CUDA product package.

Every floating-point input is converted to float64 exactly (the callers hand FP32
values); every result is float64 except masks and flags.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cv_oracle.c")
_LIB = os.path.join(_HERE, "libcv_oracle.so")
_lib = None

def build(force=False):
    """Compile cv_oracle.c with gcc (plain -O2, IEEE semantics, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"]
    subprocess.check_call(cmd)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        _lib.orc_concretize.argtypes = [I, P, D, P, P, P, P]
        _lib.orc_root_crown.argtypes = [I, P, P, P, P, P, I, P, P, P, P, P, P, P, P]
        _lib.orc_row_check.argtypes = [I, P, D, P, P, P, P, P]
        _lib.orc_row_check.restype = I
        _lib.orc_relaxed_clip_row.argtypes = [I, P, D, P, P, P, P]
        _lib.orc_relaxed_clip_parallel.argtypes = [I, I, P, P, P, P, P, P]
        _lib.orc_relaxed_clip_parallel.restype = I
        _lib.orc_relaxed_clip_sequential.argtypes = [I, I, P, P, P, P, P, P]
        _lib.orc_relaxed_clip_sequential.restype = I
        _lib.orc_row_order.argtypes = [I, I, P, P, P, P, ctypes.POINTER(ctypes.c_int)]
        _lib.orc_row_order.restype = None
        _lib.orc_input_split.argtypes = [I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_input_split.restype = I
        _lib.orc_activation_split.argtypes = [I, I, I] + [P] * 20
        _lib.orc_activation_split.restype = I
        _lib.orc_select_targets.argtypes = [I, I, P, P, P, P, P, I, P, P]
        _lib.orc_select_targets.restype = I
        _lib.orc_complete_clip.argtypes = [I, P, D, I, P, P, P, P, I, P, P]
        _lib.orc_complete_clip.restype = D
        _lib.orc_dual_value.argtypes = [I, P, D, I, P, P, P, P, P]
        _lib.orc_dual_value.restype = D
        _lib.orc_bound_batch.argtypes = ([I, P, P, P] + [I, P, P, P, P, P] + [P, P, P] +
                                         [I, P, P, P, P] + [P, P] + [P, P, P] + [I, P, P] +
                                         [P, I] + [P, P] + [I, I, I] +
                                         [P] * 14 + [I])
        _lib.orc_bound_batch.restype = I
        _lib.orc_alpha_grad.argtypes = [I, P, P, P, P, P, P, P, P, I, P, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_adam_step_range.argtypes = [ctypes.c_long, P, P, P, P, I, D, D, D, D, D, D]
        _lib.orc_alpha_grad.restype = I
        _lib.orc_adam_step.argtypes = [ctypes.c_long, P, P, P, P, I, D, D, D, D]
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# network: conv layers become dense matrices written out from the definition
# --------------------------------------------------------------------------
def conv_to_dense(ly):
    """The dense matrix of a 2-D convolution with zero padding (output index
    (oc, oy, ox), input index (ic, iy, ix), row-major C,H,W flattening):
    W[(oc,oy,ox),(ic,iy,ix)] = K[oc,ic,ky,kx] where iy = oy*s - p + ky, ix = ox*s - p + kx."""
    K = np.asarray(ly["W"], np.float64)
    oc_n, ic_n, kh, kw = K.shape
    _, H, Wd = ly["in_shape"]
    _, Ho, Wo = ly["out_shape"]
    s, p = ly["stride"], ly["pad"]
    M = np.zeros((oc_n * Ho * Wo, ic_n * H * Wd))
    for oc in range(oc_n):
        for oy in range(Ho):
            for ox in range(Wo):
                r = (oc * Ho + oy) * Wo + ox
                for ic in range(ic_n):
                    for ky in range(kh):
                        iy = oy * s - p + ky
                        if iy < 0 or iy >= H:
                            continue
                        for kx in range(kw):
                            ix = ox * s - p + kx
                            if ix < 0 or ix >= Wd:
                                continue
                            M[r, (ic * H + iy) * Wd + ix] += K[oc, ic, ky, kx]
    bias = np.repeat(np.asarray(ly["b"], np.float64), Ho * Wo)
    return M, bias


class Net:
    """Dense FP64 view of a layer list (dicts from the workload generators)."""

    def __init__(self, layers):
        Ws, bs = [], []
        dims = [int(np.prod(layers[0]["in_shape"]))]
        for ly in layers:
            if ly["kind"] == 1:
                M, bb = conv_to_dense(ly)
            else:
                M, bb = np.asarray(ly["W"], np.float64), np.asarray(ly["b"], np.float64)
            Ws.append(M)
            bs.append(bb)
            dims.append(M.shape[0])
        self.Ws = Ws
        self.bs = bs
        self.dims = np.asarray(dims, np.int32)
        self.L = len(Ws)
        self.H = int(sum(dims[1:-1]))
        self.Wflat = _f64(np.concatenate([w.ravel() for w in Ws]))
        self.bflat = _f64(np.concatenate(bs))

    def forward(self, x):
        """Exact-ish FP64 forward pass; returns (output, list of pre-activations)."""
        z = np.asarray(x, np.float64)
        pre = []
        for i, (W, b) in enumerate(zip(self.Ws, self.bs)):
            z = z @ W.T + b
            if i < self.L - 1:
                pre.append(z.copy())
                z = np.maximum(z, 0.0)
        return z, pre


# --------------------------------------------------------------------------
# wrappers
# --------------------------------------------------------------------------
def concretize(a, c, lo, hi):
    lib = _load()
    a, lo, hi = _f64(a), _f64(lo), _f64(hi)
    vmin, vmax = ctypes.c_double(), ctypes.c_double()
    lib.orc_concretize(a.size, _p(a), float(c), _p(lo), _p(hi), ctypes.byref(vmin), ctypes.byref(vmax))
    return vmin.value, vmax.value


def root_crown(net: Net, lo, hi, alpha_mode=0):
    """Root CROWN bounds and planes of every hidden neuron (dict of float64 arrays)."""
    lib = _load()
    lo, hi = _f64(lo), _f64(hi)
    H, n0 = net.H, int(net.dims[0])
    out = dict(l=np.zeros(H), u=np.zeros(H), lA=np.zeros((H, n0)), lc=np.zeros(H),
               uA=np.zeros((H, n0)), uc=np.zeros(H), pscale=np.zeros(H), bscale=np.zeros(H))
    rc = lib.orc_root_crown(net.L, _p(net.dims), _p(net.Wflat), _p(net.bflat), _p(lo), _p(hi),
                            int(alpha_mode), _p(out["l"]), _p(out["u"]), _p(out["lA"]), _p(out["lc"]),
                            _p(out["uA"]), _p(out["uc"]), _p(out["pscale"]), _p(out["bscale"]))
    assert rc == 0
    return out


def make_cache(root):
    """Cache of the root-unstable neurons (Section 3.4): slots in global-id order."""
    l, u = root["l"], root["u"]
    ids = np.nonzero((l < 0.0) & (u > 0.0))[0].astype(np.int32)
    return dict(ids=ids, lA=root["lA"][ids], lc=root["lc"][ids], uA=root["uA"][ids], uc=root["uc"][ids],
                root_l=root["l"], root_u=root["u"], pscale=root["pscale"])


def cache_as_f32(cache):
    """The cache as the FP32 arrays both sides consume (values rounded to nearest)."""
    out = dict(cache)
    for k in ("lA", "lc", "uA", "uc"):
        out[k] = np.asarray(cache[k], np.float32).astype(np.float64)
    return out


def row_check(g, h, lo, hi):
    lib = _load()
    g, lo, hi = _f64(g), _f64(lo), _f64(hi)
    vmin, vmax, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    f = lib.orc_row_check(g.size, _p(g), float(h), _p(lo), _p(hi), ctypes.byref(vmin),
                          ctypes.byref(vmax), ctypes.byref(s))
    return f, vmin.value, vmax.value, s.value


def relaxed_clip(G, h, lo, hi, sequential=False):
    lib = _load()
    G, h, lo, hi = _f64(np.atleast_2d(G)), _f64(np.atleast_1d(h)), _f64(lo), _f64(hi)
    lo2, hi2 = np.zeros_like(lo), np.zeros_like(hi)
    fn = lib.orc_relaxed_clip_sequential if sequential else lib.orc_relaxed_clip_parallel
    inf = fn(lo.size, G.shape[0], _p(G), _p(h), _p(lo), _p(hi), _p(lo2), _p(hi2))
    return lo2, hi2, bool(inf)


def row_order(G, h, lo, hi):
    """Constraint importance heuristic (Appendix, details of heuristics): the row indices in
    ascending distance |g.xhat + h| / ||g||_2 of their hyperplanes from the box centre (stable)."""
    lib = _load()
    G, h, lo, hi = _f64(np.atleast_2d(G)), _f64(np.atleast_1d(h)), _f64(lo), _f64(hi)
    R = G.shape[0]
    perm = np.zeros(max(R, 1), np.int32)
    lib.orc_row_order(lo.size, R, _p(G), _p(h), _p(lo), _p(hi), perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return perm[:R]


def input_split(lo, hi, final_A, final_c, lower, verified, infeasible):
    """Input-BaB split step (Algorithm 4: Domain_Filter, Batch_Split sharing the parents' planes).
    lo, hi [B x n0]; final_A [B x m x n0]; final_c, lower [B x m]; verified, infeasible [B].
    Returns dict(lo, hi [2K x n0], row_off [2K+1], G [rows x n0], h [rows], parent [2K])."""
    lib = _load()
    f32 = lambda x: np.ascontiguousarray(np.asarray(x, np.float32))
    u8 = lambda x: np.ascontiguousarray(np.asarray(x, np.uint8))
    lo, hi, A, c, lower = f32(lo), f32(hi), f32(final_A), f32(final_c), f32(lower)
    B, n0 = lo.shape
    m = lower.shape[1] if lower.ndim == 2 else 1
    ver, inf = u8(verified), u8(infeasible)
    lo2 = np.zeros((2 * max(B, 1), n0), np.float32)
    hi2 = np.zeros_like(lo2)
    ro = np.zeros(2 * B + 1, np.int32)
    G = np.zeros((2 * max(B, 1), n0), np.float32)
    h = np.zeros(2 * max(B, 1), np.float32)
    par = np.zeros(2 * max(B, 1), np.int32)
    pf = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    n = lib.orc_input_split(B, n0, m, pf(lo), pf(hi), pf(A), pf(c), pf(lower), pf(ver), pf(inf), pf(lo2), pf(hi2),
                            pf(ro), pf(G), pf(h), pf(par))
    nr = int(ro[n])
    return dict(lo=lo2[:n], hi=hi2[:n], row_off=ro[:n + 1], G=G[:nr], h=h[:nr], parent=par[:n])


def _pf(x):
    return x.ctypes.data_as(ctypes.c_void_p)


def activation_split(ids, split_off, split_ids, lo, hi, l, u, mask, weight, verified, infeasible):
    """Activation-BaB split step (Algorithm 5: Domain_Filter, Batch_Split on the highest BaBSR score).
    Returns dict(split_off, split_ids, lo, hi, l, u, parent, branched [children], stuck [B])."""
    lib = _load()
    f32 = lambda x: np.ascontiguousarray(np.asarray(x, np.float32))
    i32 = lambda x: np.ascontiguousarray(np.asarray(x, np.int32))
    lo, hi, l, u = f32(lo), f32(hi), f32(l), f32(u)
    B, n0 = lo.shape
    U = l.shape[1]
    mask = np.ascontiguousarray(np.asarray(mask, np.int8))
    ver, inf = (np.ascontiguousarray(np.asarray(x, np.uint8)) for x in (verified, infeasible))
    so = i32(split_off) if split_off is not None else np.zeros(B + 1, np.int32)
    si = i32(split_ids) if split_ids is not None and len(split_ids) else np.zeros(1, np.int32)
    w = f32(weight) if weight is not None else None
    cap = 2 * max(B, 1)
    so2 = np.zeros(2 * B + 1, np.int32)
    si2 = np.zeros(2 * (int(so[-1]) + B) + 1, np.int32)
    lo2, hi2 = np.zeros((cap, n0), np.float32), np.zeros((cap, n0), np.float32)
    l2, u2 = np.zeros((cap, U), np.float32), np.zeros((cap, U), np.float32)
    par, br = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    stuck = np.zeros(max(B, 1), np.uint8)
    n = lib.orc_activation_split(B, U, n0, _pf(i32(ids)), _pf(so), _pf(si), _pf(lo), _pf(hi), _pf(l), _pf(u),
                                 _pf(mask), _pf(w) if w is not None else None, _pf(ver), _pf(inf), _pf(so2),
                                 _pf(si2), _pf(lo2), _pf(hi2), _pf(l2), _pf(u2), _pf(par), _pf(br), _pf(stuck))
    return dict(split_off=so2[:n + 1], split_ids=si2[:so2[n]], lo=lo2[:n], hi=hi2[:n], l=l2[:n], u=u2[:n],
                parent=par[:n], branched=br[:n], stuck=stuck[:B])


def layer_of_slots(net, ids):
    """Hidden layer (1-based) of every cache slot, from the global ids (hidden layer i holds ids
    hoff_i .. hoff_i + n_i - 1)."""
    hoff = np.cumsum([0] + list(net.dims[1:-1]))
    return (np.searchsorted(hoff, np.asarray(ids), side="right")).astype(np.int32)


def select_targets(layer_of, l, u, mask, weight, k):
    """Top-k BaBSR targets per subdomain and hidden layer, in slot order (CSR)."""
    lib = _load()
    l = np.ascontiguousarray(np.asarray(l, np.float32))
    u = np.ascontiguousarray(np.asarray(u, np.float32))
    mask = np.ascontiguousarray(np.asarray(mask, np.int8))
    B, U = l.shape
    w = np.ascontiguousarray(np.asarray(weight, np.float32)) if weight is not None else None
    off = np.zeros(B + 1, np.int32)
    ids = np.zeros(max(B * U, 1), np.int32)
    n = lib.orc_select_targets(B, U, _pf(np.ascontiguousarray(layer_of, dtype=np.int32)), _pf(l), _pf(u), _pf(mask),
                               _pf(w) if w is not None else None, int(k), _pf(off), _pf(ids))
    return off, ids[:n]


def complete_clip(a, c, G, h, lo, hi, sweeps):
    """Algorithm 1 repeated `sweeps` times: (value, beta, scale)."""
    lib = _load()
    a, G, h, lo, hi = _f64(a), _f64(np.atleast_2d(G)), _f64(np.atleast_1d(h)), _f64(lo), _f64(hi)
    R = G.shape[0] if G.size else 0
    beta = np.zeros(max(R, 1))
    sc = ctypes.c_double()
    v = lib.orc_complete_clip(a.size, _p(a), float(c), R, _p(G), _p(h), _p(lo), _p(hi), int(sweeps),
                              _p(beta), ctypes.byref(sc))
    return v, beta[:R], sc.value


def dual_value(a, c, G, h, lo, hi, beta):
    lib = _load()
    a, G, h, lo, hi, beta = (_f64(a), _f64(np.atleast_2d(G)), _f64(np.atleast_1d(h)), _f64(lo),
                             _f64(hi), _f64(beta))
    return lib.orc_dual_value(a.size, _p(a), float(c), G.shape[0], _p(G), _p(h), _p(lo), _p(hi), _p(beta))


def bound_batch(net: Net, cache, lo, hi, *, l_in=None, u_in=None, split_off=None, split_ids=None,
                row_off=None, G=None, h=None, C, t, alpha=None, alpha_mode=0,
                tgt_off=None, tgt_ids=None, relaxed=1, sweeps=0, enforce_splits=1, want_final=False,
                want_weight=False, nthreads=0):
    """One BaB round (a2..a8) for B subdomains.  Returns a dict of outputs (with want_weight, also
    "babsr_weight" [B x U]: the BaBSR weight of every cached neuron from the spec back-substitution;
    0 for infeasible subdomains)."""
    lib = _load()
    lo, hi = _f64(lo), _f64(hi)
    B, n0 = lo.shape
    ids = _i32(cache["ids"])
    U = ids.size
    m = int(np.asarray(C).shape[0])
    lA, lc, uA, uc = (_f64(cache[k]) for k in ("lA", "lc", "uA", "uc"))
    rl, ru, ps = _f64(cache["root_l"]), _f64(cache["root_u"]), _f64(cache["pscale"])
    if lA.size == 0:
        lA = np.zeros((1, n0)); uA = np.zeros((1, n0)); lc = np.zeros(1); uc = np.zeros(1)
    l_in = None if l_in is None else _f64(l_in)
    u_in = None if u_in is None else _f64(u_in)
    so = None if split_off is None else _i32(split_off)
    si = None if split_ids is None else _i32(split_ids)
    if si is not None and si.size == 0:
        si = np.zeros(1, np.int32)
    ro = None if row_off is None else _i32(row_off)
    Gx = None if G is None else _f64(G)
    hx = None if h is None else _f64(h)
    if Gx is not None and Gx.size == 0:
        Gx = np.zeros((1, n0)); hx = np.zeros(1)
    Cx, tx = _f64(C), _f64(t)
    al = None if alpha is None else _f64(alpha)
    to = None if tgt_off is None else _i32(tgt_off)
    ti = None if tgt_ids is None else _i32(tgt_ids)
    if ti is not None and ti.size == 0:
        ti = np.zeros(1, np.int32)
    Uo = max(U, 1)
    out = dict(lower=np.zeros((B, m)), lower_scale=np.zeros((B, m)),
               lo_clip=np.zeros((B, n0)), hi_clip=np.zeros((B, n0)),
               l=np.zeros((B, Uo)), u=np.zeros((B, Uo)), l_scale=np.zeros((B, Uo)), u_scale=np.zeros((B, Uo)),
               mask=np.zeros((B, Uo), np.int8), infeasible=np.zeros(B, np.uint8), verified=np.zeros(B, np.uint8))
    fA = np.zeros((B, m, n0)) if want_final else None
    fc = np.zeros((B, m)) if want_final else None
    bw = np.zeros((B, Uo)) if want_weight else None
    rc = lib.orc_bound_batch(net.L, _p(net.dims), _p(net.Wflat), _p(net.bflat),
                             U, _p(ids), _p(lA), _p(lc), _p(uA), _p(uc), _p(rl), _p(ru), _p(ps),
                             B, _p(lo), _p(hi), _p(l_in), _p(u_in), _p(so), _p(si), _p(ro), _p(Gx), _p(hx),
                             m, _p(Cx), _p(tx), _p(al), int(alpha_mode), _p(to), _p(ti),
                             int(relaxed), int(sweeps), int(enforce_splits),
                             _p(out["lower"]), _p(out["lower_scale"]), _p(out["lo_clip"]), _p(out["hi_clip"]),
                             _p(out["l"]), _p(out["u"]), _p(out["l_scale"]), _p(out["u_scale"]),
                             _p(out["mask"]), _p(out["infeasible"]), _p(out["verified"]), _p(fA), _p(fc),
                             _p(bw), int(nthreads))
    assert rc == 0
    if U == 0:
        for k in ("l", "u", "l_scale", "u_scale", "mask"):
            out[k] = out[k][:, :0]
    if want_final:
        out["final_A"], out["final_c"] = fA, fc
    if want_weight:
        out["babsr_weight"] = bw[:, :U]
    return out


def alpha_grad(net: Net, hl, hu, hs, lo, hi, C, t, alpha, grad_f=None, beta=None, bsign=None, zmag=None,
               want_scale=False):
    """f [m] and d(sum grad_f*f)/d alpha [m x H] for one subdomain; with split multipliers beta [m x H]
    and split signs bsign [H] (+1: z >= 0, -1: z <= 0, 0: none) also d/d beta [m x H]; with want_scale,
    last, the bounds' magnitude scales [m] (hidden magnitudes zmag, default max(|hl|, |hu|))."""
    lib = _load()
    m = int(np.asarray(C).shape[0])
    hl, hu, lo, hi, Cx, tx, al = _f64(hl), _f64(hu), _f64(lo), _f64(hi), _f64(C), _f64(t), _f64(alpha)
    hs = np.ascontiguousarray(np.asarray(hs, np.int8))
    gf = None if grad_f is None else _f64(grad_f)
    f = np.zeros(m)
    g = np.zeros((m, net.H))
    bt = None if beta is None else _f64(beta)
    bs = None if beta is None else np.ascontiguousarray(np.asarray(bsign, np.int8))
    gb = None if beta is None else np.zeros((m, net.H))
    zm = None if zmag is None else _f64(zmag)
    sc = np.zeros(m) if want_scale else None
    rc = lib.orc_alpha_grad(net.L, _p(net.dims), _p(net.Wflat), _p(net.bflat), _p(hl), _p(hu), _p(hs),
                            _p(lo), _p(hi), m, _p(Cx), _p(tx), _p(al), _p(gf), _p(f), _p(g), _p(bt), _p(bs), _p(gb),
                            _p(zm), _p(sc))
    assert rc == 0
    out = (f, g) if beta is None else (f, g, gb)
    return out + (sc,) if want_scale else out


def adam_step_range(x, m1, m2, g, t, lr, lo, hi, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam ascent step with clamp to [lo, hi] on float64 arrays."""
    lib = _load()
    for a in (x, m1, m2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib.orc_adam_step_range(x.size, _p(x), _p(m1), _p(m2), _p(_f64(g)), int(t), float(lr), float(b1), float(b2),
                            float(eps), float(lo), float(hi))


def adam_step(alpha, m1, m2, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam ascent step with clamp to [0,1] on float64 arrays."""
    lib = _load()
    for a in (alpha, m1, m2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib.orc_adam_step(alpha.size, _p(alpha), _p(m1), _p(m2), _p(g), int(t), float(lr), float(b1),
                      float(b2), float(eps))


def _babsr_scores(l, u, mask, w):
    """The BaBSR scores as orc_activation_split / orc_select_targets take them (FP32, -1 for stable
    neurons), for the near-tie margins only."""
    l, u = np.asarray(l, np.float32), np.asarray(u, np.float32)
    un = (np.asarray(mask) == 0) & (l < 0) & (u > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (np.maximum(np.float32(0), -l) * np.maximum(np.float32(0), u)) / (u - l)
    if w is not None:
        s = s * np.maximum(np.float32(0), -np.asarray(w, np.float32))
    return np.where(un, s, np.float32(-1)).astype(np.float32)


def activation_bab(net: Net, cache, lo0, hi0, C, t, *, batch, top_k, capacity, max_depth, max_iters,
                   relaxed=1, sweeps=10, enforce_splits=1, alpha_mode=0):
    """Algorithm 5 (Clip-and-Verify for activation branch and bound) with the oracle's steps, one
    iteration after another in the paper's order:
      Init             a round on the B0 initial domains (no splits), Domain_Filter
      Batch_Pick_Out   the last P = min(batch, |D|, capacity - |D|) domains of the list
      Batch_Split      activation_split on them (BaBSR score with the stored weight)
      Top-K_Heuristic  select_targets on the children (parent's bounds, parent's mask with the new
                       split fixed, parent's weight); top_k < 0: every unstable neuron
      Domain_Clipper / Domain_Update / Solve_Bound   bound_batch on the children (want_weight)
      Domain_Filter    drop verified, infeasible and (unverified) max_depth children; push the rest
    The list is a stack (the pick order is a reading: the paper leaves it open).  Returns a dict:
      iters [dicts of counts per call, Init first], lists [split-code lists of the list after each
      call], status ("verified" | "unknown"), and the near-tie margins of every decision taken:
      branch_gap (relative gap of the best score to the next), topk_gap (at the k-th place of each
      layer), lower_gap (|lower_min| / its scale for the verified decisions)."""
    lo0, hi0 = np.atleast_2d(_f64(lo0)), np.atleast_2d(_f64(hi0))
    ids = np.asarray(cache["ids"])
    U = ids.size
    lay = layer_of_slots(net, ids)
    m = np.asarray(C).shape[0]
    D = []          # the stack: dicts(codes, lo, hi, l, u, mask, w, lmin)
    rec = dict(iters=[], lists=[], branch_gap=[], topk_gap=[], lower_gap=[])

    def filter_push(out, codes, lo, hi):
        st = dict(verified=0, infeasible=0, depth_limited=0, pushed=0, lower_min=np.inf)
        for k in range(len(codes)):
            lm = float(np.min(out["lower"][k])) if m else np.inf
            inf, ver = bool(out["infeasible"][k]), bool(out["verified"][k])
            if not inf:
                scale = float(np.max(out["lower_scale"][k]))
                rec["lower_gap"].append(abs(lm) / max(scale, 1e-300))
            if inf:
                st["infeasible"] += 1
            elif ver:
                st["verified"] += 1
            elif len(codes[k]) >= max_depth:
                st["depth_limited"] += 1
            else:
                st["pushed"] += 1
                st["lower_min"] = min(st["lower_min"], lm)
                D.append(dict(codes=list(codes[k]), lo=out["lo_clip"][k].copy(), hi=out["hi_clip"][k].copy(),
                              l=out["l"][k].copy(), u=out["u"][k].copy(), mask=out["mask"][k].copy(),
                              w=out["babsr_weight"][k].copy(), lmin=lm))
        return st

    def snapshot(st):
        st["remaining"] = len(D)
        rec["iters"].append(st)
        rec["lists"].append([list(d["codes"]) for d in D])

    out = bound_batch(net, cache, lo0, hi0, C=C, t=t, relaxed=relaxed, sweeps=sweeps,
                      enforce_splits=enforce_splits, alpha_mode=alpha_mode, want_weight=True)
    st = filter_push(out, [[] for _ in range(lo0.shape[0])], lo0, hi0)
    st.update(picked=0, stuck=0, children=lo0.shape[0])
    snapshot(st)
    for _ in range(max_iters):
        if not D:
            break
        P = min(batch, len(D), capacity - len(D))
        if P <= 0:
            raise RuntimeError("domain list full")
        parents = D[len(D) - P:]
        del D[len(D) - P:]
        st = dict(picked=P, stuck=0, children=0)
        if U == 0:
            st.update(stuck=P, verified=0, infeasible=0, depth_limited=0, pushed=0, lower_min=np.inf)
            snapshot(st)
            continue
        so = np.concatenate([[0], np.cumsum([len(p["codes"]) for p in parents])]).astype(np.int32)
        si = np.array([c for p in parents for c in p["codes"]], np.int32)
        L_ = np.array([p["l"] for p in parents]); U_ = np.array([p["u"] for p in parents])
        Mk = np.array([p["mask"] for p in parents]); W_ = np.array([p["w"] for p in parents])
        sp = activation_split(ids, so, si, np.array([p["lo"] for p in parents]), np.array([p["hi"] for p in parents]),
                              L_, U_, Mk, W_, np.zeros(P), np.zeros(P))
        st["stuck"] = int(np.sum(sp["stuck"]))
        for b in range(P):   # the branching decisions' margins
            sc = _babsr_scores(L_[b], U_[b], Mk[b], W_[b])
            top = np.sort(sc)[::-1]
            if top.size >= 2 and top[0] > 0:      # (ties at a zero weight factor are exact on any side)
                rec["branch_gap"].append(float((top[0] - top[1]) / top[0]))
        n = sp["parent"].size
        st["children"] = n
        if n == 0:
            st.update(verified=0, infeasible=0, depth_limited=0, pushed=0, lower_min=np.inf)
            snapshot(st)
            continue
        codes, lo_c, hi_c, l_c, u_c, mk_c, w_c = [], [], [], [], [], [], []
        for k in range(n):
            p = parents[sp["parent"][k]]
            br = int(sp["branched"][k])
            side = 1 if (k & 1) else -1
            codes.append(p["codes"] + [side * (int(ids[br]) + 1)])
            lo_c.append(p["lo"]); hi_c.append(p["hi"]); l_c.append(p["l"]); u_c.append(p["u"])
            mk = p["mask"].copy(); mk[br] = side
            mk_c.append(mk); w_c.append(p["w"])
        l_c, u_c, mk_c, w_c = np.array(l_c), np.array(u_c), np.array(mk_c, np.int8), np.array(w_c)
        tgt_off = tgt_ids = None
        if top_k >= 0:
            tgt_off, tgt_ids = select_targets(lay, l_c, u_c, mk_c, w_c, top_k)
            for k in range(n):   # the k-th place of every layer
                sc = _babsr_scores(l_c[k], u_c[k], mk_c[k], w_c[k])
                for h in np.unique(lay):
                    v = np.sort(sc[(lay == h) & (sc >= 0)])[::-1]
                    if v.size > top_k >= 1 and v[top_k - 1] > 0:
                        rec["topk_gap"].append(float((v[top_k - 1] - v[top_k]) / v[top_k - 1]))
        so_c = np.concatenate([[0], np.cumsum([len(c) for c in codes])]).astype(np.int32)
        si_c = np.array([c for cs in codes for c in cs], np.int32)
        out = bound_batch(net, cache, np.array(lo_c), np.array(hi_c), l_in=l_c, u_in=u_c, split_off=so_c,
                          split_ids=si_c, C=C, t=t, tgt_off=tgt_off, tgt_ids=tgt_ids, relaxed=relaxed, sweeps=sweeps,
                          enforce_splits=enforce_splits, alpha_mode=alpha_mode, want_weight=True)
        st.update(filter_push(out, codes, None, None))
        snapshot(st)
    rec["status"] = "verified" if not D and all(s["stuck"] == 0 and s["depth_limited"] == 0
                                                 for s in rec["iters"]) else "unknown"
    rec["remaining"] = len(D)
    return rec
