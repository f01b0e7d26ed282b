"""Thin Python binding of libclipverify.so (the C-ABI in include/clipverify.h).

Functions carry the C names and only marshal arguments: torch CUDA tensors become device
pointers, numpy arrays become host pointers, None becomes NULL, and a non-OK status raises
CVError with the library's message.  PyTorch is used only for device memory and streams.
There is no fallback: if the library is missing every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libclipverify.so")

CV_OK = 0
CV_LAYER_DENSE = 0
CV_LAYER_CONV2D = 1
CV_PREC_FP32 = 0
CV_PREC_BF16X8 = 1
CV_RELAX_OFF = 0
CV_RELAX_PARALLEL = 1
CV_RELAX_SEQUENTIAL = 2
CV_RELAX_SEQUENTIAL_ORDERED = 3
CV_ALPHA_ADAPTIVE = 0
CV_ALPHA_ONE = 1
CV_ALPHA_ZERO = 2
CV_EINVAL, CV_ESHAPE, CV_ENAN, CV_ECUDA, CV_ETIMEOUT, CV_ENOMEM, CV_EUNSUPPORTED, CV_EWORKSPACE, CV_EDEVICE = range(1, 10)
STATUS_NAMES = {0: "CV_OK", 1: "CV_EINVAL", 2: "CV_ESHAPE", 3: "CV_ENAN", 4: "CV_ECUDA", 5: "CV_ETIMEOUT",
                6: "CV_ENOMEM", 7: "CV_EUNSUPPORTED", 8: "CV_EWORKSPACE", 9: "CV_EDEVICE"}

P = ctypes.c_void_p
I = ctypes.c_int


class CVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class cv_layer_desc(ctypes.Structure):
    _fields_ = [("kind", I), ("in_c", I), ("in_h", I), ("in_w", I), ("out_c", I), ("out_h", I), ("out_w", I),
                ("k", I), ("stride", I), ("pad", I), ("weight", P), ("bias", P)]


class cv_options(ctypes.Structure):
    _fields_ = [("relaxed", I), ("sweeps", I), ("precision", I), ("alpha_mode", I), ("enforce_splits", I),
                ("timer", P), ("babsr_weight", I)]


class cv_batch_in(ctypes.Structure):
    _fields_ = [("B", I), ("lo", P), ("hi", P), ("l_in", P), ("u_in", P), ("split_off", P), ("split_ids", P),
                ("max_splits", I), ("row_off", P), ("G", P), ("h", P), ("max_rows", I), ("m", I), ("C", P),
                ("t", P), ("alpha", P), ("tgt_off", P), ("tgt_ids", P)]


class cv_alpha_in(ctypes.Structure):
    _fields_ = [("B", I), ("m", I), ("lo", P), ("hi", P), ("l", P), ("u", P), ("mask", P), ("C", P), ("t", P),
                ("alpha", P), ("grad_f", P), ("precision", I), ("beta", P), ("split_sign", P), ("grad_beta", P)]


class cv_bab_params(ctypes.Structure):
    _fields_ = [("batch", I), ("top_k", I), ("capacity", I), ("max_depth", I), ("opt", cv_options)]


class cv_bab_stats(ctypes.Structure):
    _fields_ = [("picked", I), ("stuck", I), ("children", I), ("verified", I), ("infeasible", I),
                ("depth_limited", I), ("pushed", I), ("remaining", I), ("lower_min", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cv_batch_out(ctypes.Structure):
    _fields_ = [("lower", P), ("lo_clip", P), ("hi_clip", P), ("l", P), ("u", P), ("mask", P),
                ("infeasible", P), ("verified", P), ("err_bound", P), ("final_A", P), ("final_c", P),
                ("babsr_weight", P)]


_lib = None


def load():
    """The loaded library; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libclipverify.so not found at {LIB_PATH}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    sigs = {
        "cv_last_error": ([], ctypes.c_char_p),
        "cv_net_create": ([P, I, ctypes.POINTER(P)], I),
        "cv_net_destroy": ([P], None),
        "cv_net_dims": ([P, P, P, P], I),
        "cv_device_status": ([P, P, P], I),
        "cv_cache_build": ([P, P, P, I, ctypes.POINTER(P), P], I),
        "cv_cache_create": ([P, P, P, P, P, I, P, P, P, P, P, ctypes.POINTER(P)], I),
        "cv_cache_size": ([P, P], I),
        "cv_cache_read": ([P, P, P, P, P, P, P, P], I),
        "cv_cache_destroy": ([P], None),
        "cv_options_default": ([P], None),
        "cv_bound_batch_workspace": ([P, P, P, P, P], I),
        "cv_batch_check": ([P, P, P, P, P], I),
        "cv_fp32_fma_peak": ([P, P, P], I),
        "cv_bound_batch": ([P, P, P, P, P, P, ctypes.c_size_t, P], I),
        "cv_timer_create": ([ctypes.POINTER(P)], I),
        "cv_timer_destroy": ([P], None),
        "cv_timer_read": ([P, P, P, P], I),
        "cv_timer_read_cc": ([P, P], I),
        "cv_relaxed_clip_static": ([P, P, P, P, P, P, I, P], I),
        "cv_graph_capture": ([P, P, P, P, P, P, ctypes.c_size_t, ctypes.POINTER(P)], I),
        "cv_graph_launch": ([P, P], I),
        "cv_graph_destroy": ([P], None),
        "cv_alpha_grad_workspace": ([P, I, I, P], I),
        "cv_alpha_grad": ([P, P, P, P, P, P, ctypes.c_size_t, P], I),
        "cv_alpha_adam": ([P, P, P, P, ctypes.c_longlong, I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, P], I),
        "cv_cc_items_set": ([P, P], I),
        "cv_cc_items_get": ([P, P], I),
        "cv_autotune_cc": ([P, P, P, P, P, P, ctypes.c_size_t, P, P, P], I),
        "cv_spec_clip_workspace": ([P, P, P, P], I),
        "cv_spec_clip": ([P, P, P, P, P, P, ctypes.c_size_t, P], I),
        "cv_activation_split_workspace": ([I, P], I),
        "cv_activation_split": ([P, P, I] + [P] * 21 + [ctypes.c_size_t, P], I),
        "cv_select_targets_workspace": ([I, I, P], I),
        "cv_select_targets": ([P, P, I, P, P, P, P, I, P, P, P, ctypes.c_size_t, P], I),
        "cv_round_summary": ([I, I, P, P, P, P, P, P], I),
        "cv_split_signs": ([P, I, P, P, P, P], I),
        "cv_adam_range": ([P, P, P, P, ctypes.c_longlong, I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, ctypes.c_float, ctypes.c_float, P], I),
        "cv_bab_params_default": ([P], None),
        "cv_bab_create": ([P, P, I, P, P, P, ctypes.POINTER(P)], I),
        "cv_bab_init": ([P, I, P, P, P, P], I),
        "cv_bab_step": ([P, P, P], I),
        "cv_bab_run": ([P, I, P, P, P], I),
        "cv_bab_read": ([P, P, P, P, P, P], I),
        "cv_bab_destroy": ([P], None),
        "cv_input_split_workspace": ([I, P], I),
        "cv_input_split": ([I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_size_t, P], I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return [n for n in ("cv_last_error", "cv_net_create", "cv_net_destroy", "cv_net_dims", "cv_device_status",
                        "cv_cache_build", "cv_cache_create", "cv_cache_size", "cv_cache_read", "cv_cache_destroy",
                        "cv_options_default", "cv_bound_batch_workspace", "cv_batch_check", "cv_fp32_fma_peak", "cv_bound_batch", "cv_timer_create",
                        "cv_timer_destroy", "cv_timer_read", "cv_timer_read_cc", "cv_relaxed_clip_static", "cv_alpha_grad_workspace",
                        "cv_alpha_grad", "cv_alpha_adam", "cv_graph_capture", "cv_graph_launch", "cv_graph_destroy",
                        "cv_cc_items_set", "cv_cc_items_get", "cv_autotune_cc", "cv_input_split_workspace",
                        "cv_input_split", "cv_spec_clip_workspace", "cv_spec_clip",
                        "cv_activation_split_workspace", "cv_activation_split", "cv_select_targets_workspace",
                        "cv_select_targets", "cv_bab_params_default", "cv_bab_create", "cv_bab_init",
                        "cv_bab_step", "cv_bab_run", "cv_bab_read", "cv_bab_destroy", "cv_round_summary",
                        "cv_split_signs", "cv_adam_range")]


def _check(st):
    if st != CV_OK:
        raise CVError(st, load().cv_last_error().decode(errors="replace"))


def ptr(x):
    """Device pointer of a torch tensor, host pointer of a numpy array, NULL for None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(P)
    return P(x.data_ptr())


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return P(s.cuda_stream)


# ---------------------------------------------------------------- entry points
def cv_net_create(layers):
    """layers: list of dicts from workloads.he_mlp / he_cnn (numpy float32 weights)."""
    lib = load()
    descs = (cv_layer_desc * len(layers))()
    keep = []
    for i, ly in enumerate(layers):
        W = np.ascontiguousarray(ly["W"], np.float32)
        b = np.ascontiguousarray(ly["b"], np.float32)
        keep += [W, b]
        d = descs[i]
        d.kind = ly["kind"]
        if ly["kind"] == CV_LAYER_DENSE:
            d.in_c, d.out_c = W.shape[1], W.shape[0]
            d.in_h = d.in_w = d.out_h = d.out_w = 1
        else:
            d.in_c, d.in_h, d.in_w = ly["in_shape"]
            d.out_c, d.out_h, d.out_w = ly["out_shape"]
            d.k, d.stride, d.pad = W.shape[2], ly["stride"], ly["pad"]
        d.weight = W.ctypes.data_as(P)
        d.bias = b.ctypes.data_as(P)
    h = P()
    _check(lib.cv_net_create(ctypes.cast(descs, P), len(layers), ctypes.byref(h)))
    return h


def cv_net_destroy(h):
    load().cv_net_destroy(h)


def cv_net_dims(h):
    lib = load()
    L = ctypes.c_int()
    _check(lib.cv_net_dims(h, ctypes.byref(L), None, None))
    dims = (ctypes.c_int * (L.value + 1))()
    H = ctypes.c_int()
    _check(lib.cv_net_dims(h, None, ctypes.cast(dims, P), ctypes.byref(H)))
    return list(dims), H.value


def cv_device_status(h, stream=None):
    code = ctypes.c_int()
    _check(load().cv_device_status(h, stream_ptr(stream), ctypes.byref(code)))
    return code.value


def cv_cache_build(net, root_lo, root_hi, alpha_mode=CV_ALPHA_ADAPTIVE, stream=None):
    h = P()
    _check(load().cv_cache_build(net, ptr(root_lo), ptr(root_hi), int(alpha_mode), ctypes.byref(h),
                                 stream_ptr(stream)))
    return h


def cv_cache_create(net, root_lo, root_hi, root_l, root_u, ids, lA, lc, uA, uc):
    """All host numpy arrays (float32 / int32)."""
    arrs = [np.ascontiguousarray(a, np.float32) for a in (root_lo, root_hi, root_l, root_u)]
    ids = np.ascontiguousarray(ids, np.int32)
    planes = [np.ascontiguousarray(a, np.float32) for a in (lA, lc, uA, uc)]
    h = P()
    _check(load().cv_cache_create(net, *[ptr(a) for a in arrs], int(ids.size), ptr(ids),
                                  *[ptr(a) for a in planes], ctypes.byref(h)))
    return h


def cv_cache_size(cache):
    U = ctypes.c_int()
    _check(load().cv_cache_size(cache, ctypes.byref(U)))
    return U.value


def cv_cache_read(cache, n0, H):
    U = cv_cache_size(cache)
    out = dict(ids=np.zeros(U, np.int32), lA=np.zeros((U, n0), np.float32), lc=np.zeros(U, np.float32),
               uA=np.zeros((U, n0), np.float32), uc=np.zeros(U, np.float32), root_l=np.zeros(H, np.float32),
               root_u=np.zeros(H, np.float32))
    _check(load().cv_cache_read(cache, *[ptr(out[k]) if out[k].size else None
                                         for k in ("ids", "lA", "lc", "uA", "uc", "root_l", "root_u")]))
    return out


def cv_cache_destroy(cache):
    load().cv_cache_destroy(cache)


def cv_options_default():
    o = cv_options()
    load().cv_options_default(ctypes.byref(o))
    return o


def make_batch_in(B, lo, hi, m, C, t, l_in=None, u_in=None, split_off=None, split_ids=None, max_splits=0,
                  row_off=None, G=None, h=None, max_rows=0, alpha=None, tgt_off=None, tgt_ids=None):
    bi = cv_batch_in()
    bi.B, bi.m, bi.max_splits, bi.max_rows = int(B), int(m), int(max_splits), int(max_rows)
    for name, v in dict(lo=lo, hi=hi, l_in=l_in, u_in=u_in, split_off=split_off, split_ids=split_ids,
                        row_off=row_off, G=G, h=h, C=C, t=t, alpha=alpha, tgt_off=tgt_off,
                        tgt_ids=tgt_ids).items():
        setattr(bi, name, ptr(v))
    return bi


def make_batch_out(lower, lo_clip, hi_clip, l, u, mask, infeasible, verified, err_bound=None, final_A=None,
                   final_c=None, babsr_weight=None):
    bo = cv_batch_out()
    for name, v in dict(lower=lower, lo_clip=lo_clip, hi_clip=hi_clip, l=l, u=u, mask=mask,
                        infeasible=infeasible, verified=verified, err_bound=err_bound, final_A=final_A,
                        final_c=final_c, babsr_weight=babsr_weight).items():
        setattr(bo, name, ptr(v))
    return bo


def cv_batch_check(net, cache, bi, stream=None):
    """(status, bits) of the device-side input check; does not raise."""
    code = ctypes.c_int()
    st = load().cv_batch_check(net, cache, ctypes.byref(bi), ctypes.byref(code), stream_ptr(stream))
    return st, code.value


def cv_fp32_fma_peak(stream=None):
    """(lane FMAs per second, ms of the timed launch) of the FFMA probe kernel."""
    v = ctypes.c_double()
    ms = ctypes.c_float()
    _check(load().cv_fp32_fma_peak(ctypes.byref(v), ctypes.byref(ms), stream_ptr(stream)))
    return v.value, ms.value


def cv_device_status_raw(net, stream=None):
    """(status, raw device status word) without raising."""
    code = ctypes.c_int()
    st = load().cv_device_status(net, stream_ptr(stream), ctypes.byref(code))
    return st, code.value


def cv_bound_batch_workspace(net, cache, bi, opt):
    n = ctypes.c_size_t()
    _check(load().cv_bound_batch_workspace(net, cache, ctypes.byref(bi), ctypes.byref(opt), ctypes.byref(n)))
    return n.value


def cv_bound_batch(net, cache, bi, bo, opt, workspace, workspace_bytes, stream=None):
    _check(load().cv_bound_batch(net, cache, ctypes.byref(bi), ctypes.byref(bo), ctypes.byref(opt),
                                 ptr(workspace), int(workspace_bytes), stream_ptr(stream)))


N_PHASES = 4


def cv_timer_create():
    h = P()
    _check(load().cv_timer_create(ctypes.byref(h)))
    return h


def cv_timer_destroy(t):
    load().cv_timer_destroy(t)


def cv_timer_read(t):
    """(per-phase ms list, kernel launches, complete-clipping row steps) of the last timed call."""
    ms = (ctypes.c_float * N_PHASES)()
    n = ctypes.c_int()
    steps = ctypes.c_longlong()
    _check(load().cv_timer_read(t, ctypes.cast(ms, P), ctypes.byref(n), ctypes.byref(steps)))
    return list(ms), n.value, steps.value


def cv_timer_read_cc(t):
    """Complete clipping's decision counters of the last timed call: (certified row steps, with several
    candidates, with a widened window, left with the FP32 decision, of those over the candidate limit)."""
    st = (ctypes.c_longlong * 5)()
    _check(load().cv_timer_read_cc(t, ctypes.cast(st, P)))
    return tuple(int(v) for v in st)


def cv_spec_clip_workspace(net, cache, bi):
    n = ctypes.c_size_t()
    _check(load().cv_spec_clip_workspace(net, cache, ctypes.byref(bi), ctypes.byref(n)))
    return n.value


def cv_spec_clip(net, cache, bi, bo, opt, workspace, workspace_bytes, stream=None):
    """Complete clipping of the spec rows' final planes after a round (see the header)."""
    _check(load().cv_spec_clip(net, cache, ctypes.byref(bi), ctypes.byref(bo), ctypes.byref(opt), ptr(workspace),
                               int(workspace_bytes), stream_ptr(stream)))


def cv_activation_split_workspace(B):
    n = ctypes.c_size_t()
    _check(load().cv_activation_split_workspace(int(B), ctypes.byref(n)))
    return n.value


def cv_activation_split(net, cache, B, split_off, split_ids, lo, hi, l, u, mask, weight, verified, infeasible,
                        split_off_out, split_ids_out, lo_out, hi_out, l_out, u_out, parent, branched, stuck,
                        n_children, workspace, workspace_bytes, stream=None):
    """Activation-BaB split step (Algorithm 5, BaBSR branching); device tensors (see the header)."""
    _check(load().cv_activation_split(net, cache, int(B), ptr(split_off), ptr(split_ids), ptr(lo), ptr(hi), ptr(l),
                                      ptr(u), ptr(mask), ptr(weight), ptr(verified), ptr(infeasible),
                                      ptr(split_off_out), ptr(split_ids_out), ptr(lo_out), ptr(hi_out), ptr(l_out),
                                      ptr(u_out), ptr(parent), ptr(branched), ptr(stuck), ptr(n_children),
                                      ptr(workspace), int(workspace_bytes), stream_ptr(stream)))


def cv_select_targets_workspace(B, U):
    n = ctypes.c_size_t()
    _check(load().cv_select_targets_workspace(int(B), int(U), ctypes.byref(n)))
    return n.value


def cv_select_targets(net, cache, B, l, u, mask, weight, k, tgt_off, tgt_ids, workspace, workspace_bytes,
                      stream=None):
    """Top-k BaBSR targets per subdomain and hidden layer (CSR of cache slots)."""
    _check(load().cv_select_targets(net, cache, int(B), ptr(l), ptr(u), ptr(mask), ptr(weight), int(k),
                                    ptr(tgt_off), ptr(tgt_ids), ptr(workspace), int(workspace_bytes),
                                    stream_ptr(stream)))


def cv_split_signs(net, B, split_off, split_ids, sign, stream=None):
    _check(load().cv_split_signs(net, int(B), ptr(split_off), ptr(split_ids), ptr(sign), stream_ptr(stream)))


def cv_adam_range(x, m1, m2, grad, t, lr, lo, hi, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().cv_adam_range(ptr(x), ptr(m1), ptr(m2), ptr(grad), int(x.numel()), int(t), float(lr), float(beta1),
                                float(beta2), float(eps), float(lo), float(hi), stream_ptr(stream)))


def cv_round_summary(B, m, lower, verified, infeasible, bounds, counts, stream=None):
    _check(load().cv_round_summary(int(B), int(m), ptr(lower), ptr(verified), ptr(infeasible), ptr(bounds),
                                   ptr(counts), stream_ptr(stream)))


def cv_bab_params_default():
    p = cv_bab_params()
    load().cv_bab_params_default(ctypes.byref(p))
    return p


def cv_bab_create(net, cache, m, C, t, params):
    h = P()
    _check(load().cv_bab_create(net, cache, int(m), ptr(C), ptr(t), ctypes.byref(params), ctypes.byref(h)))
    return h


def cv_bab_init(bab, B0, lo, hi, stream=None):
    st = cv_bab_stats()
    _check(load().cv_bab_init(bab, int(B0), ptr(lo), ptr(hi), stream_ptr(stream), ctypes.byref(st)))
    return st.as_dict()


def cv_bab_step(bab, stream=None):
    st = cv_bab_stats()
    _check(load().cv_bab_step(bab, stream_ptr(stream), ctypes.byref(st)))
    return st.as_dict()


def cv_bab_run(bab, max_iters, stream=None):
    st = cv_bab_stats()
    it = ctypes.c_int()
    _check(load().cv_bab_run(bab, int(max_iters), stream_ptr(stream), ctypes.byref(st), ctypes.byref(it)))
    return st.as_dict(), it.value


def cv_bab_read(bab, stream=None):
    """(split_off, split_ids, lower_min) of the domain list, host numpy arrays."""
    lib = load()
    n = ctypes.c_int()
    _check(lib.cv_bab_read(bab, ctypes.byref(n), None, None, None, stream_ptr(stream)))
    off = np.zeros(n.value + 1, np.int32)
    lm = np.zeros(n.value, np.float32)
    _check(lib.cv_bab_read(bab, None, off.ctypes.data, None, None, stream_ptr(stream)))
    ids = np.zeros(max(int(off[-1]), 1), np.int32)
    _check(lib.cv_bab_read(bab, None, None, ids.ctypes.data, lm.ctypes.data if n.value else None,
                           stream_ptr(stream)))
    return off, ids[:int(off[-1])], lm


def cv_bab_destroy(bab):
    load().cv_bab_destroy(bab)


def cv_input_split_workspace(B):
    n = ctypes.c_size_t()
    _check(load().cv_input_split_workspace(int(B), ctypes.byref(n)))
    return n.value


def cv_input_split(B, n0, m, lo, hi, final_A, final_c, lower, verified, infeasible, lo_out, hi_out, row_off, G, h,
                   parent, n_children, workspace, workspace_bytes, stream=None):
    """Input-BaB split step (Algorithm 4); all arrays are device tensors (see the header)."""
    _check(load().cv_input_split(int(B), int(n0), int(m), ptr(lo), ptr(hi), ptr(final_A), ptr(final_c), ptr(lower),
                                 ptr(verified), ptr(infeasible), ptr(lo_out), ptr(hi_out), ptr(row_off), ptr(G),
                                 ptr(h), ptr(parent), ptr(n_children), ptr(workspace), int(workspace_bytes),
                                 stream_ptr(stream)))


CC_ITEMS_DEFAULT = (256, 64, 16)


def cv_cc_items_set(cache, items):
    arr = (ctypes.c_int * 3)(*[int(v) for v in items])
    _check(load().cv_cc_items_set(cache, ctypes.cast(arr, P)))


def cv_cc_items_get(cache):
    arr = (ctypes.c_int * 3)()
    _check(load().cv_cc_items_get(cache, ctypes.cast(arr, P)))
    return list(arr)


def cv_autotune_cc(net, cache, bi, bo, opt, workspace, workspace_bytes, stream=None):
    """Times complete clipping of this batch over the item-size grid; keeps the fastest sizes in
    the cache and returns (sizes, their phase time in ms)."""
    best = (ctypes.c_int * 3)()
    ms = ctypes.c_float()
    _check(load().cv_autotune_cc(net, cache, ctypes.byref(bi), ctypes.byref(bo), ctypes.byref(opt),
                                 ptr(workspace), int(workspace_bytes), stream_ptr(stream), ctypes.cast(best, P),
                                 ctypes.byref(ms)))
    return list(best), ms.value


def cv_relaxed_clip_static(net, cache, bi, lo_clip, hi_clip, infeasible, relaxed=1, stream=None):
    """Rows, pre-check and relaxed clipping without any device allocation (scratch in the
    library's fixed device array); for callers that must not allocate device memory."""
    _check(load().cv_relaxed_clip_static(net, cache, ctypes.byref(bi), ptr(lo_clip), ptr(hi_clip), ptr(infeasible),
                                         int(relaxed), stream_ptr(stream)))


def make_alpha_in(B, m, lo, hi, l, u, mask, C, t, alpha, grad_f=None, precision=0, beta=None, split_sign=None,
                  grad_beta=None):
    ai = cv_alpha_in()
    ai.B, ai.m, ai.precision = int(B), int(m), int(precision)
    for name, v in dict(lo=lo, hi=hi, l=l, u=u, mask=mask, C=C, t=t, alpha=alpha, grad_f=grad_f, beta=beta,
                        split_sign=split_sign, grad_beta=grad_beta).items():
        setattr(ai, name, ptr(v))
    return ai


def cv_alpha_grad_workspace(net, B, m):
    n = ctypes.c_size_t()
    _check(load().cv_alpha_grad_workspace(net, int(B), int(m), ctypes.byref(n)))
    return n.value


def cv_alpha_grad(net, cache, ai, lower, grad_alpha, workspace, workspace_bytes, stream=None):
    _check(load().cv_alpha_grad(net, cache, ctypes.byref(ai), ptr(lower), ptr(grad_alpha), ptr(workspace),
                                int(workspace_bytes), stream_ptr(stream)))


def cv_alpha_adam(alpha, m1, m2, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().cv_alpha_adam(ptr(alpha), ptr(m1), ptr(m2), ptr(grad), int(alpha.numel()), int(t), float(lr),
                                float(beta1), float(beta2), float(eps), stream_ptr(stream)))


def cv_graph_capture(net, cache, bi, bo, opt, workspace, workspace_bytes):
    g = P()
    _check(load().cv_graph_capture(net, cache, ctypes.byref(bi), ctypes.byref(bo), ctypes.byref(opt), ptr(workspace),
                                   int(workspace_bytes), ctypes.byref(g)))
    return g


def cv_graph_launch(graph, stream=None):
    _check(load().cv_graph_launch(graph, stream_ptr(stream)))


def cv_graph_destroy(graph):
    load().cv_graph_destroy(graph)
