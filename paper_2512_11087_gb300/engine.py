"""Device-memory plumbing around the C-ABI: allocates a round's outputs and workspace with
torch and calls cv_bound_batch.  Every step of the round runs in the library's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import capi


def to_dev(x, dtype=None, device="cuda"):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype or x.dtype).contiguous()
    a = np.ascontiguousarray(x)
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device).contiguous()


class Net:
    """A network on the device (cv_net) plus its root cache (cv_cache)."""

    def __init__(self, layers):
        self.handle = capi.cv_net_create(layers)
        self.dims, self.H = capi.cv_net_dims(self.handle)
        self.n0, self.nL = self.dims[0], self.dims[-1]
        self.cache = None
        self.U = 0

    def build_cache(self, root_lo, root_hi, alpha_mode=capi.CV_ALPHA_ADAPTIVE):
        lo = to_dev(root_lo, torch.float32)
        hi = to_dev(root_hi, torch.float32)
        self._drop_cache()
        self.cache = capi.cv_cache_build(self.handle, lo, hi, alpha_mode)
        self.U = capi.cv_cache_size(self.cache)
        return self.U

    def set_cache(self, root_lo, root_hi, root_l, root_u, ids, lA, lc, uA, uc):
        self._drop_cache()
        self.cache = capi.cv_cache_create(self.handle, root_lo, root_hi, root_l, root_u, ids, lA, lc, uA, uc)
        self.U = capi.cv_cache_size(self.cache)
        return self.U

    def read_cache(self):
        return capi.cv_cache_read(self.cache, self.n0, self.H)

    def _drop_cache(self):
        if self.cache is not None:
            capi.cv_cache_destroy(self.cache)
            self.cache = None

    def close(self):
        self._drop_cache()
        if self.handle is not None:
            capi.cv_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Round:
    """Outputs and workspace for rounds of B subdomains with m spec rows."""

    def __init__(self, net: Net, B, m, max_splits=0, max_rows=0, relaxed=1, sweeps=0,
                 precision=capi.CV_PREC_FP32, alpha_mode=capi.CV_ALPHA_ADAPTIVE, enforce_splits=1,
                 want_final=False, want_weight=False, device="cuda"):
        self.net, self.B, self.m = net, B, m
        self.max_splits, self.max_rows = max_splits, max_rows
        self.opt = capi.cv_options_default()
        self.opt.relaxed, self.opt.sweeps, self.opt.precision = int(relaxed), int(sweeps), int(precision)
        self.opt.alpha_mode, self.opt.enforce_splits = int(alpha_mode), int(enforce_splits)
        self.opt.babsr_weight = 1 if want_weight else 0
        n0, U = net.n0, max(net.U, 1)
        f32 = dict(dtype=torch.float32, device=device)
        self.out = dict(lower=torch.empty(B, m, **f32), lo_clip=torch.empty(B, n0, **f32),
                        hi_clip=torch.empty(B, n0, **f32), l=torch.empty(B, U, **f32),
                        u=torch.empty(B, U, **f32), mask=torch.empty(B, U, dtype=torch.int8, device=device),
                        infeasible=torch.empty(B, dtype=torch.uint8, device=device),
                        verified=torch.empty(B, dtype=torch.uint8, device=device),
                        err_bound=torch.empty(B, m, **f32))
        if want_final:
            self.out["final_A"] = torch.empty(B, m, n0, **f32)
            self.out["final_c"] = torch.empty(B, m, **f32)
        if want_weight:
            self.out["babsr_weight"] = torch.empty(B, U, **f32)
        probe = capi.make_batch_in(B, None, None, m, None, None, max_splits=max_splits, max_rows=max_rows)
        self.ws_bytes = capi.cv_bound_batch_workspace(net.handle, net.cache, probe, self.opt)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)
        self.bo = capi.make_batch_out(**self.out)
        self.timer = None

    def __del__(self):
        if getattr(self, "timer", None) is not None:
            try:
                capi.cv_timer_destroy(self.timer)
            except Exception:
                pass
            self.timer = None

    def enable_timer(self):
        """Record phase times and complete clipping's counters on every later call (cv_timer)."""
        if self.timer is None:
            self.timer = capi.cv_timer_create()
            self.opt.timer = self.timer
        return self

    def cc_stats(self):
        """(row steps, certified row steps, with several candidates, widened, left with the FP32 decision,
        of those over the candidate limit) of the last call run with the timer."""
        _, _, steps = capi.cv_timer_read(self.timer)
        return (steps,) + capi.cv_timer_read_cc(self.timer)

    def _bi(self, lo, hi, C, t, l_in, u_in, split_off, split_ids, row_off, G, h, alpha, tgt_off, tgt_ids):
        return capi.make_batch_in(self.B, lo, hi, self.m, C, t, l_in=l_in, u_in=u_in, split_off=split_off,
                                  split_ids=split_ids, max_splits=self.max_splits, row_off=row_off, G=G, h=h,
                                  max_rows=self.max_rows, alpha=alpha, tgt_off=tgt_off, tgt_ids=tgt_ids)

    def run(self, lo, hi, C, t, l_in=None, u_in=None, split_off=None, split_ids=None, row_off=None, G=None,
            h=None, alpha=None, tgt_off=None, tgt_ids=None, stream=None):
        """All array arguments must already be device tensors (see to_dev)."""
        bi = self._bi(lo, hi, C, t, l_in, u_in, split_off, split_ids, row_off, G, h, alpha, tgt_off, tgt_ids)
        capi.cv_bound_batch(self.net.handle, self.net.cache, bi, self.bo, self.opt, self.ws, self.ws_bytes,
                            stream)
        return self.out

    def spec_clip(self, lo, hi, C, t, l_in=None, u_in=None, split_off=None, split_ids=None, row_off=None, G=None,
                  h=None, alpha=None, tgt_off=None, tgt_ids=None, stream=None):
        """After run() on the same inputs (with want_final): complete clipping of the spec rows' final
        planes (cv_spec_clip); raises out["lower"] and updates out["verified"] in place."""
        bi = self._bi(lo, hi, C, t, l_in, u_in, split_off, split_ids, row_off, G, h, alpha, tgt_off, tgt_ids)
        n = capi.cv_spec_clip_workspace(self.net.handle, self.net.cache, bi)
        if getattr(self, "_sws", None) is None or self._sws.numel() < max(n, 256):
            self._sws = torch.empty(max(n, 256), dtype=torch.uint8, device=self.ws.device)
        capi.cv_spec_clip(self.net.handle, self.net.cache, bi, self.bo, self.opt, self._sws, n, stream)
        return self.out

    def autotune(self, lo, hi, C, t, l_in=None, u_in=None, split_off=None, split_ids=None, row_off=None, G=None,
                 h=None, alpha=None, tgt_off=None, tgt_ids=None, stream=None):
        """Tunes complete clipping's work-item sizes on this batch (cv_autotune_cc); the sizes stay in
        the network's cache.  Returns (sizes, their complete-clipping time in ms)."""
        bi = self._bi(lo, hi, C, t, l_in, u_in, split_off, split_ids, row_off, G, h, alpha, tgt_off, tgt_ids)
        return capi.cv_autotune_cc(self.net.handle, self.net.cache, bi, self.bo, self.opt, self.ws, self.ws_bytes,
                                   stream)

    def capture(self, lo, hi, C, t, l_in=None, u_in=None, split_off=None, split_ids=None, row_off=None, G=None,
                h=None, alpha=None, tgt_off=None, tgt_ids=None):
        """CUDA graph of a round on these (device) buffers; replay with replay().  The tensors passed
        here are kept alive with the graph."""
        self._graph_keep = (lo, hi, C, t, l_in, u_in, split_off, split_ids, row_off, G, h, alpha, tgt_off, tgt_ids)
        bi = self._bi(*self._graph_keep)
        self.graph = capi.cv_graph_capture(self.net.handle, self.net.cache, bi, self.bo, self.opt, self.ws,
                                           self.ws_bytes)
        return self.graph

    def replay(self, stream=None):
        capi.cv_graph_launch(self.graph, stream)
        return self.out


class AlphaBound(torch.autograd.Function):
    """Spec lower bounds as a differentiable function of the slopes alpha [B x m x H].

    Forward and backward both run in the library (cv_alpha_grad): the forward computes the
    bounds and the gradient of sum f (each bound row depends only on its own slope row, so the
    gradient for any upstream gradient is that one scaled row by row); backward applies the
    upstream gradient."""

    @staticmethod
    def forward(ctx, alpha, state):
        lower, grad = state.bound_and_grad(alpha)
        ctx.save_for_backward(grad)
        return lower

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad * grad_out.unsqueeze(-1), None


class AlphaState:
    """Inputs that stay fixed during slope optimisation, plus the workspace."""

    def __init__(self, net: Net, lo, hi, l, u, mask, C, t, precision=capi.CV_PREC_FP32, split_sign=None):
        """split_sign [B x H] int8 (split_signs()) enables split multipliers beta in bound_and_grad."""
        self.net = net
        self.precision = int(precision)
        self.split_sign = split_sign
        self.B, self.n0 = lo.shape
        self.m = C.shape[0]
        self.lo, self.hi, self.l, self.u, self.mask, self.C, self.t = lo, hi, l, u, mask, C, t
        self.ws_bytes = capi.cv_alpha_grad_workspace(net.handle, self.B, self.m)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=lo.device)

    def bound_and_grad(self, alpha, grad_f=None, beta=None):
        """(lower, d/d alpha), and d/d beta as a third entry when split multipliers beta [B x m x H] are given."""
        lower = torch.empty(self.B, self.m, dtype=torch.float32, device=alpha.device)
        grad = torch.empty_like(alpha)
        gb = None
        if beta is not None:
            if self.split_sign is None:
                raise ValueError("split multipliers need the state's split_sign")
            beta = beta.detach().contiguous()
            gb = torch.empty_like(beta)
        ai = capi.make_alpha_in(self.B, self.m, self.lo, self.hi, self.l, self.u, self.mask, self.C, self.t,
                                alpha.detach().contiguous(), grad_f, precision=self.precision, beta=beta,
                                split_sign=self.split_sign if beta is not None else None, grad_beta=gb)
        capi.cv_alpha_grad(self.net.handle, self.net.cache, ai, lower, grad, self.ws, self.ws_bytes)
        return (lower, grad) if beta is None else (lower, grad, gb)


def optimize_alpha(state: AlphaState, alpha, steps=20, lr=0.1, decay=0.98, beta=None, beta_lr=None):
    """Adam ascent on the slopes (the paper's SDP-FO setting: 20 steps, lr 0.1, x0.98 per step), and on
    the split multipliers when beta is given (clamped to [0, inf), learning rate beta_lr or lr).
    Returns the final slopes (and multipliers) and the bound after each step (every step runs in
    library kernels)."""
    alpha = alpha.detach().clone().contiguous()
    m1 = torch.zeros_like(alpha)
    m2 = torch.zeros_like(alpha)
    if beta is not None:
        beta = beta.detach().clone().contiguous()
        n1, n2 = torch.zeros_like(beta), torch.zeros_like(beta)
    history = []
    for it in range(1, steps + 1):
        res = state.bound_and_grad(alpha, beta=beta)
        history.append(res[0])
        capi.cv_alpha_adam(alpha, m1, m2, res[1], it, lr * decay ** (it - 1))
        if beta is not None:
            capi.cv_adam_range(beta, n1, n2, res[2], it, (beta_lr or lr) * decay ** (it - 1), 0.0, float("inf"))
    history.append(state.bound_and_grad(alpha, beta=beta)[0])
    return (alpha, history) if beta is None else (alpha, beta, history)


def split_signs(net: Net, split_off, split_ids, B, stream=None):
    """[B x H] int8 split signs of a CSR split list (cv_split_signs): +1 for z >= 0, -1 for z <= 0."""
    sign = torch.empty(max(B, 1), max(net.H, 1), dtype=torch.int8, device="cuda")
    capi.cv_split_signs(net.handle, B, split_off, split_ids, sign, stream)
    return sign[:B, :net.H]


def input_split(lo, hi, final_A, final_c, lower, verified, infeasible, stream=None):
    """Input-BaB split step on device tensors (cv_input_split): returns dict(lo, hi [2K x n0],
    row_off [2K + 1], G [rows x n0], h [rows], parent [2K]) as device tensors."""
    B, n0 = lo.shape
    m = lower.shape[1]
    dev = lo.device
    f32 = dict(dtype=torch.float32, device=dev)
    lo2, hi2 = torch.empty(2 * max(B, 1), n0, **f32), torch.empty(2 * max(B, 1), n0, **f32)
    ro = torch.zeros(2 * B + 1, dtype=torch.int32, device=dev)
    G, h = torch.empty(2 * max(B, 1), n0, **f32), torch.empty(2 * max(B, 1), **f32)
    par = torch.empty(2 * max(B, 1), dtype=torch.int32, device=dev)
    nch = torch.zeros(1, dtype=torch.int32, device=dev)
    wsb = capi.cv_input_split_workspace(B)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
    capi.cv_input_split(B, n0, m, lo, hi, final_A, final_c, lower, verified, infeasible, lo2, hi2, ro, G, h, par,
                        nch, ws, wsb, stream)
    n = int(nch.item())
    nr = int(ro[n].item()) if n else 0
    return dict(lo=lo2[:n], hi=hi2[:n], row_off=ro[:n + 1], G=G[:nr], h=h[:nr], parent=par[:n])


def activation_split(net: Net, split_off, split_ids, lo, hi, l, u, mask, verified, infeasible, weight=None,
                     stream=None):
    """Activation-BaB split step on device tensors (cv_activation_split): dict(split_off, split_ids, lo, hi,
    l, u, parent, branched [children], stuck [B]) as device tensors."""
    B, n0 = lo.shape
    U = l.shape[1]
    dev = lo.device
    nsp = int(split_off[-1].item()) if split_off is not None and B else 0
    f32 = dict(dtype=torch.float32, device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    cap = 2 * max(B, 1)
    so2 = torch.zeros(2 * B + 1, **i32)
    si2 = torch.zeros(2 * (nsp + B) + 1, **i32)
    lo2, hi2 = torch.empty(cap, n0, **f32), torch.empty(cap, n0, **f32)
    l2, u2 = torch.empty(cap, U, **f32), torch.empty(cap, U, **f32)
    par, br = torch.empty(cap, **i32), torch.empty(cap, **i32)
    stuck = torch.zeros(max(B, 1), dtype=torch.uint8, device=dev)
    nch = torch.zeros(1, **i32)
    wsb = capi.cv_activation_split_workspace(B)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
    capi.cv_activation_split(net.handle, net.cache, B, split_off, split_ids, lo, hi, l, u, mask, weight, verified,
                             infeasible, so2, si2, lo2, hi2, l2, u2, par, br, stuck, nch, ws, wsb, stream)
    n = int(nch.item())
    ns = int(so2[n].item()) if n else 0
    return dict(split_off=so2[:n + 1], split_ids=si2[:ns], lo=lo2[:n], hi=hi2[:n], l=l2[:n], u=u2[:n],
                parent=par[:n], branched=br[:n], stuck=stuck[:B])


def select_targets(net: Net, l, u, mask, k, weight=None, stream=None):
    """Top-k BaBSR targets per subdomain and hidden layer (cv_select_targets): (tgt_off, tgt_ids)."""
    B, U = l.shape
    dev = l.device
    off = torch.zeros(B + 1, dtype=torch.int32, device=dev)
    ids = torch.empty(max(B * U, 1), dtype=torch.int32, device=dev)
    wsb = capi.cv_select_targets_workspace(B, U)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
    capi.cv_select_targets(net.handle, net.cache, B, l, u, mask, weight, k, off, ids, ws, wsb, stream)
    n = int(off[-1].item())
    return off, ids[:n]



class ActivationBaB:
    """The activation-BaB loop of Algorithm 5 on the GPU (cv_bab_*): a device-resident domain list,
    with every iteration's pick-out, split, top-k targets, round and filter in the library's kernels.
    C, t: the spec rows (device tensors or host arrays, kept on the device for the loop's lifetime)."""

    def __init__(self, net: Net, C, t, batch=1024, top_k=20, capacity=65536, max_depth=32, relaxed=1, sweeps=10,
                 precision=capi.CV_PREC_FP32, alpha_mode=capi.CV_ALPHA_ADAPTIVE, enforce_splits=1):
        self.net = net
        self.C = to_dev(C, torch.float32)
        self.t = to_dev(t, torch.float32)
        p = capi.cv_bab_params_default()
        p.batch, p.top_k, p.capacity, p.max_depth = int(batch), int(top_k), int(capacity), int(max_depth)
        p.opt.relaxed, p.opt.sweeps, p.opt.precision = int(relaxed), int(sweeps), int(precision)
        p.opt.alpha_mode, p.opt.enforce_splits = int(alpha_mode), int(enforce_splits)
        self.params = p
        self.handle = capi.cv_bab_create(net.handle, net.cache, self.C.shape[0], self.C, self.t, p)

    def init(self, lo, hi, stream=None):
        """Init: a round on the initial domains (device boxes [B0 x n0]), the survivors become the list."""
        self._keep = (to_dev(lo, torch.float32), to_dev(hi, torch.float32))
        return capi.cv_bab_init(self.handle, self._keep[0].shape[0], self._keep[0], self._keep[1], stream)

    def step(self, stream=None):
        return capi.cv_bab_step(self.handle, stream)

    def run(self, max_iters, stream=None):
        """(summed counts, iterations run) until the list is empty or max_iters."""
        return capi.cv_bab_run(self.handle, max_iters, stream)

    def domains(self, stream=None):
        """(split_off, split_ids, lower_min) of the list, on the host."""
        return capi.cv_bab_read(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            capi.cv_bab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def round_summary(out, stream=None):
    """(bounds [2] float32, counts [2] int32) device tensors of a round's outputs (cv_round_summary): the least
    spec lower bound over the feasible and over the unverified subdomains, the verified and infeasible counts."""
    B, m = out["lower"].shape
    bounds = torch.empty(2, dtype=torch.float32, device=out["lower"].device)
    counts = torch.empty(2, dtype=torch.int32, device=out["lower"].device)
    capi.cv_round_summary(B, m, out["lower"], out["verified"], out["infeasible"], bounds, counts, stream)
    return bounds, counts


def reduce_round_summary(bounds, counts, dist=None, group=None):
    """The job's summary over ranks (torch.distributed: min of the bounds, sum of the counts), as a dict.
    bounds / counts: this rank's (round_summary, or any tensors of that layout on the group's device)."""
    b, c = bounds.clone(), counts.to(torch.int64)
    if dist is not None and dist.is_initialized():
        dist.all_reduce(b, op=dist.ReduceOp.MIN, group=group)
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    b, c = b.cpu().tolist(), c.cpu().tolist()
    return dict(lower_min=b[0], lower_min_unverified=b[1], verified=int(c[0]), infeasible=int(c[1]))
