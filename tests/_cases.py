"""Seeded test cases shared by the parity tests: the inputs come from the workload generators
and (where bounds are needed to draw them) from the oracle, never from the CUDA path."""
import numpy as np

from oracle import oracle as O
from paper_2512_11087_gb300 import workloads as WL


def f32(x):
    return np.asarray(x, np.float32)


def rd32(x):
    """Round toward -inf onto the FP32 grid."""
    x = np.asarray(x, np.float64)
    f = x.astype(np.float32)
    f = np.where(f.astype(np.float64) > x, np.nextafter(f, np.float32(-np.inf)), f)
    return f.astype(np.float32)


def ru32(x):
    x = np.asarray(x, np.float64)
    f = x.astype(np.float32)
    f = np.where(f.astype(np.float64) < x, np.nextafter(f, np.float32(np.inf)), f)
    return f.astype(np.float32)


class Case:
    """A network, a root box, the oracle's root cache (as the FP32 arrays both sides use)
    and one round's batch."""

    def __init__(self, dims, B, kmin, kmax, eps, centre="unit", clip01=True, out_rows=0, seed=0,
                 m_spec=None, sweeps=0, relaxed=1, enforce=1, alpha_mode=0, layers=None, targets=None,
                 cut_rows=None):
        self.layers = layers if layers is not None else WL.he_mlp(dims, seed=seed)
        self.net = O.Net(self.layers)
        dims = list(self.net.dims)
        self.n0, self.nL = dims[0], dims[-1]
        self.lo0, self.hi0 = WL.box(self.n0, eps, seed=seed, centre=centre, clip01=clip01)
        root = O.root_crown(self.net, self.lo0, self.hi0, alpha_mode=alpha_mode)
        cache = O.make_cache(root)
        c32 = O.cache_as_f32(cache)
        c32["root_l"] = rd32(cache["root_l"]).astype(np.float64)
        c32["root_u"] = ru32(cache["root_u"]).astype(np.float64)
        self.root = root
        self.cache = c32
        self.U = cache["ids"].size
        self.B = B
        self.C, self.t = WL.margin_spec(self.nL, y=0) if m_spec is None else m_spec
        self.m = self.C.shape[0]
        self.lo, self.hi = WL.tile_box(self.lo0, self.hi0, B)
        self.split_off, self.split_ids = WL.draw_splits(cache["ids"], B, kmin, kmax, seed=seed + 1)
        self.max_splits = int(np.max(np.diff(self.split_off))) if B else 0
        self.row_off = self.G = self.h = None
        self.max_rows = 0
        if out_rows:
            # the root CROWN lower plane of the first spec row, shifted to cut each box (input-BaB rows)
            o = O.bound_batch(self.net, c32, self.lo0[None].astype(np.float64), self.hi0[None].astype(np.float64),
                              C=self.C[:1], t=self.t[:1], relaxed=0, sweeps=0, want_final=True)
            a = o["final_A"][0, 0]
            self.row_off, self.G, self.h = WL.shifted_plane_rows(a, 0.0, self.lo, self.hi, B, seed=seed + 2)
            self.max_rows = 1
        if cut_rows is not None:
            # kmin..kmax random rows cutting each box (several active rows per subdomain)
            self.row_off, self.G, self.h = WL.random_cut_rows(self.lo, self.hi, B, cut_rows[0], cut_rows[1],
                                                               seed=seed + 4)
            self.max_rows = int(np.max(np.diff(self.row_off))) if B else 0
        self.tgt_off = self.tgt_ids = None
        if targets is not None and self.U:
            self.tgt_off, self.tgt_ids = WL.random_targets(self.U, B, targets, seed=seed + 3)
        self.sweeps, self.relaxed, self.enforce, self.alpha_mode = sweeps, relaxed, enforce, alpha_mode

    def oracle(self, **kw):
        args = dict(split_off=self.split_off, split_ids=self.split_ids, row_off=self.row_off, G=self.G, h=self.h,
                    C=self.C, t=self.t, relaxed=self.relaxed, sweeps=self.sweeps, enforce_splits=self.enforce,
                    alpha_mode=self.alpha_mode, tgt_off=self.tgt_off, tgt_ids=self.tgt_ids)
        args.update(kw)
        return O.bound_batch(self.net, self.cache, self.lo.astype(np.float64), self.hi.astype(np.float64), **args)
