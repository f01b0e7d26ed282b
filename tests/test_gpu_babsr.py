"""Activation branch and bound with the BaBSR intercept score through the C-ABI: the split step
(cv_activation_split) and the top-k targets (cv_select_targets) bit-exact against the oracle on the
same inputs (integer decisions taken by both sides in FP32 in the same order), then one whole
activation-BaB iteration: a round, the branching, and the children's round with the inherited
bounds and the top-k targets, against the oracle at the parity bar."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402
from tests.test_gpu_parity import compare, gpu_round  # noqa: E402

pytestmark = pytest.mark.gpu


def _net(case):
    from paper_2512_11087_gb300 import engine as E
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    return net


def _random_bounds(rng, B, U, p_stable=0.4):
    l = rng.uniform(-2, 1, size=(B, U)).astype(np.float32)
    u = (l + rng.uniform(0.05, 3, size=(B, U))).astype(np.float32)
    mask = np.where(l >= 0, 1, np.where(u <= 0, -1, 0)).astype(np.int8)
    mask[rng.uniform(size=(B, U)) < p_stable] = -1
    return l, u, mask


def _dev(x, dt=torch.float32):
    return None if x is None else torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dt)


@pytest.mark.parametrize("B,weighted,seed", [(64, False, 1), (64, True, 2), (3001, True, 3), (1, False, 4)])
def test_activation_split_bit_exact(B, weighted, seed):
    from oracle import oracle as O
    from paper_2512_11087_gb300 import engine as E
    case = Case([12, 30, 30, 4], 2, 0, 0, 0.3, seed=5)
    net = _net(case)
    U, n0 = case.U, case.n0
    rng = np.random.default_rng(seed)
    l, u, mask = _random_bounds(rng, B, U)
    if B > 3:
        mask[3] = 1                                        # no unstable neuron: stuck
    w = rng.normal(size=(B, U)).astype(np.float32) if weighted else None
    lo = rng.uniform(0, 0.5, size=(B, n0)).astype(np.float32)
    hi = (lo + 0.3).astype(np.float32)
    from paper_2512_11087_gb300 import workloads as WL
    so, si = WL.draw_splits(case.cache["ids"], B, 0, 3, seed=seed)
    ver = (rng.uniform(size=B) < 0.2).astype(np.uint8)
    inf = (rng.uniform(size=B) < 0.1).astype(np.uint8)
    g = E.activation_split(net, _dev(so, torch.int32), _dev(si, torch.int32), _dev(lo), _dev(hi), _dev(l), _dev(u),
                           _dev(mask, torch.int8), _dev(ver, torch.uint8), _dev(inf, torch.uint8), weight=_dev(w))
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    o = O.activation_split(case.cache["ids"], so, si, lo, hi, l, u, mask, w, ver, inf)
    for k in ("split_off", "split_ids", "lo", "hi", "l", "u", "parent", "branched", "stuck"):
        assert g[k].shape == o[k].shape, k
        assert np.array_equal(np.ascontiguousarray(g[k]).view(np.uint8), np.ascontiguousarray(o[k]).view(np.uint8)), k
    net.close()


@pytest.mark.parametrize("k,weighted", [(1, True), (5, True), (5, False), (1000, True), (0, True)])
def test_select_targets_bit_exact(k, weighted):
    from oracle import oracle as O
    from paper_2512_11087_gb300 import engine as E
    case = Case([10, 40, 40, 40, 3], 2, 0, 0, 0.3, seed=6)
    net = _net(case)
    U, B = case.U, 50
    rng = np.random.default_rng(7 + k)
    l, u, mask = _random_bounds(rng, B, U)
    w = rng.normal(size=(B, U)).astype(np.float32) if weighted else None
    off, ids = E.select_targets(net, _dev(l), _dev(u), _dev(mask, torch.int8), k, weight=_dev(w))
    torch.cuda.synchronize()
    oo, oi = O.select_targets(O.layer_of_slots(case.net, case.cache["ids"]), l, u, mask, w, k)
    assert np.array_equal(off.cpu().numpy(), oo)
    assert np.array_equal(ids.cpu().numpy(), oi)
    net.close()


def test_one_activation_bab_iteration():
    from oracle import oracle as O
    from paper_2512_11087_gb300 import engine as E
    case = Case([16, 32, 32, 4], 24, 1, 3, 0.15, seed=8, sweeps=4)
    net = _net(case)
    g0 = gpu_round(case)
    d = E.to_dev
    sp = E.activation_split(net, d(case.split_off), d(case.split_ids), d(g0["lo_clip"]), d(g0["hi_clip"]),
                            d(g0["l"]), d(g0["u"]), d(g0["mask"]), d(g0["verified"]), d(g0["infeasible"]))
    torch.cuda.synchronize()
    sp = {k: v.cpu().numpy() for k, v in sp.items()}
    n = sp["lo"].shape[0]
    assert n > 0
    # children: the parent's clipped box and cached bounds, one more split each; top-2 targets a layer
    kid_mask = np.where(sp["l"] >= 0, 1, np.where(sp["u"] <= 0, -1, 0)).astype(np.int8)
    off, ids = E.select_targets(net, d(sp["l"]), d(sp["u"]), d(kid_mask), 2)
    torch.cuda.synchronize()
    kid = Case([16, 32, 32, 4], n, 0, 0, 0.15, seed=8, sweeps=4)
    kid.lo, kid.hi = sp["lo"], sp["hi"]
    kid.split_off, kid.split_ids = sp["split_off"], sp["split_ids"]
    kid.max_splits = int(np.max(np.diff(sp["split_off"])))
    kid.tgt_off, kid.tgt_ids = off.cpu().numpy(), ids.cpu().numpy()
    g1 = gpu_round(kid, l_in=d(sp["l"]), u_in=d(sp["u"]))
    o1 = kid.oracle(l_in=sp["l"].astype(np.float64), u_in=sp["u"].astype(np.float64))
    compare(kid, g1, o1)
    net.close()


def _weight_tol(case, o):
    # per subdomain and hidden layer: 2e-5 of the layer's largest weight (the FP32 products and the
    # rounding-level differences of the bounds that choose the relaxations)
    ids = case.cache["ids"]
    lay = np.searchsorted(np.cumsum(case.net.dims[1:-1]), ids, side="right")
    tol = np.zeros_like(o["babsr_weight"])
    for h in np.unique(lay):
        sel = lay == h
        tol[:, sel] = 2e-5 * np.max(np.abs(o["babsr_weight"][:, sel]), axis=1, keepdims=True) + 1e-30
    return tol


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dims,B,seed,sweeps", [([16, 32, 32, 4], 40, 11, 0), ([24, 48, 40, 40, 6], 77, 12, 3),
                                                ([784, 256, 256, 256, 10], 12, 13, 2)])
def test_babsr_weight_against_the_oracle(precision, dims, B, seed, sweeps):
    case = Case(dims, B, 0, 3, 0.05 if dims[0] > 100 else 0.15, seed=seed, sweeps=sweeps)
    g = gpu_round(case, precision=precision, want_weight=True)
    o = case.oracle(want_weight=True)
    compare(case, g, o)
    fe = ~o["infeasible"].astype(bool)
    gw, ow = g["babsr_weight"][:, :case.U], o["babsr_weight"]
    assert np.all(gw[~fe] == 0.0)
    err = np.abs(gw - ow)[fe]
    tol = _weight_tol(case, o)[fe]
    print("weight: max err / tol", float(np.max(err / tol)) if err.size else 0.0)
    assert np.all(err <= tol)
    # the sign decides the score factor max(0, -w): equal wherever the oracle's is clear of zero
    clear = np.abs(ow[fe]) > tol
    assert np.array_equal(np.sign(gw[fe])[clear], np.sign(ow[fe])[clear])
