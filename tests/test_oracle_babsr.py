"""The oracle's activation-BaB steps with the BaBSR intercept score (Appendix, neuron selection
heuristic; Algorithm 5: Domain_Filter, Batch_Split, Top-K_Heuristic).

Pins: the score of an unstable neuron is the intercept of its upper ReLU line (fitted here through
the points (l, 0) and (u, u)) times the weight term; the split branches on the best-scoring unstable
neuron and gives the two children z <= 0 and z >= 0 after the parent's own splits, with the parent's
box and bounds; verified and infeasible parents get no children, all-stable ones are flagged; the
top-k targets are the k best per hidden layer by a brute-force sort, listed in slot order."""
import numpy as np
import pytest

from oracle import oracle as O


def _intercept(l, u):
    # the upper line of the triangle relaxation passes through (l, 0) and (u, u); its value at z = 0
    slope, icpt = np.polyfit([l, u], [0.0, u], 1)
    return icpt


def _parents(rng, B, U, n0, p_stable=0.3):
    l = rng.uniform(-2, 1, size=(B, U)).astype(np.float32)
    u = (l + rng.uniform(0.1, 3, size=(B, U))).astype(np.float32)
    mask = np.where(l >= 0, 1, np.where(u <= 0, -1, 0)).astype(np.int8)
    mask[rng.uniform(size=(B, U)) < p_stable] = 1
    lo = rng.uniform(-1, 0, size=(B, n0)).astype(np.float32)
    hi = (lo + 1).astype(np.float32)
    return l, u, mask, lo, hi


def test_split_branches_on_the_largest_intercept():
    rng = np.random.default_rng(41)
    B, U, n0 = 30, 17, 5
    l, u, mask, lo, hi = _parents(rng, B, U, n0)
    ids = np.arange(100, 100 + U)
    weight = rng.normal(size=(B, U)).astype(np.float32)
    for w in (None, weight):
        out = O.activation_split(ids, None, None, lo, hi, l, u, mask, w, np.zeros(B), np.zeros(B))
        for k in range(0, len(out["parent"]), 2):
            b = out["parent"][k]
            sc = np.full(U, -1.0)
            for c in range(U):
                if mask[b, c] == 0 and l[b, c] < 0 < u[b, c]:
                    sc[c] = _intercept(float(l[b, c]), float(u[b, c])) * (1.0 if w is None else max(0.0, -float(w[b, c])))
            best = out["branched"][k]
            assert sc[best] >= sc.max() * (1 - 1e-5) - 1e-12
            assert out["split_ids"][out["split_off"][k]:out["split_off"][k + 1]].tolist() == [-(ids[best] + 1)]
            assert out["split_ids"][out["split_off"][k + 1]:out["split_off"][k + 2]].tolist() == [ids[best] + 1]


def test_split_children_filter_and_stuck():
    rng = np.random.default_rng(42)
    B, U, n0 = 12, 9, 4
    l, u, mask, lo, hi = _parents(rng, B, U, n0)
    mask[3] = 1                                       # every cached neuron stable: no branch
    ver = np.zeros(B, np.uint8); ver[0] = 1
    inf = np.zeros(B, np.uint8); inf[1] = 1
    so = np.array([0, 1, 1, 3, 3, 4, 4, 4, 5, 5, 6, 6, 6], np.int32)
    si = np.array([7, -8, 9, 10, -11, 12], np.int32)
    out = O.activation_split(np.arange(U), so, si, lo, hi, l, u, mask, None, ver, inf)
    unstable = (mask == 0) & (l < 0) & (u > 0)
    stuck = [int(not ver[b] and not inf[b] and not unstable[b].any()) for b in range(B)]
    assert stuck[3] == 1
    kept = [b for b in range(B) if not ver[b] and not inf[b] and not stuck[b]]
    assert out["parent"].tolist() == [b for b in kept for _ in (0, 1)]
    assert out["stuck"].tolist() == stuck
    for k, b in enumerate(out["parent"]):
        codes = out["split_ids"][out["split_off"][k]:out["split_off"][k + 1]].tolist()
        assert codes[:-1] == si[so[b]:so[b + 1]].tolist()
        assert codes[-1] == (1 if k % 2 else -1) * (out["branched"][k] + 1)
        for key, src in (("lo", lo), ("hi", hi), ("l", l), ("u", u)):
            assert np.array_equal(out[key][k], src[b])


@pytest.mark.parametrize("k", [1, 3, 50])
def test_top_k_targets_per_layer(k):
    rng = np.random.default_rng(43)
    B, U = 10, 40
    l, u, mask, _, _ = _parents(rng, B, U, 2)
    layer_of = np.repeat([1, 2, 3, 4], 10).astype(np.int32)
    weight = rng.normal(size=(B, U)).astype(np.float32)
    off, ids = O.select_targets(layer_of, l, u, mask, weight, k)
    for b in range(B):
        want = []
        for layer in (1, 2, 3, 4):
            cand = [c for c in range(U) if layer_of[c] == layer and mask[b, c] == 0 and l[b, c] < 0 < u[b, c]]
            sc = {c: _intercept(float(l[b, c]), float(u[b, c])) * max(0.0, -float(weight[b, c])) for c in cand}
            want += sorted(sorted(cand, key=lambda c: (-sc[c], c))[:k])
        assert ids[off[b]:off[b + 1]].tolist() == sorted(want)


def test_top_k_ties_take_the_lowest_slots():
    l = np.full((1, 6), -1.0, np.float32)
    u = np.full((1, 6), 1.0, np.float32)
    mask = np.zeros((1, 6), np.int8)
    off, ids = O.select_targets(np.array([1, 1, 1, 2, 2, 2], np.int32), l, u, mask, np.zeros((1, 6)), 2)
    assert ids.tolist() == [0, 1, 3, 4]                # weight 0: every score 0, lowest slots first


# ---------------------------------------------------------------- the BaBSR weight
# The weight of hidden neuron q of layer h is the mean over the spec rows of the coefficient of its
# post-activation in the lower bound.  With the layers above h all affine on the box (stable
# neurons only, D = diag(0/1) whatever the coefficient's sign), that coefficient is the plain
# product C W^(L) D^(L-1) W^(L-1) ... D^(h+1) W^(h+1): closed forms by matrix products.

def _stable_above(seed, dims, on_off):
    from paper_2512_11087_gb300 import workloads as WL
    layers = WL.he_mlp(dims, seed=seed)
    # hidden layer 2 made stable: biases +-50 (active / inactive by on_off)
    layers[1]["b"] = np.where(on_off, 50.0, -50.0).astype(np.float32)
    return layers


def _weight_case(layers, m_rows, seed):
    from tests._cases import Case
    rng = np.random.default_rng(seed)
    nL = layers[-1]["W"].shape[0]
    C = rng.normal(size=(m_rows, nL))
    t = rng.normal(size=m_rows)
    case = Case(None, 3, 0, 0, 0.2, seed=seed, layers=layers, m_spec=(C, t))
    o = case.oracle(want_weight=True)
    return case, o, C


def test_weight_of_the_last_hidden_layer_is_the_mean_of_C_W():
    from paper_2512_11087_gb300 import workloads as WL
    layers = WL.he_mlp([6, 12, 10, 4], seed=31)
    case, o, C = _weight_case(layers, 5, 32)
    ids = case.cache["ids"]
    W3 = np.asarray(layers[2]["W"], np.float64)
    expect = (C @ W3).mean(axis=0)            # [n_2]
    sel = [c for c, g in enumerate(ids) if g >= 12]
    assert sel, "no cached neuron in hidden layer 2"
    for b in range(case.B):
        if o["infeasible"][b]:
            continue
        for c in sel:
            assert abs(o["babsr_weight"][b, c] - expect[ids[c] - 12]) <= 1e-12 * (1 + abs(expect[ids[c] - 12]))


def test_weight_through_a_stable_layer_is_the_mean_of_C_W_D_W():
    on_off = np.array([1, 0, 1, 1, 0, 1, 0, 1, 1, 0], bool)
    layers = _stable_above(33, [6, 12, 10, 4], on_off)
    case, o, C = _weight_case(layers, 4, 34)
    ids = case.cache["ids"]
    assert all(g < 12 for g in ids), "hidden layer 2 should be stable"
    W3 = np.asarray(layers[2]["W"], np.float64)
    W2 = np.asarray(layers[1]["W"], np.float64)
    expect = (C @ W3 @ np.diag(on_off.astype(float)) @ W2).mean(axis=0)   # [n_1]
    assert len(ids) > 3
    for b in range(case.B):
        for c, g in enumerate(ids):
            assert abs(o["babsr_weight"][b, c] - expect[g]) <= 1e-12 * (1 + np.abs(C @ W3).sum() * np.abs(W2).max())


def test_weight_is_zero_without_spec_rows_and_off_by_default():
    from paper_2512_11087_gb300 import workloads as WL
    layers = WL.he_mlp([5, 8, 8, 3], seed=35)
    case, o, _ = _weight_case(layers, 2, 36)
    assert "babsr_weight" not in case.oracle()
    o0 = case.oracle(C=np.zeros((0, 3)), t=np.zeros(0), want_weight=True)
    assert np.all(o0["babsr_weight"] == 0.0)
