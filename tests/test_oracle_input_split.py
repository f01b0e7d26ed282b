"""The oracle's input-BaB split step (Algorithm 4: Domain_Filter, Batch_Split with the parents'
hyperplanes shared by both children; Section 3.3) against what the mathematics fixes.

Pins: the children of a parent cover it exactly and differ from it only on the split axis;
dropped parents give no children; the split axis has the largest extent of the unproven planes
(measured by evaluating the planes along each axis); zero planes fall back to the widest axis;
a row is inherited only when exactly one spec row is unproven; and, through a real network
evaluated point by point, every sampled point not yet proven safe lies in a child whose
inherited row it satisfies."""
import numpy as np
import pytest

from oracle import oracle as O


def _random_parents(rng, B, n0, m, p_ver=0.2, p_inf=0.1):
    lo = rng.uniform(-1, 0.5, size=(B, n0)).astype(np.float32)
    hi = (lo + rng.uniform(0.05, 1.5, size=(B, n0))).astype(np.float32)
    A = rng.normal(size=(B, m, n0)).astype(np.float32)
    c = rng.normal(size=(B, m)).astype(np.float32)
    lower = rng.normal(size=(B, m)).astype(np.float32)
    ver = (rng.uniform(size=B) < p_ver).astype(np.uint8)
    inf = (rng.uniform(size=B) < p_inf).astype(np.uint8)
    return lo, hi, A, c, lower, ver, inf


def test_children_cover_parents_and_filter():
    rng = np.random.default_rng(21)
    lo, hi, A, c, lower, ver, inf = _random_parents(rng, 40, 7, 3)
    out = O.input_split(lo, hi, A, c, lower, ver, inf)
    kept = [b for b in range(40) if not ver[b] and not inf[b]]
    assert out["parent"].tolist() == [b for b in kept for _ in (0, 1)]
    for k, b in enumerate(kept):
        l0, h0, l1, h1 = out["lo"][2 * k], out["hi"][2 * k], out["lo"][2 * k + 1], out["hi"][2 * k + 1]
        diff = np.nonzero((l0 != lo[b]) | (h0 != hi[b]) | (l1 != lo[b]) | (h1 != hi[b]))[0]
        assert diff.size <= 1
        ax = int(diff[0]) if diff.size else 0
        # [lo, mid] and [mid, hi] on the axis: together exactly the parent's interval
        assert l0[ax] == lo[b, ax] and h1[ax] == hi[b, ax] and h0[ax] == l1[ax]
        assert lo[b, ax] <= h0[ax] <= hi[b, ax]
        assert abs(float(h0[ax]) - 0.5 * (float(lo[b, ax]) + float(hi[b, ax]))) <= 1e-6 * (1 + abs(float(h0[ax])))


def test_axis_has_the_largest_extent_of_the_unproven_planes():
    rng = np.random.default_rng(22)
    lo, hi, A, c, lower, ver, inf = _random_parents(rng, 60, 9, 4, p_ver=0.0, p_inf=0.0)
    out = O.input_split(lo, hi, A, c, lower, ver, inf)
    for b in range(60):
        unproven = [r for r in range(4) if not lower[b, r] > 0]
        xc = 0.5 * (lo[b].astype(np.float64) + hi[b].astype(np.float64))
        ext = []
        for i in range(9):
            x0, x1 = xc.copy(), xc.copy()
            x0[i], x1[i] = lo[b, i], hi[b, i]
            ext.append(sum(abs(A[b, r].astype(np.float64) @ x1 - A[b, r].astype(np.float64) @ x0) for r in unproven))
        ext = np.array(ext)
        ax = int(np.nonzero(out["lo"][2 * b + 1] != lo[b])[0][0])
        if ext.max() > 0:
            assert ext[ax] >= ext.max() * (1 - 1e-5)
        else:
            assert ax == int(np.argmax(hi[b] - lo[b]))


def test_zero_planes_split_the_widest_axis_lowest_index_first():
    lo = np.zeros((2, 4), np.float32)
    hi = np.array([[1, 3, 3, 2], [1, 1, 1, 1]], np.float32)
    A = np.zeros((2, 1, 4), np.float32)
    out = O.input_split(lo, hi, A, np.zeros((2, 1)), -np.ones((2, 1)), np.zeros(2), np.zeros(2))
    assert out["hi"][0].tolist() == [1, 1.5, 3, 2]   # axis 1: widest, before axis 2
    assert out["hi"][2].tolist() == [0.5, 1, 1, 1]   # all equal: axis 0


@pytest.mark.parametrize("lower_row,rows", [([1.0, 2.0, 3.0], None), ([1.0, -2.0, 3.0], 1), ([-1.0, -2.0, 3.0], None)])
def test_row_only_for_a_single_unproven_spec_row(lower_row, rows):
    rng = np.random.default_rng(23)
    lo, hi, A, c, _, _, _ = _random_parents(rng, 1, 5, 3)
    out = O.input_split(lo, hi, A, c, np.array([lower_row], np.float32), np.zeros(1), np.zeros(1))
    if all(v > 0 for v in lower_row):
        # every row proven but not flagged verified: split, no row
        assert out["row_off"].tolist() == [0, 0, 0]
    elif rows is None:
        assert out["row_off"].tolist() == [0, 0, 0]
    else:
        assert out["row_off"].tolist() == [0, 1, 2]
        assert np.array_equal(out["G"][0], A[0, rows]) and np.array_equal(out["G"][1], A[0, rows])
        assert out["h"].tolist() == [c[0, rows], c[0, rows]]


def _forward(net, X):
    z = X.astype(np.float64)
    for i, (W, b) in enumerate(zip(net.Ws, net.bs)):
        z = z @ W.T + b
        if i < len(net.Ws) - 1:
            z = np.maximum(z, 0.0)
    return z


def test_children_keep_every_point_not_yet_proven():
    # A 3-input, 3-class ReLU net; parents bounded by the oracle's round (final planes out),
    # split, and sampled: a point where some spec value f_r(x) <= 0 (not proven safe) must lie in
    # a child of its parent and satisfy that child's inherited row.
    from paper_2512_11087_gb300 import workloads as WL
    rng = np.random.default_rng(24)
    layers = WL.he_mlp([3, 12, 12, 3], seed=5)
    net = O.Net(layers)
    lo0, hi0 = np.full(3, -1.0), np.full(3, 1.0)
    cache = O.make_cache(O.root_crown(net, lo0, hi0))
    B = 16
    centres = rng.uniform(-0.8, 0.8, size=(B, 3))
    lo, hi = centres - 0.2, centres + 0.2
    C, t = WL.margin_spec(3, y=0)
    out = O.bound_batch(net, cache, lo, hi, C=C, t=t, relaxed=0, sweeps=0, want_final=True)
    sp = O.input_split(out["lo_clip"], out["hi_clip"], out["final_A"], out["final_c"], out["lower"],
                       out["verified"], out["infeasible"])
    checked = 0
    for b in range(B):
        X = rng.uniform(lo[b], hi[b], size=(4000, 3))
        f = _forward(net, X) @ C.T.astype(np.float64) - t
        unsafe = np.min(f, axis=1) <= 0
        kids = np.nonzero(sp["parent"] == b)[0]
        if out["verified"][b]:
            assert not unsafe.any() and kids.size == 0
            continue
        for x in X[unsafe]:
            ok = False
            for ch in kids:
                inside = np.all(x >= sp["lo"][ch] - 1e-7) and np.all(x <= sp["hi"][ch] + 1e-7)
                r0, r1 = sp["row_off"][ch], sp["row_off"][ch + 1]
                rows_ok = all(sp["G"][q].astype(np.float64) @ x + sp["h"][q] <= 1e-6 for q in range(r0, r1))
                ok = ok or (inside and rows_ok)
            assert ok
            checked += 1
    assert checked > 0


def test_two_unproven_rows_pass_no_row():
    # y = (0, x1 - 0.8, x2 - 0.8) through an always-active ReLU layer on [0,1]^2, spec f_k = y_0 - y_k:
    # f_1 = 0.8 - x1 and f_2 = 0.8 - x2 fail on different corners, so a row from either plane
    # alone would drop points where only the other one fails.  No row may be passed.
    layers = [dict(kind=0, W=np.eye(2, dtype=np.float32), b=np.zeros(2, np.float32), in_shape=(2,), out_shape=(2,)),
              dict(kind=0, W=np.array([[0, 0], [1, 0], [0, 1]], np.float32), b=np.array([0, -0.8, -0.8], np.float32),
                   in_shape=(2,), out_shape=(3,))]
    net = O.Net(layers)
    lo, hi = np.zeros((1, 2)), np.ones((1, 2))
    cache = O.make_cache(O.root_crown(net, lo[0], hi[0]))
    from paper_2512_11087_gb300 import workloads as WL
    C, t = WL.margin_spec(3, y=0)
    out = O.bound_batch(net, cache, lo, hi, C=C, t=t, relaxed=0, sweeps=0, want_final=True)
    assert np.all(out["lower"][0] < 0)
    sp = O.input_split(out["lo_clip"], out["hi_clip"], out["final_A"], out["final_c"], out["lower"],
                       out["verified"], out["infeasible"])
    assert sp["row_off"].tolist() == [0, 0, 0]
    # the points x1 >= 0.8 > x2 (only f_1 fails) stay in the children
    x = np.array([0.9, 0.1])
    assert any(np.all(x >= sp["lo"][k]) and np.all(x <= sp["hi"][k]) for k in range(2))
    # with a single unproven row (f_2 dropped from the spec) the row is f_1's exact plane:
    # 0.8 - x1 <= 0, which keeps x1 >= 0.8 and drops only proven points
    out1 = O.bound_batch(net, cache, lo, hi, C=C[:1], t=t[:1], relaxed=0, sweeps=0, want_final=True)
    sp1 = O.input_split(out1["lo_clip"], out1["hi_clip"], out1["final_A"], out1["final_c"], out1["lower"],
                        out1["verified"], out1["infeasible"])
    assert sp1["row_off"].tolist() == [0, 1, 2]
    g, hh = sp1["G"][0].astype(np.float64), float(sp1["h"][0])
    assert g @ np.array([0.9, 0.5]) + hh <= 1e-6 and g @ np.array([0.5, 0.5]) + hh > 0
