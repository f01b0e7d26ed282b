"""The oracle against the paper's worked 2-D example (Appendix, '2D Toy Example')."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_2d.json")))


def F(s):
    return float(Fraction(s))


def toy():
    layers = [dict(kind=0, W=np.array(GOLD["W1"], np.float32), b=np.array(GOLD["b1"], np.float32),
                   in_shape=(2,), out_shape=(2,)),
              dict(kind=0, W=np.array([GOLD["w2"]], np.float32), b=np.array(GOLD["b2"], np.float32),
                   in_shape=(2,), out_shape=(1,))]
    net = O.Net(layers)
    lo = np.array(GOLD["box_lo"], np.float64)
    hi = np.array(GOLD["box_hi"], np.float64)
    return net, lo, hi


def test_pre_activation_bounds():
    net, lo, hi = toy()
    r = O.root_crown(net, lo, hi, alpha_mode=1)
    assert np.array_equal(r["l"], GOLD["pre_lower"])
    assert np.array_equal(r["u"], GOLD["pre_upper"])


def test_crown_lower_bound():
    net, lo, hi = toy()
    c = O.make_cache(O.root_crown(net, lo, hi, alpha_mode=1))
    out = O.bound_batch(net, c, lo[None], hi[None], C=np.array([[1.0]]), t=np.array([0.0]),
                        alpha_mode=1, relaxed=0, sweeps=0)
    assert out["lower"][0, 0] == pytest.approx(F(GOLD["crown_lower"]), abs=1e-14)


def _split_inactive_z1():
    return dict(split_off=np.array([0, 1]), split_ids=np.array([-1]))  # -(id 0 + 1): z1 <= 0


def test_relaxed_clipping_box_and_bounds():
    net, lo, hi = toy()
    c = O.make_cache(O.root_crown(net, lo, hi, alpha_mode=1))
    out = O.bound_batch(net, c, lo[None], hi[None], C=np.array([[1.0]]), t=np.array([0.0]),
                        alpha_mode=1, relaxed=1, sweeps=0, enforce_splits=0, **_split_inactive_z1())
    # the stored box is the exact box rounded outward to FP32
    for got, want, up in [(out["lo_clip"][0], GOLD["relaxed_box_lo"], False),
                          (out["hi_clip"][0], GOLD["relaxed_box_hi"], True)]:
        for g, w in zip(got, want):
            w = F(w)
            assert abs(g - w) <= 1.2e-7 * max(1.0, abs(w))
            assert (g >= w) if up else (g <= w)
    l, u = out["l"][0], out["u"][0]
    for k in range(2):
        assert l[k] == pytest.approx(F(GOLD["relaxed_pre_lower"][k]), rel=1e-6, abs=1e-6)
        assert u[k] == pytest.approx(F(GOLD["relaxed_pre_upper"][k]), rel=1e-6, abs=1e-6)
        assert u[k] >= F(GOLD["relaxed_pre_upper"][k])  # never tighter than the exact box's value
    assert out["lower"][0, 0] == pytest.approx(F(GOLD["relaxed_lower"]), rel=1e-6)


def test_complete_clipping_single_constraint():
    net, lo, hi = toy()
    W1, b1 = np.array(GOLD["W1"], np.float64), np.array(GOLD["b1"], np.float64)
    g, h = W1[0], b1[0]  # z1 <= 0
    # upper bound of z2 = max W1[1].x + b1[1]  ->  minimise -(W1[1].x + b1[1])
    v, beta, _ = O.complete_clip(-W1[1], -b1[1], [g], [h], lo, hi, sweeps=1)
    assert beta[0] == F(GOLD["complete_beta"])
    assert -v == F(GOLD["complete_upper"][1])
    v1, _, _ = O.complete_clip(-W1[0], -b1[0], [g], [h], lo, hi, sweeps=1)
    assert -v1 == F(GOLD["complete_upper"][0])
    # the dual is concave piecewise linear with these breakpoints: D(beta) at the kinks
    q = sorted(F(x) for x in GOLD["complete_breakpoints"])
    d = [O.dual_value(-W1[1], -b1[1], [g], [h], lo, hi, [b]) for b in [0.0] + q + [q[-1] + 1.0]]
    # slopes between consecutive points are the printed supergradients of the minimisation
    # form (sign flipped: the walk-through writes the upper-bound problem as a minimum)
    xs = [0.0] + q + [q[-1] + 1.0]
    slopes = [(d[i + 1] - d[i]) / (xs[i + 1] - xs[i]) for i in range(len(xs) - 1)]
    want = [-F(s) for s in GOLD["complete_subgradients"]]
    assert slopes == pytest.approx(want, abs=1e-12)


def test_complete_clipping_pipeline_verifies():
    net, lo, hi = toy()
    c = O.make_cache(O.root_crown(net, lo, hi, alpha_mode=1))
    out = O.bound_batch(net, c, lo[None], hi[None], C=np.array([[1.0]]), t=np.array([0.0]),
                        alpha_mode=1, relaxed=0, sweeps=1, enforce_splits=0, **_split_inactive_z1())
    assert np.array_equal(out["u"][0], [F(x) for x in GOLD["complete_upper"]])
    assert out["lower"][0, 0] == F(GOLD["complete_final_lower"])
    assert np.array_equal(out["mask"][0], [-1, -1])
