"""Complete clipping of the final spec plane (Theorem 1, Algorithm 1 applied to a round's final
linear bound under the subdomain's split rows), on the oracle: the clipped value is a valid lower
bound of the spec over the feasible part of the subdomain (checked through the network on sampled
feasible points) and never below the plane's plain concretisation."""
import numpy as np

from oracle import oracle as O


def _forward(net, X):
    z = X.astype(np.float64)
    for i, (W, b) in enumerate(zip(net.Ws, net.bs)):
        z = z @ W.T + b
        if i < len(net.Ws) - 1:
            z = np.maximum(z, 0.0)
    return z


def split_rows(cache, codes):
    """Rows g.x + h <= 0 of split codes (Section 3.4): z >= 0 -> -Abar.x - cbar, z <= 0 -> Aund.x + cund."""
    G, h = [], []
    slot = {int(g): i for i, g in enumerate(cache["ids"])}
    for code in codes:
        s = slot[abs(int(code)) - 1]
        if code > 0:
            G.append(-cache["uA"][s]); h.append(-cache["uc"][s])
        else:
            G.append(cache["lA"][s]); h.append(cache["lc"][s])
    return np.array(G), np.array(h)


def test_clipped_spec_plane_is_sound_and_not_looser():
    from paper_2512_11087_gb300 import workloads as WL
    rng = np.random.default_rng(31)
    net = O.Net(WL.he_mlp([4, 16, 16, 3], seed=2))
    lo0, hi0 = np.full(4, -1.0), np.full(4, 1.0)
    cache = O.make_cache(O.root_crown(net, lo0, hi0))
    B = 12
    so, si = WL.draw_splits(cache["ids"], B, 2, 4, seed=8)
    lo, hi = np.tile(lo0, (B, 1)), np.tile(hi0, (B, 1))
    C, t = WL.margin_spec(3, y=0)
    out = O.bound_batch(net, cache, lo, hi, split_off=so, split_ids=si, C=C, t=t, relaxed=1, sweeps=0,
                        want_final=True)
    X = rng.uniform(-1, 1, size=(40000, 4))
    F = _forward(net, X) @ C.T.astype(np.float64) - t
    raised = 0
    for b in range(B):
        if out["infeasible"][b]:
            continue
        G, h = split_rows(cache, si[so[b]:so[b + 1]])
        feas = np.all(X @ G.T + h <= 1e-12, axis=1)
        lb, ub = out["lo_clip"][b], out["hi_clip"][b]
        for r in range(C.shape[0]):
            # the plane in FP32 (the form both sides clip), its intercept lowered by the rounding's
            # largest effect over the box so that it stays a lower bound of f_r
            a64 = out["final_A"][b, r]
            a32 = a64.astype(np.float32).astype(np.float64)
            c32 = out["final_c"][b, r] - np.abs(a64 - a32) @ np.maximum(np.abs(lb), np.abs(ub))
            v, beta, _ = O.complete_clip(a32, c32, G, h, lb, ub, 10)
            plain = O.dual_value(a32, c32, G, h, lb, ub, np.zeros(len(h)))
            assert v >= plain - 1e-9 * (1 + abs(plain))
            if feas.any():
                assert v <= F[feas, r].min() + 1e-9
            raised += v > plain + 1e-9
    assert raised > 0
