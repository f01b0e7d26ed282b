"""The activation-BaB loop of Algorithm 5 on the GPU (cv_bab_*) against the oracle's loop, iteration by
iteration: the same counts (picked, stuck, children, verified, infeasible, depth-limited, pushed,
remaining) and the same domain list (every domain's split codes, in stack order) after Init and after
every iteration, and the same final answer.  Both sides take their integer decisions (branching,
top-k, verified) from their own bounds, so the cases are checked for near-ties first: every
branching and top-k decision of the oracle's run is clear by a relative gap of 1e-4 (exact ties at a
zero weight factor excepted) and every filtered lower bound by 1e-4 of its scale."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402

pytestmark = pytest.mark.gpu

KEYS = ("picked", "stuck", "children", "verified", "infeasible", "depth_limited", "pushed", "remaining")


def _net(case):
    from paper_2512_11087_gb300 import engine as E
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    return net


def _lists(off, ids):
    return [list(map(int, ids[off[k]:off[k + 1]])) for k in range(len(off) - 1)]


def _case(dims, eps, seed, m_rows, shift):
    from oracle import oracle as O
    from paper_2512_11087_gb300 import workloads as WL
    layers = WL.he_mlp(dims, seed=seed)
    rng = np.random.default_rng(seed + 100)
    C = rng.normal(size=(m_rows, dims[-1]))
    case = Case(None, 1, 0, 0, eps, seed=seed, layers=layers, m_spec=(C, np.zeros(m_rows)), clip01=False)
    # thresholds: the spec at the box centre plus a shift, so that the root is not verified at once
    y = np.asarray(case.lo0 + case.hi0, np.float64) / 2
    for W, b in zip(case.net.Ws[:-1], case.net.bs[:-1]):
        y = np.maximum(W @ y + b, 0)
    y = case.net.Ws[-1] @ y + case.net.bs[-1]
    t = -(C @ y) + shift
    case.C, case.t = C, t
    return case


@pytest.mark.parametrize("dims,eps,seed,m_rows,shift,batch,top_k,iters", [
    ([4, 12, 12, 3], 0.4, 1, 2, 0.25, 4, -1, 12),
    ([4, 12, 12, 3], 0.4, 2, 2, 0.3, 8, 2, 12),
    ([6, 16, 16, 16, 4], 0.3, 3, 3, 0.5, 16, 3, 8),
    ([6, 16, 16, 16, 4], 0.3, 4, 1, 0.2, 5, -1, 8),
    ([5, 20, 20, 3], 0.3, 6, 2, 2.0, 8, 2, 12),          # ends verified after 4 iterations
])
@pytest.mark.parametrize("precision", [0, 1])
def test_loop_matches_the_oracle_iteration_by_iteration(dims, eps, seed, m_rows, shift, batch, top_k, iters,
                                                        precision):
    from oracle import oracle as O
    from paper_2512_11087_gb300 import capi, engine as E
    case = _case(dims, eps, seed, m_rows, shift)
    max_depth, capacity, sweeps = 10, 2048, 4
    rec = O.activation_bab(case.net, case.cache, case.lo0[None], case.hi0[None], case.C, case.t, batch=batch,
                           top_k=top_k, capacity=capacity, max_depth=max_depth, max_iters=iters, sweeps=sweeps)
    near = [g for g in rec["branch_gap"] + rec["topk_gap"] if g < 1e-4] + [g for g in rec["lower_gap"] if g < 1e-4]
    assert not near, f"near-ties in the oracle's run: {near}"
    assert len(rec["iters"]) > 2, "the case ends too soon to test the loop"
    net = _net(case)
    bab = E.ActivationBaB(net, case.C, case.t, batch=batch, top_k=top_k, capacity=capacity, max_depth=max_depth,
                          sweeps=sweeps, precision=precision)
    got = [bab.init(f32(case.lo0[None]), f32(case.hi0[None]))]
    lists = [_lists(*bab.domains()[:2])]
    while len(got) < len(rec["iters"]):
        got.append(bab.step())
        lists.append(_lists(*bab.domains()[:2]))
    torch.cuda.synchronize()
    for k, (g, o) in enumerate(zip(got, rec["iters"])):
        for key in KEYS:
            assert g[key] == o[key], (k, key, g, o)
        assert lists[k] == rec["lists"][k], k
    # one more step on the GPU when the oracle stopped at an empty list: nothing to do
    if rec["remaining"] == 0:
        assert bab.step()["picked"] == 0
    assert capi.cv_device_status(net.handle) == 0
    bab.close()
    net.close()


def test_run_sums_the_iterations_and_respects_the_capacity():
    from paper_2512_11087_gb300 import capi, engine as E
    case = _case([4, 12, 12, 3], 0.4, 1, 2, 0.3)
    net = _net(case)
    kw = dict(batch=4, top_k=-1, capacity=64, max_depth=10, sweeps=4)
    a = E.ActivationBaB(net, case.C, case.t, **kw)
    a.init(f32(case.lo0[None]), f32(case.hi0[None]))
    steps = [a.step() for _ in range(5)]
    b = E.ActivationBaB(net, case.C, case.t, **kw)
    b.init(f32(case.lo0[None]), f32(case.hi0[None]))
    tot, it = b.run(5)
    assert it == sum(1 for s in steps if s["picked"] > 0) or it == 5
    for key in ("picked", "stuck", "children", "verified", "infeasible", "depth_limited", "pushed"):
        assert tot[key] == sum(s[key] for s in steps), key
    assert tot["remaining"] == steps[-1]["remaining"] <= 64
    assert np.array_equal(a.domains()[0], b.domains()[0])
    a.close(); b.close()
    # bad parameters are refused before anything is allocated
    bad = capi.cv_bab_params_default()
    bad.capacity = bad.batch
    with pytest.raises(capi.CVError):
        capi.cv_bab_create(net.handle, net.cache, 2, E.to_dev(case.C, torch.float32), E.to_dev(case.t, torch.float32),
                           bad)
    net.close()
