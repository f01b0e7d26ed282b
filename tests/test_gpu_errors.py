"""Error paths of the C-ABI, driven from the host with bad inputs (no kernel is made to fault).

Every device-side check reports a bit of the network's status word and skips the access it guards
(split CSR counts above max_splits leave the subdomain without rows; out-of-range split codes give
no row; a non-finite box only propagates NaN through bounded loops; out-of-range target slots are
skipped).  cv_batch_check finds the same problems before a round, with CV_EINVAL / CV_ENAN.  After
each bad round the status word is read and cleared, and a clean round on the same network gives the
same outputs as before: the context stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2512_11087_gb300 import engine as E
    case = Case([24, 32, 32, 6], 8, 1, 3, 0.1, sweeps=3, seed=21)
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    yield case, net
    net.close()


def _round(case, net, sweeps=None, **over):
    from paper_2512_11087_gb300 import engine as E
    args = dict(lo=case.lo, hi=case.hi, split_off=case.split_off, split_ids=case.split_ids, tgt_off=None,
                tgt_ids=None)
    args.update(over)
    max_splits = over.get("max_splits", case.max_splits)
    rnd = E.Round(net, case.B, case.m, max_splits=max_splits, sweeps=case.sweeps if sweeps is None else sweeps)
    d = E.to_dev
    out = rnd.run(d(args["lo"]), d(args["hi"]), d(case.C), d(case.t), split_off=d(args["split_off"]),
                  split_ids=d(args["split_ids"]), tgt_off=d(args["tgt_off"]), tgt_ids=d(args["tgt_ids"]))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().copy() for k, v in out.items()}


def _check(case, net, **over):
    from paper_2512_11087_gb300 import capi, engine as E
    d = E.to_dev
    a = dict(lo=case.lo, hi=case.hi, split_off=case.split_off, split_ids=case.split_ids, tgt_off=None, tgt_ids=None)
    a.update(over)
    keep = [d(a["lo"]), d(a["hi"]), d(case.C), d(case.t), d(a["split_off"]), d(a["split_ids"]), d(a["tgt_off"]),
            d(a["tgt_ids"])]
    bi = capi.make_batch_in(case.B, keep[0], keep[1], case.m, keep[2], keep[3], split_off=keep[4],
                            split_ids=keep[5], max_splits=over.get("max_splits", case.max_splits), tgt_off=keep[6],
                            tgt_ids=keep[7])
    return capi.cv_batch_check(net.handle, net.cache, bi)


def _status(net):
    from paper_2512_11087_gb300 import capi
    return capi.cv_device_status_raw(net.handle)


def _clean_round_unchanged(case, net, ref):
    from paper_2512_11087_gb300 import capi
    g = _round(case, net)
    assert _status(net) == (capi.CV_OK, 0)
    for k in ref:
        assert np.array_equal(ref[k], g[k]), k


def test_clean_batch_passes_the_check(setup):
    from paper_2512_11087_gb300 import capi
    case, net = setup
    assert _check(case, net) == (capi.CV_OK, 0)
    _round(case, net)
    assert _status(net) == (capi.CV_OK, 0)


def test_csr_count_above_max_splits(setup):
    from paper_2512_11087_gb300 import capi
    case, net = setup
    ref = _round(case, net)
    # subdomain 0 gets one split more than max_splits allows (valid codes)
    lists = [list(case.split_ids[case.split_off[b]:case.split_off[b + 1]]) for b in range(case.B)]
    used = {abs(int(x)) for x in lists[0]}
    extra = [int(g) + 1 for g in case.cache["ids"] if int(g) + 1 not in used][:case.max_splits + 1 - len(lists[0])]
    lists[0] = lists[0] + [-e for e in extra]
    so = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int32)
    si = np.array([x for l in lists for x in l], np.int32)
    assert so[1] - so[0] == case.max_splits + 1
    st, bits = _check(case, net, split_off=so, split_ids=si, max_splits=case.max_splits)
    assert st == capi.CV_EINVAL and bits & 1
    _round(case, net, split_off=so, split_ids=si, max_splits=case.max_splits)
    st, word = _status(net)
    assert st == capi.CV_EDEVICE and word & 1
    assert _status(net) == (capi.CV_OK, 0)  # read and cleared
    _clean_round_unchanged(case, net, ref)


def test_split_code_out_of_range(setup):
    from paper_2512_11087_gb300 import capi
    case, net = setup
    ref = _round(case, net)
    si = case.split_ids.copy()
    si[0] = net.H + 5
    st, bits = _check(case, net, split_ids=si)
    assert st == capi.CV_EINVAL and bits & 2
    _round(case, net, split_ids=si)
    st, word = _status(net)
    assert st == capi.CV_EDEVICE and word & 2
    _clean_round_unchanged(case, net, ref)


def test_non_finite_box(setup):
    from paper_2512_11087_gb300 import capi
    case, net = setup
    ref = _round(case, net)
    lo = case.lo.copy()
    lo[3, 5] = np.nan
    st, bits = _check(case, net, lo=lo)
    assert st == capi.CV_ENAN and bits & 4
    _round(case, net, sweeps=0, lo=lo)
    st, word = _status(net)
    assert st == capi.CV_EDEVICE and word & 4
    _clean_round_unchanged(case, net, ref)


def test_target_slot_out_of_range(setup):
    from paper_2512_11087_gb300 import capi
    case, net = setup
    ref = _round(case, net)
    U = net.U
    off = np.arange(0, 3 * case.B + 1, 3, dtype=np.int32)
    ids = np.tile(np.array([0, 1, U + 3], np.int32), case.B)
    st, bits = _check(case, net, tgt_off=off, tgt_ids=ids)
    assert st == capi.CV_EINVAL and bits & 8
    _round(case, net, tgt_off=off, tgt_ids=ids)
    st, word = _status(net)
    assert st == capi.CV_EDEVICE and word & 8
    _clean_round_unchanged(case, net, ref)


def test_empty_box_is_refused_by_the_check(setup):
    from paper_2512_11087_gb300 import capi
    case, net = setup
    lo, hi = case.lo.copy(), case.hi.copy()
    lo[1, 2], hi[1, 2] = hi[1, 2] + 1.0, lo[1, 2]
    st, bits = _check(case, net, lo=lo, hi=hi)
    assert st == capi.CV_EINVAL and bits & 32


def test_host_checks_before_any_launch(setup):
    from paper_2512_11087_gb300 import capi, engine as E
    case, net = setup
    opt = capi.cv_options_default()
    for B, msp, mrw in ((-1, 0, 0), (2, 2 ** 30, 2 ** 30), (1 << 20, 4096, 0)):
        bi = capi.make_batch_in(B, None, None, case.m, None, None, max_splits=msp, max_rows=mrw)
        with pytest.raises(capi.CVError) as e:
            capi.cv_bound_batch_workspace(net.handle, net.cache, bi, opt)
        assert e.value.status == capi.CV_EINVAL
    # a workspace smaller than the plan is refused, and nothing ran
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, sweeps=case.sweeps)
    d = E.to_dev
    keep = [d(case.lo), d(case.hi), d(case.C), d(case.t), d(case.split_off), d(case.split_ids)]
    bi = capi.make_batch_in(case.B, keep[0], keep[1], case.m, keep[2], keep[3], split_off=keep[4],
                            split_ids=keep[5], max_splits=case.max_splits)
    with pytest.raises(capi.CVError) as e:
        capi.cv_bound_batch(net.handle, net.cache, bi, rnd.bo, rnd.opt, rnd.ws, rnd.ws_bytes - 256)
    assert e.value.status == capi.CV_EWORKSPACE
    assert _status(net) == (capi.CV_OK, 0)


def test_misaligned_workspace_is_refused_before_any_launch(setup):
    """cv_bound_batch and cv_alpha_grad take a 256-byte aligned workspace (their kernels use 16-byte
    vector accesses and TMA into it); a misaligned one is refused with CV_EINVAL and nothing runs."""
    from paper_2512_11087_gb300 import capi, engine as E
    case, net = setup
    ref = _round(case, net)
    d = E.to_dev
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, sweeps=case.sweeps)
    keep = [d(case.lo), d(case.hi), d(case.C), d(case.t), d(case.split_off), d(case.split_ids)]
    bi = capi.make_batch_in(case.B, keep[0], keep[1], case.m, keep[2], keep[3], split_off=keep[4],
                            split_ids=keep[5], max_splits=case.max_splits)
    bad = torch.empty(rnd.ws_bytes + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.CVError) as e:
        capi.cv_bound_batch(net.handle, net.cache, bi, rnd.bo, rnd.opt, bad[4:], rnd.ws_bytes)
    assert e.value.status == capi.CV_EINVAL
    # the slope gradient, on this round's bounds and masks
    st = E.AlphaState(net, d(case.lo), d(case.hi), d(ref["l"]), d(ref["u"]), d(ref["mask"]), d(case.C), d(case.t))
    alpha = torch.full((case.B, case.m, net.H), 0.5, dtype=torch.float32, device="cuda")
    lower = torch.empty(case.B, case.m, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(alpha)
    ai = capi.make_alpha_in(st.B, st.m, st.lo, st.hi, st.l, st.u, st.mask, st.C, st.t, alpha, None)
    bad = torch.empty(st.ws_bytes + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.CVError) as e:
        capi.cv_alpha_grad(net.handle, net.cache, ai, lower, grad, bad[4:], st.ws_bytes)
    assert e.value.status == capi.CV_EINVAL
    torch.cuda.synchronize()
    assert _status(net) == (capi.CV_OK, 0)
    _clean_round_unchanged(case, net, ref)
