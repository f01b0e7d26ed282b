"""The allocation-free entry point (cv_relaxed_clip_static) against cv_bound_batch.

cv_relaxed_clip_static is for callers that cannot allocate device memory while they bound
subdomains (a framework whose allocator must own every device byte, or a loop where the device
synchronisation of cudaMalloc is not acceptable).  It runs the constraint rows, pre-check and
relaxed clipping with their scratch in the library's fixed device array.  Its clipped boxes and
infeasible flags must equal those of the workspace-based cv_bound_batch on the same inputs (run
without split clamping or complete clipping, so that it flags infeasibility in the same steps),
over two calls in a row with different batches (the shared array keeps the previous call's
contents).
This file is collected last so that a stop at the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402

pytestmark = pytest.mark.gpu


def _net_for(case):
    from paper_2512_11087_gb300 import engine as E
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    return net


def _reference_box(case, net):
    from paper_2512_11087_gb300 import engine as E
    # without split clamping or complete clipping, cv_bound_batch flags infeasibility only in the
    # pre-check and relaxed clipping, the steps the allocation-free entry runs
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, max_rows=case.max_rows, relaxed=1, sweeps=0,
                  enforce_splits=0)
    d = E.to_dev
    out = rnd.run(d(case.lo), d(case.hi), d(case.C), d(case.t), split_off=d(case.split_off),
                  split_ids=d(case.split_ids), row_off=d(case.row_off), G=d(case.G), h=d(case.h))
    torch.cuda.synchronize()
    return {k: out[k].cpu().numpy().copy() for k in ("lo_clip", "hi_clip", "infeasible")}


def _static_box(case, net):
    from paper_2512_11087_gb300 import capi, engine as E
    d = E.to_dev
    keep = [d(case.lo), d(case.hi), d(case.split_off), d(case.split_ids), d(case.row_off), d(case.G), d(case.h)]
    bi = capi.make_batch_in(case.B, keep[0], keep[1], case.m, None, None, split_off=keep[2], split_ids=keep[3],
                            max_splits=case.max_splits, row_off=keep[4], G=keep[5], h=keep[6],
                            max_rows=case.max_rows)
    lo = torch.full((case.B, case.n0), float("nan"), device="cuda")
    hi = torch.full((case.B, case.n0), float("nan"), device="cuda")
    inf = torch.full((case.B,), 7, dtype=torch.uint8, device="cuda")
    capi.cv_relaxed_clip_static(net.handle, net.cache, bi, lo, hi, inf, relaxed=1)
    torch.cuda.synchronize()
    assert capi.cv_device_status(net.handle) == 0
    return dict(lo_clip=lo.cpu().numpy(), hi_clip=hi.cpu().numpy(), infeasible=inf.cpu().numpy())


def _same(ref, got):
    # same kernels on the same inputs: the boxes agree to the bit, within the tests' box tolerance
    assert np.array_equal(ref["infeasible"], got["infeasible"])
    for k in ("lo_clip", "hi_clip"):
        assert np.array_equal(ref[k], got[k])


def test_static_scratch_matches_bound_batch_twice():
    a = Case([5] + [50] * 6 + [5], 256, 0, 8, 0.05, centre="pm1", clip01=False, out_rows=1, seed=0)
    b = Case([40, 64, 64, 6], 64, 1, 4, 0.1, seed=5)
    na, nb = _net_for(a), _net_for(b)
    ref_a, ref_b = _reference_box(a, na), _reference_box(b, nb)
    # two calls in a row on different batches: the second must not see the first one's scratch
    _same(ref_a, _static_box(a, na))
    _same(ref_b, _static_box(b, nb))
    _same(ref_a, _static_box(a, na))
    na.close(); nb.close()


def test_static_scratch_rejects_batches_above_the_limit():
    from paper_2512_11087_gb300 import capi, engine as E
    a = Case([6, 8, 3], 4, 0, 1, 0.1, seed=1)
    net = _net_for(a)
    d = E.to_dev
    lo, hi = d(a.lo), d(a.hi)
    # 2^20 subdomains x 2 rows x 9 bytes > 8 MiB: refused on the host, nothing launched
    bi = capi.make_batch_in(1 << 20, lo, hi, 1, None, None, split_off=d(a.split_off), split_ids=d(a.split_ids),
                            max_splits=2)
    with pytest.raises(capi.CVError) as ei:
        capi.cv_relaxed_clip_static(net.handle, net.cache, bi, lo, hi, torch.empty(1, dtype=torch.uint8,
                                                                                  device="cuda"))
    assert ei.value.status == 8
    net.close()


def test_static_calls_allocate_no_device_memory():
    # After a first call (which looks up the array's device address and loads the kernels), further
    # calls leave the device's free memory unchanged: the entry point itself allocates nothing.
    from paper_2512_11087_gb300 import capi, engine as E
    a = Case([40, 64, 64, 6], 64, 1, 4, 0.1, seed=5)
    net = _net_for(a)
    d = E.to_dev
    keep = [d(a.lo), d(a.hi), d(a.split_off), d(a.split_ids)]
    bi = capi.make_batch_in(a.B, keep[0], keep[1], a.m, None, None, split_off=keep[2], split_ids=keep[3],
                            max_splits=a.max_splits)
    lo = torch.empty((a.B, a.n0), device="cuda")
    hi = torch.empty((a.B, a.n0), device="cuda")
    inf = torch.empty((a.B,), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    capi.cv_relaxed_clip_static(net.handle, net.cache, bi, lo, hi, inf, relaxed=1, stream=stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        capi.cv_relaxed_clip_static(net.handle, net.cache, bi, lo, hi, inf, relaxed=1, stream=stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert capi.cv_device_status(net.handle) == 0
    net.close()
