"""Complete clipping's work-item sizes (cv_cc_items_set / cv_cc_items_get) and their autotuner
(cv_autotune_cc), through the C-ABI: the item size changes no output bit, the tuner keeps sizes
from its grid in the cache, and bad arguments are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import Case, f32  # noqa: E402

pytestmark = pytest.mark.gpu

GRID = ({128, 256, 512, 1024}, {32, 64, 128, 256}, {8, 16, 32, 64, 128})


def _setup(case):
    from paper_2512_11087_gb300 import engine as E
    net = E.Net(case.layers)
    c = case.cache
    net.set_cache(f32(case.lo0), f32(case.hi0), f32(c["root_l"]), f32(c["root_u"]), c["ids"], f32(c["lA"]),
                  f32(c["lc"]), f32(c["uA"]), f32(c["uc"]))
    rnd = E.Round(net, case.B, case.m, max_splits=case.max_splits, max_rows=case.max_rows, relaxed=case.relaxed,
                  sweeps=case.sweeps)
    d = E.to_dev
    args = (d(case.lo), d(case.hi), d(case.C), d(case.t))
    kw = dict(split_off=d(case.split_off), split_ids=d(case.split_ids), row_off=d(case.row_off), G=d(case.G),
              h=d(case.h))
    return net, rnd, args, kw


def _outputs(rnd, args, kw):
    out = rnd.run(*args, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().copy() for k, v in out.items()}


@pytest.fixture(scope="module")
def tuned():
    # 1-8 active rows per subdomain: items of all three classes, and the launch for more than four rows
    case = Case([32, 40, 40, 6], 48, 0, 2, 0.1, sweeps=6, cut_rows=(0, 6), seed=2)
    net, rnd, args, kw = _setup(case)
    yield case, net, rnd, args, kw
    net.close()


def test_item_sizes_change_no_output(tuned):
    from paper_2512_11087_gb300 import capi
    case, net, rnd, args, kw = tuned
    assert capi.cv_cc_items_get(net.cache) == list(capi.CC_ITEMS_DEFAULT)
    ref = _outputs(rnd, args, kw)
    for items in ([1, 1, 1], [512, 128, 64], [7, 3, 2]):
        capi.cv_cc_items_set(net.cache, items)
        assert capi.cv_cc_items_get(net.cache) == items
        got = _outputs(rnd, args, kw)
        for k in ref:
            assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), (items, k)
    capi.cv_cc_items_set(net.cache, capi.CC_ITEMS_DEFAULT)
    # the oracle agrees with these outputs at the parity bar
    from tests.test_gpu_parity import compare
    compare(case, ref, case.oracle())


def test_item_sizes_out_of_range_are_refused(tuned):
    from paper_2512_11087_gb300 import capi
    _, net, _, _, _ = tuned
    for bad in ([0, 64, 16], [256, 5000, 16], [256, 64, -1]):
        with pytest.raises(RuntimeError, match=r"\[1, 4096\]"):
            capi.cv_cc_items_set(net.cache, bad)
    assert capi.cv_cc_items_get(net.cache) == list(capi.CC_ITEMS_DEFAULT)


def test_autotune_keeps_sizes_from_its_grid(tuned):
    from paper_2512_11087_gb300 import capi
    case, net, rnd, args, kw = tuned
    ref = _outputs(rnd, args, kw)
    best, ms = rnd.autotune(*args, **kw)
    assert ms > 0.0
    for c in range(3):
        assert best[c] in GRID[c] | {capi.CC_ITEMS_DEFAULT[c]}
    assert capi.cv_cc_items_get(net.cache) == best
    got = _outputs(rnd, args, kw)
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint8), got[k].view(np.uint8)), k
    capi.cv_cc_items_set(net.cache, capi.CC_ITEMS_DEFAULT)


def test_autotune_needs_complete_clipping():
    case = Case([8, 10, 3], 4, 1, 2, 0.1, sweeps=0)
    net, rnd, args, kw = _setup(case)
    with pytest.raises(RuntimeError, match="sweeps = 0"):
        rnd.autotune(*args, **kw)
    net.close()
