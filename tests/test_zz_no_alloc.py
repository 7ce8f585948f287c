"""ws_estimate_batch_noalloc: estimation for callers that cannot allocate device memory.

Some applications embed the estimator where device memory belongs to someone else (a
fixed pool of a serving runtime, a captured steady state that must not allocate); they
call this entry point, which takes all device scratch from a fixed 32 MiB array inside
the library.  This file checks it through the C ABI against ws_estimate_batch, twice in
a row; that those calls create no CUDA resource at all (no device or page-locked host
allocation, stream or event: the library's own resource counters stay put, and so does
the device's free memory); that the caller's current device is left as it was; and that
an oversized batch is refused with WS_ENOMEM.  It is named to be collected last.
"""
import numpy as np
import pytest

from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import workloads as W
from test_oracle_pins import random_tiny

pytestmark = pytest.mark.gpu
RTOL = 1e-12


def workload():
    rng = W.SplitMix64(404)
    cfgs = [W.stencil_7pt_128()] + W.stencil_25pt_sweep(N=(160, 128, 96))[::25]
    cfgs += [random_tiny(rng) for _ in range(40)]
    return cfgs


def same(a, b):
    for k in B.RESULT_INT + ["limiter", "status"]:
        assert np.array_equal(a[k], b[k]), k
    for k in B.RESULT_DBL:
        assert np.allclose(a[k], b[k], rtol=RTOL, atol=0.0), k


def test_noalloc_matches_estimate_batch_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    hw = W.a100()
    cfgs = workload()
    arrays = B.marshal(cfgs)
    with B.Context(0, 2 << 30) as ctx:
        ref, ref_order = B.ws_estimate_batch(ctx, hw=hw, arrays=arrays)
    assert (ref["status"] == 0).all()
    torch.cuda.synchronize()
    counts_before = B.ws_resource_counts()
    res1, order1 = B.ws_estimate_batch_noalloc(0, hw=hw, arrays=arrays)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(0)
    res2, order2 = B.ws_estimate_batch_noalloc(0, hw=hw, arrays=arrays)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(0)
    counts_after = B.ws_resource_counts()
    for res, order in ((res1, order1), (res2, order2)):
        same(res, ref)
        assert list(order) == list(ref_order)
    assert free_after == free_before
    assert counts_after == counts_before, (counts_before, counts_after)
    assert torch.cuda.current_device() == 0


def test_noalloc_on_a_torch_stream_and_oversized_batch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    hw = W.a100()
    cfgs = [W.stencil_7pt_128()]
    s = torch.cuda.Stream()
    res, order = B.ws_estimate_batch_noalloc(0, cfgs, hw, stream=s)
    assert res[0]["wave_load_sectors"] == 832 and res[0]["ov_z"] == 480
    # a 25-point candidate on a 1024^3 domain with 4x1x64 blocks folded 4z: one field's
    # bitmaps alone (about 57 MiB) exceed the fixed scratch, refused before device work
    N = (1024, 1024, 1024)
    big = [W.Config(N=N, B=(4, 1, 64), fields=W.copy_fields(N, W.star_offsets(4)), fold_axis=2, fold=4)]
    with pytest.raises(B.WsError) as e:
        B.ws_estimate_batch_noalloc(0, big, hw)
    assert e.value.code == B.WS_ENOMEM
    assert "fixed" in str(e.value)
