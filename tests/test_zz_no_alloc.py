"""acom_bounds_static: the spectral bounds computed with the scratch in the
library's fixed device array, for callers that cannot allocate device memory
while they run (an acquisition loop that reserved its whole device budget up
front, or a process whose device memory belongs to another allocator).
Checked against acom_bounds on two calls in a row, through the C ABI.
Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before these."""

import numpy as np
import pytest

import synth

from gpu_common import gpu_plan, to_dev

pytestmark = pytest.mark.gpu

STATIC_BYTES = 32 << 20        # the library's fixed scratch array


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _allocs():
    from paper_2111_00171_gb300 import acom
    return acom.load_library().acom_device_allocations()


def test_bounds_static_first_call_takes_at_most_its_array():
    """The first call on a device may commit the 32 MiB array (lazy module
    loading); nothing else.  Measured after acom_bounds has loaded the raster
    and contraction kernels.  Later calls request no allocation at all."""
    import torch
    plan = gpu_plan("au_2deg_75x180", precision=0)
    inputs = to_dev(synth.random_patterns(4241, n_patterns=300))
    ref = plan.bounds(*inputs)
    out = torch.empty_like(ref)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    a0 = _allocs()
    plan.bounds_static(*inputs, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert _allocs() == a0
    assert free0 - free1 <= STATIC_BYTES + (16 << 20), (free0, free1)
    b = ref.cpu().numpy()
    np.testing.assert_allclose(out.cpu().numpy(), b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    plan.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "bf16"])
def test_bounds_static_matches_bounds_twice(precision):
    import torch
    plan = gpu_plan("au_2deg_75x180", precision=precision)
    # more patterns than one chunk of the static array holds for this plan
    scan = synth.random_patterns(4242, n_patterns=1000)
    inputs = to_dev(scan)
    ref = plan.bounds(*inputs)
    out = torch.full_like(ref, float("nan"))
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        a0 = _allocs()
        plan.bounds_static(*inputs, out=out)
        torch.cuda.synchronize()
        assert _allocs() == a0            # the call requested no device memory
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    # nor does device memory shrink over a further call
    free0, _ = torch.cuda.mem_get_info()
    plan.bounds_static(*inputs, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    plan.close()


@pytest.mark.parametrize("precision", [2, 3], ids=["fp16", "fp8"])
def test_bounds_static_reduced_plans_take_fp32_path(precision):
    """FP16 and E4M3 plans' static bounds are computed on the FP32 path: they
    equal an FP32 plan's bounds."""
    import torch
    pq = gpu_plan("au_2deg_75x180", precision=precision)
    p32 = gpu_plan("au_2deg_75x180", precision=0)
    inputs = to_dev(synth.random_patterns(4243, n_patterns=200))
    ref = p32.bounds(*inputs)
    out = torch.full_like(ref, float("nan"))
    pq.bounds_static(*inputs, out=out)
    torch.cuda.synchronize()
    b = ref.cpu().numpy()
    np.testing.assert_allclose(out.cpu().numpy(), b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    pq.close()
    p32.close()


def test_bounds_static_rejects_what_bounds_rejects():
    """A row pointer not starting at 0 is bad input for both entry points (the
    arrays hold one unused leading peak, so every read stays in bounds); a
    wrong output tensor is refused by the binding before the call; after a
    good call the thread's error message is empty again."""
    import torch
    from paper_2111_00171_gb300 import acom
    plan = gpu_plan("au_2deg_75x180", precision=0)
    scan = synth.random_patterns(4244, n_patterns=50)
    rp = np.asarray(scan.row_ptr, np.int64) + 1
    pad = lambda a: np.concatenate([np.zeros(1, np.float32), np.asarray(a, np.float32)])
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bad = (d(rp), d(pad(scan.qx)), d(pad(scan.qy)), d(pad(scan.I)))
    out = torch.empty((scan.n_patterns, plan.info["n_za"]), dtype=torch.float32, device="cuda")
    with pytest.raises(acom.AcomError) as e1:
        plan.bounds(*bad)
    assert e1.value.status == 6
    with pytest.raises(acom.AcomError) as e2:
        plan.bounds_static(*bad, out=out)
    assert e2.value.status == 6
    good = to_dev(scan)
    for wrong in (out[:, :-1], out.double(), out.t().contiguous().t(), out.cpu()):
        with pytest.raises(ValueError):
            plan.bounds_static(*good, out=wrong)
    plan.bounds_static(*good, out=out)
    lib = acom.load_library()
    assert lib.acom_last_error() == b""
    ref = plan.bounds(*good)
    b = ref.cpu().numpy()
    np.testing.assert_allclose(out.cpu().numpy(), b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    plan.close()
