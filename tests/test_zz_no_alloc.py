"""acom_bounds_static: the spectral bounds computed with the scratch in the
library's fixed device array, for callers that must not allocate device
memory during the call.  Checked against acom_bounds on two calls in a row,
through the C ABI.  Collected last on purpose (file name)."""

import numpy as np
import pytest

import synth

from gpu_common import gpu_plan, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


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
        plan.bounds_static(*inputs, out=out)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    # no device memory is taken by further calls
    free0, _ = torch.cuda.mem_get_info()
    plan.bounds_static(*inputs, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    plan.close()


def test_bounds_static_fp16_plan_takes_fp32_path():
    """An FP16 plan's static bounds are computed on the FP32 path: they equal
    an FP32 plan's bounds."""
    import torch
    p16 = gpu_plan("au_2deg_75x180", precision=2)
    p32 = gpu_plan("au_2deg_75x180", precision=0)
    inputs = to_dev(synth.random_patterns(4243, n_patterns=200))
    ref = p32.bounds(*inputs)
    out = torch.full_like(ref, float("nan"))
    p16.bounds_static(*inputs, out=out)
    torch.cuda.synchronize()
    b = ref.cpu().numpy()
    np.testing.assert_allclose(out.cpu().numpy(), b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    p16.close()
    p32.close()
