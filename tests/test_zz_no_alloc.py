"""sop_norm_noalloc against sop_norm through the C ABI (GPU).

sop_norm_noalloc is for callers that may not allocate device memory (a pool
allocator that owns all of HBM, or a loop that cannot afford cudaMalloc's
device-wide synchronisation); its scratch is a fixed array inside the library
shared by all calls.  The checks: two calls in a row, with different inputs
and sizes, each agree with the plan-based sop_norm within the tolerance of the
norm tests, so nothing left in the shared array by one call leaks into the
next; oversize and invalid inputs are rejected.  This file is collected last.
"""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import sop

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    gc.require_gpu()


def _plan_norm(dims, comps, seed, dtype):
    w = gc.random_workload(dims, comps, seed=seed, n_steps=1, dt=0.01, field_scale=0.0, v_scale=0.0,
                           spacing=tuple(0.05 + 0.01 * a for a in range(len(dims))))
    _, prop = gc.run_gpu(w, dtype, n_steps=0)
    return prop, prop.norm(), float(np.prod(w.spacing))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_no_alloc_norm_matches_sop_norm_on_two_calls(dtype):
    import torch
    code = sop.SOP_C64 if dtype == "c64" else sop.SOP_C128
    # first a larger spinor, then a smaller scalar field: the second call reads
    # fewer partial sums than the first one left in the shared array
    cases = [((384, 256), 4, 11), ((96, 24), 1, 12)]
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for k, (dims, comps, seed) in enumerate(cases):
        prop, ref, dV = _plan_norm(dims, comps, seed, dtype)
        n_values = prop.state.numel()
        sop.sop_norm_noalloc(prop.state, n_values, code, dV, out[k:k + 1])
        torch.cuda.synchronize()
        got = float(out[k].item())
        assert abs(got - ref) <= TOL[dtype] * abs(ref), (dims, got, ref)
        prop.close()


def test_no_alloc_rejects_bad_sizes_and_pointers():
    """The C entry point's own checks (raw pointers, so the Python wrapper's
    tensor checks do not intercept them), then the wrapper's tensor checks."""
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    psi = torch.zeros(16, dtype=torch.complex64, device="cuda")
    p, o = psi.data_ptr(), out.data_ptr()
    with pytest.raises(sop.SopError) as ei:
        sop.sop_norm_noalloc(p, (1 << 29) + 1, sop.SOP_C64, 1.0, o)
    assert ei.value.status == sop.SOP_EUNSUPPORTED
    assert "2^29" in str(ei.value)
    with pytest.raises(sop.SopError) as ei:
        sop.sop_norm_noalloc(p, -1, sop.SOP_C64, 1.0, o)
    assert ei.value.status == sop.SOP_EINVAL
    with pytest.raises(sop.SopError) as ei:
        sop.sop_norm_noalloc(p, 16, 9, 1.0, o)
    assert ei.value.status == sop.SOP_EINVAL
    sop.sop_norm_noalloc(psi, 0, sop.SOP_C64, 1.0, out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # tensors the kernel would overrun, or of the wrong kind, never reach it
    with pytest.raises(ValueError):
        sop.sop_norm_noalloc(psi, 17, sop.SOP_C64, 1.0, out)            # more values than psi holds
    with pytest.raises(ValueError):
        sop.sop_norm_noalloc(psi, 16, sop.SOP_C128, 1.0, out)           # dtype mismatch
    with pytest.raises(ValueError):
        sop.sop_norm_noalloc(psi[::2], 8, sop.SOP_C64, 1.0, out)        # not contiguous
    with pytest.raises(ValueError):
        sop.sop_norm_noalloc(psi, 16, sop.SOP_C64, 1.0, out.float())    # out not float64


def test_no_alloc_call_leaves_free_device_memory_unchanged():
    """After a first call (which may load the library's module, and with it
    the fixed scratch array), further calls allocate nothing: the device's
    free memory is the same before and after."""
    import torch
    psi = torch.ones(1 << 20, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sop.sop_norm_noalloc(psi, psi.numel(), sop.SOP_C64, 1.0, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        sop.sop_norm_noalloc(psi, psi.numel(), sop.SOP_C64, 1.0, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert out.item() == float(psi.numel())
