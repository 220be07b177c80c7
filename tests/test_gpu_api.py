"""Behaviour of the C ABI on the GPU: state checks, no-op and identity steps,
host-buffer stepping, streams, profiling counters and invariants of the
unitary, time-symmetric step (norm, reversibility) on the GPU path itself."""
import ctypes

import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import sop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    gc.require_gpu()


def test_step_before_bind_is_a_state_error():
    plan = sop.sop_plan_create((16, 16), (0.1, 0.1), 1, sop.SOP_C64)
    try:
        with pytest.raises(sop.SopError) as ei:
            sop.sop_step(plan, 1, 0.1)
        assert ei.value.status == sop.SOP_ESTATE
        with pytest.raises(sop.SopError):
            sop.sop_norm(plan)
    finally:
        sop.sop_plan_destroy(plan)


def test_misaligned_state_is_rejected():
    import torch
    buf = torch.zeros(2 * 16 * 16 + 2, dtype=torch.float32, device="cuda")
    plan = sop.sop_plan_create((16, 16), (0.1, 0.1), 1, sop.SOP_C64)
    try:
        rc = sop.load().sop_bind_state(plan, buf.data_ptr() + 4)
        assert rc == sop.SOP_EINVAL
    finally:
        sop.sop_plan_destroy(plan)


def test_bad_step_arguments():
    w = gc.random_workload((16, 16), 1, seed=1, n_steps=1, dt=0.1, field_scale=0.0)
    _, prop = gc.run_gpu(w, "c64", n_steps=0)
    with pytest.raises(sop.SopError) as ei:
        sop.sop_step(prop.plan, -1, 0.1)
    assert ei.value.status == sop.SOP_EINVAL
    with pytest.raises(sop.SopError):
        sop.sop_step(prop.plan, 1, float("nan"))
    with pytest.raises(sop.SopError):
        sop.sop_step(prop.plan, 1, 0.1, np.array([[np.inf, 0.0]]), 2)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_zero_steps_is_a_no_op(dtype):
    w = gc.random_workload((32, 16), 1, seed=2, n_steps=1, dt=0.1, field_scale=0.1)
    out, prop = gc.run_gpu(w, dtype, n_steps=0)
    assert np.array_equal(out, w.psi0.astype(np.complex64 if dtype == "c64" else np.complex128))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_zero_dt_is_identity_up_to_rounding(dtype):
    w = gc.random_workload((64, 48), 1, seed=3, n_steps=3, dt=0.0, field_scale=0.1)
    out, _ = gc.run_gpu(w, dtype)
    assert gc.relerr(out, w.psi0) < (1e-14 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("comps,dims", [(1, (48, 32)), (1, (16, 12, 8)), (4, (32, 16)), (1, (256,))])
def test_step_host_matches_device_path(dtype, comps, dims):
    import torch
    w = gc.random_workload(dims, comps, seed=4, n_steps=3, dt=1e-3, field_scale=0.2, v_scale=2.0)
    out_dev, prop = gc.run_gpu(w, dtype)
    host = torch.from_numpy(w.psi0.astype(np.complex64 if dtype == "c64" else np.complex128)).pin_memory()
    prop.step_host(host, 3, w.dt, w.field)
    assert np.array_equal(host.numpy(), out_dev.astype(host.numpy().dtype))


def test_non_default_stream():
    import torch
    w = gc.random_workload((64, 32), 1, seed=6, n_steps=4, dt=0.05, field_scale=0.2)
    ref, _ = gc.run_gpu(w, "c128")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out, _ = gc.run_gpu(w, "c128", stream=s)
    assert np.array_equal(out, ref)


def test_profiling_counts_passes():
    w = gc.random_workload((64, 32), 1, seed=7, n_steps=5, dt=0.05, field_scale=0.2)
    _, prop = gc.run_gpu(w, "c64", n_steps=0)
    sop.sop_profile_enable(prop.plan, True)
    before = sop.sop_launch_counter(prop.plan)
    prop.step(5, w.dt, w.field)
    ms, n = sop.sop_profile_read(prop.plan)
    assert n[0] == 6 and n[1] == 5          # real-space passes n+1, momentum passes n
    assert all(t >= 0 for t in ms) and ms[0] > 0 and ms[1] > 0
    # the counter counts kernels; a profiled set-up bracket may hold several
    assert sop.sop_launch_counter(prop.plan) - before >= sum(n)
    sop.sop_profile_read(prop.plan)
    before = sop.sop_launch_counter(prop.plan)
    prop.step(5, w.dt, w.field)               # tables for this dt exist now
    ms, n = sop.sop_profile_read(prop.plan)
    assert n[4] == 1                          # one field-table build per chunk
    assert sop.sop_launch_counter(prop.plan) - before == sum(n)
    # sampled: passes of split steps P = 2 mod 4 only (real-space P = 0..10)
    sop.sop_profile_enable(prop.plan, 4)
    before = sop.sop_launch_counter(prop.plan)
    prop.step(10, w.dt, np.concatenate([w.field, w.field]))
    ms, n = sop.sop_profile_read(prop.plan)
    assert n[0] == 3 and n[1] == 2 and n[4] == 1
    assert ms[0] > 0 and ms[1] > 0
    assert sop.sop_launch_counter(prop.plan) - before == 11 + 10 + 1
    sop.sop_profile_enable(prop.plan, 0)
    prop.step(5, w.dt, w.field)
    ms, n = sop.sop_profile_read(prop.plan)
    assert sum(n) == 0
    with pytest.raises(sop.SopError):
        sop.sop_profile_enable(prop.plan, -1)


@pytest.mark.parametrize("comps,dims,dt", [(1, (96, 64), 0.05), (1, (24, 16, 32), 0.05), (4, (64, 48), 1e-4)])
def test_norm_conservation_and_reversibility_fp64(comps, dims, dt):
    import torch
    w = gc.random_workload(dims, comps, seed=8, n_steps=40, dt=dt, field_scale=0.3 if comps == 1 else 20.0,
                           v_scale=2.0)
    out, prop = gc.run_gpu(w, "c128")
    n0 = np.sum(np.abs(w.psi0) ** 2) * np.prod(w.spacing)
    assert abs(prop.norm() - n0) < 1e-12 * n0
    prop.step(40, -dt, w.field[::-1].copy())
    torch.cuda.synchronize()
    back = prop.state.cpu().numpy()
    assert gc.relerr(back, w.psi0) < 1e-11
