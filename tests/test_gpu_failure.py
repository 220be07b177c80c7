"""Failure detection of the persistent passes without faulting the GPU: a
wait limit of 1 ns makes the pass kernels' tile-copy waits give up while the
copies themselves complete normally.  The next synchronising call must report
SOP_ETIMEOUT, and after the default limit is restored the same plan must step
correctly again (element by element against the oracle)."""
import numpy as np
import pytest
import torch

import gpu_cases as gc
from paper_1012_3911_gb300 import sop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("dims", [(2048, 2048), (128, 192, 256)])
def test_bounded_wait_gives_up_then_the_plan_recovers(dtype, dims):
    """Lattices with several tiles per CTA and single-buffer launch shapes
    (complex128 strided passes keep one buffer by default), so that each CTA
    waits for a tile whose copy was issued just before the wait."""
    w = gc.random_workload(dims, 1, seed=31 + len(dims), n_steps=4, dt=0.01, field_scale=0.05)
    prop = sop.Propagator(w.dims, w.spacing, 1, dtype)
    prop.set_state(torch.from_numpy(w.psi0))
    prop.set_potential(w.V)
    prop.set_pass_shape(0, 1)   # one pencil group per CTA, one tile buffer
    prop.set_pass_shape(1, 1)
    sop.sop_set_wait_limit(prop.plan, 1)
    status = None
    for _ in range(5):   # a wait gives up unless every copy landed before its first poll
        prop.step(w.n_steps, w.dt, w.field)
        try:
            prop.norm()
        except sop.SopError as e:
            status = e.status
            break
    assert status == sop.SOP_ETIMEOUT
    assert "bounded wait" in sop.sop_last_error()
    # the error word and the tile counters were cleared by that report
    sop.sop_set_wait_limit(prop.plan, 0)
    prop.set_state(torch.from_numpy(w.psi0))
    prop.step(w.n_steps, w.dt, w.field)
    assert abs(prop.norm() - gc.oracle.norm(w.psi0, w.spacing)) < 1e-4
    out = prop.state.cpu().numpy()
    ref = gc.run_oracle(w)
    err = gc.relerr(out, ref)
    prop.close()
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT), err


def test_every_allocation_failure_of_plan_creation_is_reported_and_cleaned_up():
    """Injected out-of-memory at each device allocation of plan creation,
    potential set-up and a first step in turn: the call that needed it returns
    SOP_ENOMEM, nothing leaks (free memory returns to its level), and once the
    injection is off the same sequence succeeds and matches the oracle."""
    w = gc.random_workload((64, 48), 1, seed=7, n_steps=3, dt=0.01, field_scale=0.05)

    def sequence():
        p = sop.Propagator(w.dims, w.spacing, 1, "c64")
        try:
            p.set_state(torch.from_numpy(w.psi0))
            p.set_potential(w.V)
            p.step(w.n_steps, w.dt, w.field)
            torch.cuda.synchronize()
            return p.state.cpu().numpy()
        finally:
            p.close()

    sequence()                       # warm: library loaded, kernels and caches set up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(64):
        sop.sop_debug_fail_alloc(k)
        try:
            sequence()
        except sop.SopError as e:
            assert e.status == sop.SOP_ENOMEM, e
            assert "injected" in str(e)
            failures += 1
            continue
        finally:
            sop.sop_debug_fail_alloc(-1)
        break                        # k exceeds the allocations the sequence makes
    assert failures >= 5
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    out = sequence()
    assert gc.relerr(out, gc.run_oracle(w)) < gc.TOL_F32_SHORT


def test_non_finite_potential_is_rejected():
    w = gc.random_workload((32, 24), 1, seed=8, n_steps=2, dt=0.01, field_scale=0.0)
    p = sop.Propagator(w.dims, w.spacing, 1, "c64")
    V = w.V.copy()
    V[3, 5] = np.nan
    with pytest.raises(sop.SopError) as ei:
        p.set_potential(V)
    assert ei.value.status == sop.SOP_EINVAL and "finite" in str(ei.value)
    p.set_potential(w.V)             # a finite potential afterwards is accepted
    p.close()
