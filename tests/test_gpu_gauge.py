"""Velocity-gauge Schroedinger steps on the GPU (sop_set_gauge; Eq. 13 with
the vector potential) against the oracle's velocity-gauge step, which the CPU
tests pin to exact plane-wave phases and the lattice-momentum gauge shift."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def _run(w, dtype, gauge, field, n=None, chunks=None):
    import torch
    n = w.n_steps if n is None else n
    p = sop.Propagator(w.dims, w.spacing, 1, dtype)
    p.set_gauge(gauge)
    p.set_state(torch.from_numpy(w.psi0))
    if w.V is not None:
        p.set_potential(w.V)
    if chunks is None:
        p.step(n, w.dt, field)
    else:
        done = 0
        for c in chunks:
            p.step(c, w.dt, None if field is None else field[done:done + c])
            done += c
    torch.cuda.synchronize()
    out = p.state.cpu().numpy().astype(np.complex128)
    p.close()
    return out


def _case(dims, n, seed, zero_axes=()):
    w = gc.random_workload(dims, 1, seed, n, 0.02, 0.0, v_scale=0.5)
    A = wl.random_field(n, len(dims), seed + 5, 3.0) + 0.5
    for a in zero_axes:
        A[:, a] = 0.0
    return w, A


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("dims,n,zero", [((256,), 600, ()), ((64, 48), 530, ()), ((96, 64), 40, (0,)),
                                         ((32, 24, 16), 30, ()), ((24, 16, 32), 12, (1,))])
def test_velocity_gauge_matches_oracle(orc, dtype, dims, n, zero):
    """Random A (some components zero), random potential; step counts that
    cross the 512-step boundary of the kinetic rows."""
    w, A = _case(dims, n, 40 + len(dims), zero)
    ref = orc.schrodinger_propagate(w.psi0, w.V, w.spacing, w.dt, n, A, gauge="velocity")
    out = _run(w, dtype, "velocity", A)
    tol = gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL
    assert gc.relerr(out, ref) < tol, gc.relerr(out, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_velocity_gauge_split_calls(dtype):
    """One call of 700 steps equals calls of 300, 1 and 399 steps up to the
    merging of the real-space halves (rounding only)."""
    w, A = _case((128, 96), 700, 77)
    one = _run(w, dtype, "velocity", A)
    split = _run(w, dtype, "velocity", A, chunks=(300, 1, 399))
    assert gc.relerr(split, one) < (1e-12 if dtype == "c128" else 2e-5)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_velocity_gauge_zero_field_is_field_free(dtype):
    """A = 0 keeps the plan's own kinetic tables: bit-identical to no field."""
    w, A = _case((64, 48), 20, 78)
    A[:] = 0.0
    assert np.array_equal(_run(w, dtype, "velocity", A), _run(w, dtype, "length", None))


def test_velocity_gauge_lattice_shift_on_gpu():
    """q A a lattice momentum: psi_vel = G U_0 G^dag psi (G = exp(i q A.x)),
    both sides on the GPU in complex128 (the relation the oracle pin checks)."""
    dims, sp = (48, 32), (0.3, 0.4)
    L = np.array(dims) * np.array(sp)
    q = -1.0
    A = (2 * np.pi * np.array([2.0, -1.0]) / L) / q
    X = wl.mesh(dims, sp)
    G = np.exp(1j * q * (A[0] * X[0] + A[1] * X[1]))
    V = -2.0 * np.exp(-(X[0] ** 2 + X[1] ** 2) / (2 * 1.5 ** 2))
    psi0 = wl.gaussian(dims, sp, (0.5, -0.4), 1.0)
    n = 12
    wv = wl.Workload("shift", dims, sp, 1, psi0, V, 0.05, n, None)
    wf = wl.Workload("shift0", dims, sp, 1, np.conj(G) * psi0, V, 0.05, n, None)
    vel = _run(wv, "c128", "velocity", np.tile(A, (n, 1)))
    ref = G * _run(wf, "c128", "length", None)
    assert gc.relerr(vel, ref) < 1e-10


def test_gauge_argument_errors():
    import torch
    p = sop.Propagator((32, 32), (0.1, 0.1), 1, "c64")
    with pytest.raises(sop.SopError):
        sop.sop_set_gauge(p.plan, 2)
    p.set_gauge("velocity")
    p.set_state(torch.from_numpy(wl.gaussian((32, 32), (0.1, 0.1), (0.0, 0.0), 0.5)))
    phi = torch.zeros_like(p.state)
    with pytest.raises(sop.SopError):
        p.adjoint_gradient(phi, 4, 0.01)
    with pytest.raises(sop.SopError):
        sop.Batch([p])
    p.set_gauge("length")
    p.adjoint_gradient(phi, 4, 0.01)
    p.close()
    d = sop.Propagator((32, 32), (0.1, 0.1), 4, "c64")
    with pytest.raises(sop.SopError):
        d.set_gauge("velocity")
    d.close()
