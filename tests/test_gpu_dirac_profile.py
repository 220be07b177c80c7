"""Dirac steps with a vector potential that varies along x_1 (a plane-wave
pulse travelling along x_1, as in the paper's scattering example) on the GPU
against the oracle's per-column mixing, which the CPU tests pin to the
uniform case, translation covariance and a NumPy composition of the pinned
factors."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def _pulse(n_steps, dims, sp, dt, nd, seed):
    """A_y (and a small A_x, A_z) = A0 sin(k x - w t) f(k x - w t): a pulse
    moving along x_1 with a random phase; A0 = 40 a.u."""
    rng = np.random.default_rng(seed)
    L = dims[0] * sp[0]
    x = wl.lattice(dims[0], sp[0])
    k = 2 * np.pi / L
    w = 137.036 * k
    t = (np.arange(n_steps) + 0.5) * dt
    eta = k * x[None, :] - w * t[:, None] + rng.uniform(0, 2 * np.pi)
    env = np.exp(-((eta % (2 * np.pi)) - np.pi) ** 2)
    A = np.zeros((n_steps, dims[0], nd))
    A[:, :, 1] = 40.0 * np.sin(eta) * env
    A[:, :, 0] = 5.0 * np.cos(eta) * env
    if nd == 3:
        A[:, :, 2] = 3.0 * env
    return A


def _run(dims, sp, psi0, V, dt, steps, A, dtype, chunks=None):
    import torch
    p = sop.Propagator(dims, sp, 4, dtype)
    p.set_field_profile(True)
    p.set_state(torch.from_numpy(psi0))
    if V is not None:
        p.set_potential(V)
    if chunks is None:
        p.step(steps, dt, A)
    else:
        done = 0
        for c in chunks:
            p.step(c, dt, A[done:done + c])
            done += c
    torch.cuda.synchronize()
    out = p.state.cpu().numpy().astype(np.complex128)
    return out, p


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("dims,steps", [((32, 24), 70), ((48, 32), 20), ((16, 12, 8), 10), ((24, 16, 16), 66)])
def test_profile_matches_oracle(orc, dtype, dims, steps):
    nd = len(dims)
    sp = tuple(4.0 / n for n in dims)
    psi0 = wl.random_smooth_state(dims, sp, 90 + nd, comps=4)
    X = wl.mesh(dims, sp)
    V = -1.0 / np.sqrt(sum(x * x for x in X) + 0.05)
    dt = 1e-4
    A = _pulse(steps, dims, sp, dt, nd, 91)
    ref = orc.dirac_propagate_profile(psi0, V, sp, dt, steps, A)
    out, p = _run(dims, sp, psi0, V, dt, steps, A, dtype)
    p.close()
    tol = gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT
    print(f"profile {dims} x {steps} {dtype}: relL2 {gc.relerr(out, ref):.3e}")
    assert gc.relerr(out, ref) < tol, gc.relerr(out, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_profile_benchmark_workload_full_length(orc, dtype):
    """The benchmark's pulse workload (config-4 packet and soft core, A_y of a
    pulse travelling along x) on a 256^2 lattice for the config's full 1000
    steps: the full-length FP32 bar 2e-4."""
    w = wl.config4(n=256, n_steps=1000)
    n, T = w.dims[0], w.n_steps
    x = wl.lattice(n, w.spacing[0])
    kx = 2 * np.pi / (n * w.spacing[0])
    t = (np.arange(T) + 0.5) * w.dt
    eta = kx * x[None, :] - 137.036 * kx * t[:, None]
    A = np.zeros((T, n, 2))
    A[:, :, 1] = 20.0 * np.sin(eta) * np.sin(0.5 * eta) ** 2
    ref = orc.dirac_propagate_profile(w.psi0, w.V, w.spacing, w.dt, T, A)
    out, p = _run(w.dims, w.spacing, w.psi0, w.V, w.dt, T, A, dtype)
    p.close()
    err = gc.relerr(out, ref)
    print(f"pulse 256^2 x {T} {dtype}: relL2 {err:.3e}")
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL), err


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_profile_split_calls_and_uniform(orc, dtype):
    """Split calls equal one call (rounding); a column-independent profile
    gives the uniform-A result of the fused 2D path."""
    import torch
    dims, sp, steps = (32, 16), (0.1, 0.12), 40
    psi0 = wl.random_smooth_state(dims, sp, 95, comps=4)
    A = _pulse(steps, dims, sp, 1e-4, 2, 96)
    one, p1 = _run(dims, sp, psi0, None, 1e-4, steps, A, dtype)
    split, p2 = _run(dims, sp, psi0, None, 1e-4, steps, A, dtype, chunks=(17, 1, 22))
    p1.close()
    p2.close()
    assert gc.relerr(split, one) < (1e-12 if dtype == "c128" else 2e-5)
    Au = wl.random_field(steps, 2, 97, 30.0)
    prof = np.repeat(Au[:, None, :], dims[0], axis=1)
    a, pa = _run(dims, sp, psi0, None, 1e-4, steps, prof, dtype)
    pa.close()
    q = sop.Propagator(dims, sp, 4, dtype)
    q.set_state(torch.from_numpy(psi0))
    q.step(steps, 1e-4, Au)
    b = q.state.cpu().numpy().astype(np.complex128)
    q.close()
    assert gc.relerr(a, b) < (1e-12 if dtype == "c128" else 2e-5)


def test_profile_errors():
    p = sop.Propagator((32, 32), (0.1, 0.1), 1, "c64")
    with pytest.raises(sop.SopError):
        p.set_field_profile(True)
    p.close()
    q = sop.Propagator((64,), (0.1,), 2, "c64")
    with pytest.raises(sop.SopError):
        q.set_field_profile(True)
    q.close()
