"""The three-dimensional four-component Dirac step on the GPU (alpha_3
couples all components; the 4x4 factors run inside four-component x and z
passes) against the oracle's 3D Dirac step, which the CPU tests
pin to exact free evolution with alpha_3, uniform-A convergence with all
three components and the energy."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def _case(dims, seed, steps):
    sp = tuple(2.0 / n for n in dims)
    psi0 = wl.random_smooth_state(dims, sp, seed, comps=4)
    X = wl.mesh(dims, sp)
    V = -1.0 / np.sqrt(sum(x * x for x in X) + 0.05) + 0.2 * wl.random_potential(dims, seed + 1)
    A = 15.0 * wl.random_field(steps, 3, seed + 2, 1.0)
    return sp, psi0, V, A


def _gpu_run(dims, sp, psi0, V, dt, steps, A, dtype, chunks=None):
    import torch
    p = sop.Propagator(dims, sp, 4, dtype)
    p.set_state(torch.from_numpy(psi0))
    if V is not None:
        p.set_potential(V)
    if chunks is None:
        p.step(steps, dt, A)
    else:
        done = 0
        for c in chunks:
            p.step(c, dt, None if A is None else A[done:done + c])
            done += c
    torch.cuda.synchronize()
    return p.state.cpu().numpy().astype(np.complex128), p


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("dims,steps", [((16, 12, 8), 12), ((32, 24, 16), 20), ((24, 16, 48), 8), ((64, 32, 32), 5)])
def test_dirac3d_matches_oracle(orc, dtype, dims, steps):
    sp, psi0, V, A = _case(dims, 70 + dims[0], steps)
    dt = 1e-4
    ref = orc.dirac_propagate(psi0, V, sp, dt, steps, A)
    out, p = _gpu_run(dims, sp, psi0, V, dt, steps, A, dtype)
    p.close()
    tol = gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT
    print(f"3D Dirac {dims} x {steps} {dtype}: relL2 {gc.relerr(out, ref):.3e}")
    assert gc.relerr(out, ref) < tol, gc.relerr(out, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac3d_free_and_split_calls(orc, dtype):
    dims, steps = (16, 16, 24), 15
    sp, psi0, _, A = _case(dims, 81, steps)
    ref = orc.dirac_propagate(psi0, None, sp, 1e-4, steps, None)
    out, p = _gpu_run(dims, sp, psi0, None, 1e-4, steps, None, dtype)
    p.close()
    assert gc.relerr(out, ref) < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT)
    one, p1 = _gpu_run(dims, sp, psi0, None, 1e-4, steps, A, dtype)
    split, p2 = _gpu_run(dims, sp, psi0, None, 1e-4, steps, A, dtype, chunks=(6, 1, 8))
    assert gc.relerr(split, one) < (1e-12 if dtype == "c128" else 2e-5)
    p1.close()
    p2.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac3d_norm_energy(orc, dtype):
    dims, steps = (32, 16, 16), 10
    sp, psi0, V, A = _case(dims, 82, steps)
    out, p = _gpu_run(dims, sp, psi0, V, 1e-4, steps, A, dtype)
    assert abs(p.norm() - orc.norm(psi0, sp, 4)) < (1e-11 if dtype == "c128" else 2e-5)
    e_ref = orc.energy(out, V, sp, 4)
    assert abs(p.energy() - e_ref) < (1e-9 if dtype == "c128" else 2e-5) * abs(e_ref)
    p.close()


def test_dirac3d_plane_wave_spectral(orc):
    """A free positive-energy plane wave with momentum along all three axes
    is an eigenstate of the split step: chi_n = exp(-i E t_n)."""
    import torch
    dims, sp = (16, 12, 8), (0.05, 0.06, 0.07)
    c = 137.036
    p = np.array([2 * np.pi * k / (n * h) for k, n, h in zip((2, -1, 1), dims, sp)])
    E = np.sqrt(c ** 4 + c * c * (p @ p))
    v = np.conj(orc.dirac_u(p)[0])
    X = wl.mesh(dims, sp)
    wave = np.exp(1j * (p[0] * X[0] + p[1] * X[1] + p[2] * X[2]))
    psi0 = np.stack([vk * wave for vk in v]) / np.sqrt(np.prod(np.array(dims) * np.array(sp)))
    q = sop.Propagator(dims, sp, 4, "c128")
    q.set_state(torch.from_numpy(psi0))
    chi, _, _ = q.spectral(40, 2e-4, [E], False)
    q.close()
    assert np.abs(chi - np.exp(-1j * E * 2e-4 * np.arange(41))).max() < 1e-10


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac3d_benchmark_workload_full_length(orc, dtype):
    """The benchmark's 3D Dirac workload (soft core a^2 = 0.01 on [-4,4)^3,
    A = (20 cos 2t, 5 sin 2t, 2), positive-energy packet sigma 0.5, p0 = (50,
    0, 0)) on a 64^3 lattice for 200 steps: the full-length FP32 bar 2e-4."""
    n, steps, dt = 64, 200, 1e-4
    h = 8.0 / n
    dims, sp = (n, n, n), (h, h, h)
    X = wl.mesh(dims, sp)
    V = -1.0 / np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2 + 0.01)
    psi0 = wl.dirac_positive_spin_up(wl.gaussian(dims, sp, (0.0, 0.0, 0.0), 0.5, (50.0, 0.0, 0.0)), dims, sp)
    t = (np.arange(steps) + 0.5) * dt
    A = np.stack([20.0 * np.cos(2.0 * t), 5.0 * np.sin(2.0 * t), 2.0 * np.ones_like(t)], axis=1)
    ref = orc.dirac_propagate(psi0, V, sp, dt, steps, A)
    out, p = _gpu_run(dims, sp, psi0, V, dt, steps, A, dtype)
    p.close()
    err = gc.relerr(out, ref)
    print(f"3D Dirac 64^3 x {steps} {dtype}: relL2 {err:.3e}")
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL), err
