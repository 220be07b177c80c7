"""The one-dimensional two-component Dirac equation on the GPU (components =
2, the whole-step kernel) against the oracle's 1D Dirac step, which the CPU
tests pin to exact free evolution, the (1,4) pair of the 2D four-component
step and uniform-A convergence."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def _case(n, seed, steps, h=None, field=True):
    h = (8.0 / n) if h is None else h
    psi0 = wl.random_smooth_state((n,), (h,), seed, comps=2)
    X = wl.lattice(n, h)
    V = -1.0 / np.sqrt(X * X + 0.01) + 0.1 * wl.random_potential((n,), seed + 1)
    A = 20.0 * wl.random_field(steps, 1, seed + 2, 1.0)[:, 0] if field else None
    return (h,), psi0, V, A


def _gpu_run(n, sp, psi0, V, dt, steps, A, dtype, chunks=None):
    import torch
    p = sop.Propagator((n,), sp, 2, dtype)
    p.set_state(torch.from_numpy(psi0))
    if V is not None:
        p.set_potential(V)
    if chunks is None:
        p.step(steps, dt, None if A is None else A.reshape(steps, 1))
    else:
        done = 0
        for c in chunks:
            p.step(c, dt, None if A is None else A[done:done + c].reshape(c, 1))
            done += c
    torch.cuda.synchronize()
    out = p.state.cpu().numpy().astype(np.complex128)
    return out, p


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,steps", [(8, 5), (12, 7), (96, 60), (256, 200), (1024, 100), (3072, 20), (4096, 30)])
def test_dirac1d_matches_oracle(orc, dtype, n, steps):
    sp, psi0, V, A = _case(n, 50 + n, steps)
    dt = 1e-4
    ref = orc.dirac1d_propagate(psi0, V, sp, dt, steps, A)
    out, p = _gpu_run(n, sp, psi0, V, dt, steps, A, dtype)
    p.close()
    tol = gc.TOL_F64 if dtype == "c128" else (gc.TOL_F32_FULL if steps >= 100 else gc.TOL_F32_SHORT)
    assert out.shape == (2, n)
    assert gc.relerr(out, ref) < tol, gc.relerr(out, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac1d_no_field_no_potential(orc, dtype):
    n, steps = 512, 40
    sp, psi0, _, _ = _case(n, 61, steps)
    ref = orc.dirac1d_propagate(psi0, None, sp, 1e-4, steps)
    out, p = _gpu_run(n, sp, psi0, None, 1e-4, steps, None, dtype)
    p.close()
    assert gc.relerr(out, ref) < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac1d_split_calls_norm_energy(orc, dtype):
    """Calls of 30 + 1 + 49 steps equal one call of 80 (rounding); norm is
    kept; energy matches the oracle's on the GPU state."""
    n, steps = 768, 80
    sp, psi0, V, A = _case(n, 62, steps)
    one, p1 = _gpu_run(n, sp, psi0, V, 1e-4, steps, A, dtype)
    split, p2 = _gpu_run(n, sp, psi0, V, 1e-4, steps, A, dtype, chunks=(30, 1, 49))
    assert gc.relerr(split, one) < (1e-12 if dtype == "c128" else 2e-5)
    assert abs(p1.norm() - orc.norm(psi0, sp, 2)) < (1e-11 if dtype == "c128" else 2e-5)
    e_ref = orc.energy(one, V, sp, 2)
    assert abs(p1.energy() - e_ref) < (1e-9 if dtype == "c128" else 2e-5) * abs(e_ref)
    p1.close()
    p2.close()


def test_dirac1d_plane_wave_spectral(orc):
    """A positive-energy plane wave, u(p)^dag e_1 e^{ipx}, is an eigenstate of
    the split step: the spectral method's chi_n is exp(-i E t_n)."""
    import torch
    n, h, c = 256, 0.02, 137.036
    p0 = 2 * np.pi * 5 / (n * h)
    E = np.sqrt(c ** 4 + c * c * p0 * p0)
    v = np.conj(orc.dirac1d_u(p0)[0])
    x = wl.lattice(n, h)
    psi0 = np.stack([vk * np.exp(1j * p0 * x) for vk in v]) / np.sqrt(n * h)
    q = sop.Propagator((n,), (h,), 2, "c128")
    q.set_state(torch.from_numpy(psi0))
    dt, N = 2e-4, 100
    chi, _, _ = q.spectral(N, dt, [E], False)
    q.close()
    assert np.abs(chi - np.exp(-1j * E * dt * np.arange(N + 1))).max() < 1e-10


def test_dirac1d_plan_errors():
    with pytest.raises(sop.SopError):
        sop.Propagator((32, 32), (0.1, 0.1), 2, "c64")
    p = sop.Propagator((64,), (0.1,), 2, "c64")
    with pytest.raises(sop.SopError):
        p.set_gauge("velocity")
    p.close()
