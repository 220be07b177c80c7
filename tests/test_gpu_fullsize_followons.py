"""Full-size parity of the follow-on forms in the launch configurations the
benchmark times: the spectral method on the 2048^2 soft-core lattice, the
velocity gauge on the benchmark lattice, the 3D four-component Dirac step at
128^3 and the Dirac pulse along x at 1024^2, each for a few steps against the
oracle (which needs seconds per step at these sizes)."""
import numpy as np
import pytest

import gpu_cases as gc
from oracle import spectral as osp
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def test_spectral_2048_vs_oracle():
    import torch
    n, h, N = 2048, 0.2, 16
    V = wl.soft_core((n, n), (h, h), 0.791 ** 2)
    psi0 = wl.gaussian((n, n), (h, h), (0.5, -0.3), 1.2)
    E = [-0.55, -0.5, -0.45]
    chi_r, spec_r, psiE_r = osp.spectral(psi0, V, (h, h), 0.05, N, E)
    q = sop.Propagator((n, n), (h, h), 1, "c64")
    q.set_state(torch.from_numpy(psi0))
    q.set_potential(V)
    chi, spec, psiE = q.spectral(N, 0.05, E, True)
    q.close()
    assert np.abs(chi - chi_r).max() < 2e-5
    assert np.abs(spec - spec_r).max() < 2e-5 * np.abs(spec_r).max()
    assert np.abs(psiE.cpu().numpy() - psiE_r).max() < 2e-5 * np.abs(psiE_r).max()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_velocity_gauge_2048_vs_oracle(orc, dtype):
    import torch
    w = wl.config2()
    A = -np.cumsum(w.field, axis=0)[:2] * w.dt + 0.3
    ref = orc.schrodinger_propagate(w.psi0, w.V, w.spacing, w.dt, 2, A, gauge="velocity")
    p = sop.Propagator(w.dims, w.spacing, 1, dtype)
    p.set_gauge("velocity")
    p.set_state(torch.from_numpy(w.psi0))
    p.set_potential(w.V)
    p.step(2, w.dt, A)
    out = p.state.cpu().numpy().astype(np.complex128)
    p.close()
    assert gc.relerr(out, ref) < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac3d_128_vs_oracle(orc, dtype):
    import torch
    n = 128
    h = 8.0 / n
    dims, sp = (n, n, n), (h, h, h)
    X = wl.mesh(dims, sp)
    V = -1.0 / np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2 + 0.01)
    psi0 = wl.dirac_positive_spin_up(wl.gaussian(dims, sp, (0.0, 0.0, 0.0), 0.5, (50.0, 0.0, 0.0)), dims, sp)
    A = np.array([[20.0, 5.0, 2.0], [19.0, 6.0, 2.0]])
    ref = orc.dirac_propagate(psi0, V, sp, 1e-4, 2, A)
    p = sop.Propagator(dims, sp, 4, dtype)
    p.set_state(torch.from_numpy(psi0))
    p.set_potential(V)
    p.step(2, 1e-4, A)
    out = p.state.cpu().numpy().astype(np.complex128)
    p.close()
    assert gc.relerr(out, ref) < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac_pulse_1024_vs_oracle(orc, dtype):
    import torch
    w = wl.config4(n_steps=2)
    n = w.dims[0]
    x = wl.lattice(n, w.spacing[0])
    k = 2 * np.pi / (n * w.spacing[0])
    eta = k * x[None, :] - 137.036 * k * ((np.arange(2) + 0.5) * w.dt)[:, None]
    A = np.zeros((2, n, 2))
    A[:, :, 1] = 20.0 * np.sin(eta) * np.sin(0.5 * eta) ** 2
    A[:, :, 0] = 3.0
    ref = orc.dirac_propagate_profile(w.psi0, w.V, w.spacing, w.dt, 2, A)
    p = sop.Propagator(w.dims, w.spacing, 4, dtype)
    p.set_field_profile(True)
    p.set_state(torch.from_numpy(w.psi0))
    p.set_potential(w.V)
    p.step(2, w.dt, A)
    out = p.state.cpu().numpy().astype(np.complex128)
    p.close()
    assert gc.relerr(out, ref) < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT)
