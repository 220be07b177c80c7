"""The spectral method for eigenstates on the GPU (sop_spectral) against the
oracle's FP64 spectral method, which the CPU tests pin to plane-wave phases,
harmonic levels and lattice diagonalisation; plus the eigenstates
subsection's soft-core statements (zeta = 1.4133 in 1D, 0.791 in 2D: ground
state near -1/2) and an exact Dirac plane-wave autocorrelation."""
import numpy as np
import pytest
import scipy.linalg as sl

import gpu_cases as gc
from oracle import spectral as osp
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def _gpu_spectral(dims, spacing, psi0, V, dt, N, energies, dtype, eigen=True, comps=1):
    import torch
    p = sop.Propagator(dims, spacing, comps, dtype)
    p.set_state(torch.from_numpy(psi0))
    if V is not None:
        p.set_potential(V)
    chi, spec, psiE = p.spectral(N, dt, energies, eigen)
    out = (chi, spec, None if psiE is None else psiE.cpu().numpy(), p.state.cpu().numpy())
    p.close()
    return out


def _soft_core_case(dims, seed):
    """A soft-core well (the eigenstates subsection's potential) with a small
    random perturbation, an off-centre Gaussian trial state."""
    sp = (0.15, 0.16, 0.17)[:len(dims)]
    V = wl.soft_core(dims, sp, 0.791 ** 2) + 0.05 * wl.random_potential(dims, seed)
    psi0 = wl.gaussian(dims, sp, [0.4] + [-0.3] * (len(dims) - 1), 1.1)
    return sp, V, psi0


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("dims,N", [((256,), 300), ((96,), 64), ((64, 48), 120), ((32, 24, 16), 40),
                                    ((48, 24), 1)])
def test_spectral_matches_oracle(orc, dtype, dims, N):
    sp, V, psi0 = _soft_core_case(dims, 31)
    Es = np.array([-0.55, -0.5, -0.31, 0.0, 0.4])
    dt = 0.05
    chi_r, spec_r, psiE_r = osp.spectral(psi0, V, sp, dt, N, Es)
    chi, spec, psiE, psiN = _gpu_spectral(dims, sp, psi0, V, dt, N, Es, dtype)
    tol = 1e-10 if dtype == "c128" else 2e-4
    assert chi.shape == (N + 1,) and spec.shape == (len(Es),) and psiE.shape == (len(Es),) + psi0.shape
    assert np.abs(chi - chi_r).max() <= tol, np.abs(chi - chi_r).max()
    smax = max(np.abs(spec_r).max(), 1e-300)
    assert np.abs(spec - spec_r).max() <= tol * max(smax, dt), np.abs(spec - spec_r).max() / smax
    pmax = np.abs(psiE_r).max()
    assert np.abs(psiE - psiE_r).max() <= tol * max(pmax, dt * np.abs(psi0).max())
    # the bound state ends at psi_N
    ref_N = orc.schrodinger_propagate(psi0, V, sp, dt, N, None)
    assert gc.relerr(psiN, ref_N) <= tol


def test_spectral_without_energies_and_eigenfunctions():
    """K = 0 gives chi alone; eigenfunctions off leaves the spectrum equal."""
    dims = (64, 48)
    sp, V, psi0 = _soft_core_case(dims, 32)
    chi0, spec0, _, _ = _gpu_spectral(dims, sp, psi0, V, 0.05, 50, [], "c128", eigen=False)
    assert spec0.shape == (0,)
    chi1, spec1, psiE1, _ = _gpu_spectral(dims, sp, psi0, V, 0.05, 50, [-0.4, 0.1], "c128", eigen=False)
    chi2, spec2, psiE2, _ = _gpu_spectral(dims, sp, psi0, V, 0.05, 50, [-0.4, 0.1], "c128", eigen=True)
    assert psiE1 is None and psiE2 is not None
    assert np.array_equal(chi0, chi1) and np.array_equal(chi1, chi2) and np.array_equal(spec1, spec2)


def test_spectral_argument_errors():
    import torch
    dims = (32, 32)
    sp, V, psi0 = _soft_core_case(dims, 33)
    p = sop.Propagator(dims, sp, 1, "c128")
    p.set_state(torch.from_numpy(psi0))
    too_many = np.linspace(-1, 1, sop.SOP_SPECTRAL_MAX_EIGEN + 1)
    with pytest.raises(sop.SopError):
        p.spectral(10, 0.05, too_many, True)
    with pytest.raises(sop.SopError):
        p.spectral(0, 0.05, [0.0])
    with pytest.raises(sop.SopError):
        p.spectral(10, 0.0, [0.0])
    with pytest.raises(sop.SopError):
        p.spectral(10, 0.05, [np.nan])
    # nothing ran: the state is unchanged
    assert np.array_equal(p.state.cpu().numpy(), psi0)
    # a spectrum scan may take any number of energies without eigenfunctions
    _, spec, _ = p.spectral(10, 0.05, too_many, False)
    assert spec.shape == too_many.shape
    p.close()


def _lattice_h1(n, L, V):
    h = L / n
    k = 2 * np.pi * np.fft.fftfreq(n, d=h)
    F = np.fft.fft(np.eye(n), axis=0)
    T = np.real(np.conj(F).T @ np.diag(k ** 2 / 2) @ F) / n
    return T + np.diag(V)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_soft_core_1d_ground_state(dtype):
    """zeta = 1.4133: the 1D soft-core ground state lies at about -1/2; the
    GPU spectrum peaks at the lattice Hamiltonian's lowest eigenvalue and
    Psi_E there is its eigenvector."""
    n, L, dt, N = 512, 80.0, 0.05, 4000
    sp = (L / n,)
    V = wl.soft_core((n,), sp, 1.4133 ** 2)
    evals, evecs = sl.eigh(_lattice_h1(n, L, V))
    psi0 = wl.gaussian((n,), sp, (0.7,), 1.5)
    Es = np.linspace(-0.6, -0.4, 801)
    _, spec, _, _ = _gpu_spectral((n,), sp, psi0, V, dt, N, Es, dtype, eigen=False)
    e0 = osp.peak(Es, spec)
    assert abs(e0 + 0.5) < 2e-3
    assert abs(e0 - evals[0]) < 5e-4, (e0, evals[0])
    _, _, psiE, _ = _gpu_spectral((n,), sp, psi0, V, dt, N, [e0], dtype)
    v = psiE[0] / np.linalg.norm(psiE[0])
    assert abs(np.vdot(evecs[:, 0], v)) > 0.999


def test_soft_core_2d_ground_state():
    """zeta = 0.791 in 2D: ground state near -1/2, found on a 256^2 lattice in
    complex64 with 4000 steps."""
    n, L, dt, N = 256, 40.0, 0.05, 4000
    sp = (L / n, L / n)
    V = wl.soft_core((n, n), sp, 0.791 ** 2)
    psi0 = wl.gaussian((n, n), sp, (0.5, -0.3), 1.2)
    Es = np.linspace(-0.6, -0.4, 401)
    _, spec, _, _ = _gpu_spectral((n, n), sp, psi0, V, dt, N, Es, "c64", eigen=False)
    assert abs(osp.peak(Es, spec) + 0.5) < 6e-3


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_dirac_plane_wave_autocorrelation(orc, dtype):
    """A free positive-energy Dirac plane wave is an eigenstate of the split
    step (the kinetic factor of Eq. 33 is exact per momentum): chi_n =
    exp(-i E t_n) with E = sqrt(m^2 c^4 + c^2 p^2), and the spectrum peaks at E."""
    dims, sp = (32, 24), (0.05, 0.06)
    c = 137.036
    p = np.array([2 * np.pi * 3 / (dims[0] * sp[0]), -2 * np.pi * 2 / (dims[1] * sp[1])])
    E = np.sqrt(c ** 4 + c * c * (p @ p))
    v = np.conj(orc.dirac_u(p)[0])   # the positive-energy spinor
    H = orc.dirac_h(p)
    assert np.abs(H @ v - E * v).max() < 1e-9 * E
    X = wl.mesh(dims, sp)
    wave = np.exp(1j * (p[0] * X[0] + p[1] * X[1]))
    psi0 = np.stack([vk * wave for vk in v]) / np.sqrt(dims[0] * sp[0] * dims[1] * sp[1])
    dt, N = 2e-4, 200
    Es = E + np.linspace(-300.0, 300.0, 61)
    chi, spec, _, _ = _gpu_spectral(dims, sp, psi0, None, dt, N, Es, dtype, eigen=False, comps=4)
    t = dt * np.arange(N + 1)
    tol = 1e-10 if dtype == "c128" else 2e-4
    assert np.abs(chi - np.exp(-1j * E * t)).max() < tol
    assert abs(osp.peak(Es, spec) - E) < 1.0
