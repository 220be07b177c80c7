"""The oracle's spectral method (autocorrelation, windowed spectrum,
eigenfunctions) against closed forms and direct diagonalisation (CPU)."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse.linalg as ssl

from oracle import spectral as osp
from paper_1012_3911_gb300 import workloads as wl


def _lattice_h1(n, L, V, mass=1.0):
    """The periodic lattice Hamiltonian p^2/2m (spectral, as the split step's
    kinetic factor) + V, dense, 1D."""
    h = L / n
    k = 2 * np.pi * np.fft.fftfreq(n, d=h)
    F = np.fft.fft(np.eye(n), axis=0)
    T = np.real(np.conj(F).T @ np.diag(k ** 2 / (2 * mass)) @ F) / n
    return T + np.diag(V)


def test_plane_wave_autocorrelation_is_exact():
    n, L, dt, N = 64, 20.0, 0.05, 40
    x = wl.lattice(n, L / n)
    k = 2 * np.pi * 3 / L
    psi0 = np.exp(1j * k * x) / np.sqrt(L)
    chi, spec, _ = osp.spectral(psi0, np.zeros(n), (L / n,), dt, N, [0.0])
    t = dt * np.arange(N + 1)
    assert np.abs(chi - np.exp(-0.5j * k * k * t)).max() < 1e-12


def test_eigenfunction_of_an_exact_eigenstate_is_absolute():
    """A lattice plane wave is an exact eigenvector of the free split step,
    psi_n = exp(-i E0 t_n) psi_0 with E0 = k^2/2, so the accumulated
    eigenfunction has a closed form that fixes its dt factor, window weights
    and phase sign (not only its direction):
      Psi_{E0}            = dt sum_n w_n psi_0 = N dt psi_0 = T psi_0,
      Psi_{E0 + 2 pi / T} = -T/2 psi_0,
      Psi_{E0 + 4 pi / T} = 0,
    since sum_{n=0}^{N} (1 - cos(2 pi n/N)) exp(2 pi i m n/N) = N, -N/2, 0 for
    m = 0, 1, 2 (N > 4)."""
    n, L, dt, N = 64, 20.0, 0.05, 40
    T = N * dt
    x = wl.lattice(n, L / n)
    k = 2 * np.pi * 3 / L
    psi0 = np.exp(1j * k * x) / np.sqrt(L)
    E0 = 0.5 * k * k
    Es = [E0, E0 + 2 * np.pi / T, E0 + 4 * np.pi / T]
    _, _, psiE = osp.spectral(psi0, np.zeros(n), (L / n,), dt, N, Es)
    scale = T * np.abs(psi0).max()
    assert np.abs(psiE[0] - T * psi0).max() < 1e-12 * scale
    assert np.abs(psiE[1] + 0.5 * T * psi0).max() < 1e-12 * scale
    assert np.abs(psiE[2]).max() < 1e-12 * scale


def test_harmonic_levels():
    """V = w^2 x^2 / 2: peaks at w (k + 1/2)."""
    n, L, w, dt, N = 128, 40.0, 0.5, 0.05, 3000
    x = wl.lattice(n, L / n)
    psi0 = wl.gaussian((n,), (L / n,), (1.5,), 1.0 / np.sqrt(w))
    Es = np.linspace(0.0, 1.6, 801)
    _, spec, _ = osp.spectral(psi0, 0.5 * w * w * x * x, (L / n,), dt, N, Es)
    for lev in range(3):
        sel = np.abs(Es - w * (lev + 0.5)) < 0.1
        e = osp.peak(Es[sel], spec[sel])
        assert abs(e - w * (lev + 0.5)) < 2e-3, (lev, e)


def test_soft_core_1d_ground_state_and_eigenfunction():
    """zeta = 1.4133: the ground state of the 1D soft core sits at about
    -Z^2/2 (the eigenstates subsection); peak and eigenfunction against the
    lattice Hamiltonian's own ground state."""
    n, L, dt, N = 256, 60.0, 0.05, 2000
    x = wl.lattice(n, L / n)
    V = -1.0 / np.sqrt(x * x + 1.4133 ** 2)
    evals, evecs = sl.eigh(_lattice_h1(n, L, V))
    assert abs(evals[0] + 0.5) < 1e-3
    psi0 = wl.gaussian((n,), (L / n,), (0.7,), 1.5)
    Es = np.linspace(-0.6, -0.4, 401)
    _, spec, _ = osp.spectral(psi0, V, (L / n,), dt, N, Es)
    e0 = osp.peak(Es, spec)
    assert abs(e0 - evals[0]) < 1e-3
    _, _, psiE = osp.spectral(psi0, V, (L / n,), dt, N, [evals[0]])
    v = psiE[0] / np.linalg.norm(psiE[0])
    assert abs(np.vdot(evecs[:, 0], v)) > 0.999


def test_soft_core_2d_ground_state():
    """zeta = 0.791 in 2D: ground state about -Z^2/2; the spectral peak
    against the lattice Hamiltonian's lowest eigenvalue (sparse solver)."""
    n, L, dt, N = 64, 24.0, 0.05, 1000
    h = L / n
    X = wl.mesh((n, n), (h, h))
    V = -1.0 / np.sqrt(X[0] ** 2 + X[1] ** 2 + 0.791 ** 2)
    k = 2 * np.pi * np.fft.fftfreq(n, d=h)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    T = 0.5 * (KX ** 2 + KY ** 2)

    def mv(u):
        u = u.reshape(n, n)
        return (np.fft.ifft2(T * np.fft.fft2(u)) + V * u).ravel()
    e_ref = ssl.eigsh(ssl.LinearOperator((n * n, n * n), matvec=mv, dtype=complex), k=1, which="SA",
                      tol=1e-10)[0][0]
    assert abs(e_ref + 0.5) < 6e-3
    psi0 = wl.gaussian((n, n), (h, h), (0.5, -0.3), 1.2)
    Es = np.linspace(-0.6, -0.4, 201)
    _, spec, _ = osp.spectral(psi0, V, (h, h), dt, N, Es)
    assert abs(osp.peak(Es, spec) - e_ref) < 2e-3


def test_window_and_unitarity():
    n, L, dt, N = 64, 20.0, 0.05, 30
    x = wl.lattice(n, L / n)
    psi0 = wl.gaussian((n,), (L / n,), (0.5,), 1.0)
    chi, spec, psiE = osp.spectral(psi0, 0.1 * x * x, (L / n,), dt, N, [0.3, -0.2])
    assert chi[0] == pytest.approx(1.0, abs=1e-12)
    assert np.abs(chi).max() <= 1.0 + 1e-12
    # the window removes both ends: dropping them changes nothing
    t = dt * np.arange(N + 1)
    win = 1 - np.cos(2 * np.pi * t / (N * dt))
    assert abs(win[0]) < 1e-15 and abs(win[-1]) < 1e-12
    ref = dt * np.sum((chi * win * np.exp(1j * t * 0.3))[1:-1])
    assert abs(spec[0] - ref) < 1e-12


def test_dirac_plane_wave_spectrum():
    """Spinor form: a positive-energy 1D Dirac plane wave has chi_n =
    exp(-i E t_n) exactly and the spectrum peaks at E (the window is symmetric
    about it on a grid centred there)."""
    import oracle
    oracle.build()
    n, h, c = 64, 0.02, 137.036
    p0 = 2 * np.pi * 3 / (n * h)
    E = np.sqrt(c ** 4 + c * c * p0 * p0)
    v = np.conj(oracle.dirac1d_u(p0)[0])
    x = wl.lattice(n, h)
    psi0 = np.stack([vk * np.exp(1j * p0 * x) for vk in v]) / np.sqrt(n * h)
    dt, N = 2e-4, 60
    Es = E + np.linspace(-400.0, 400.0, 81)
    chi, spec, _ = osp.spectral(psi0, None, (h,), dt, N, Es,
                                propagate=lambda s, t: oracle.dirac1d_propagate(s, None, (h,), t, 1))
    assert np.abs(chi - np.exp(-1j * E * dt * np.arange(N + 1))).max() < 1e-11
    assert abs(osp.peak(Es, spec) - E) < 1e-6 * E
