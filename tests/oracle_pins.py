"""Pins of the FP64 oracle to facts outside the oracle.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with
what the paper (Bauke & Keitel, arXiv:1012.3911) or the mathematics fixes:
brute-force DFTs and NumPy/SciPy library routines, closed-form solutions, the
Dirac algebra, invariants of the unitary, time-symmetric Strang step, and the
centre-of-mass velocity printed in Sec. 5.1.  The expected values are built
here from textbook formulas and library routines, never from the oracle's own
code.  ``test_oracle_pins.py`` runs them against the oracle and
``test_oracle_mutants.py`` re-runs them against copies of the oracle with
planted mistakes to show that each mistake is caught.
"""
from __future__ import annotations

import json
import os

import numpy as np
import scipy.linalg

from paper_1012_3911_gb300 import workloads as wl

C = 137.036
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# --------------------------------------------------------------------------
# FFT (Sec. 2.1: the continuous transform becomes a DFT on the lattice)
# --------------------------------------------------------------------------

FFT_SIZES = [1, 2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27, 48, 96]


def pin_fft_brute_force(orc):
    """Own radix-2/3 FFT == the DFT matrix written out, both signs."""
    rng = np.random.default_rng(7)
    for n in FFT_SIZES:
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        j = np.arange(n)
        for sign in (-1, +1):
            Fm = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
            ref = Fm @ x
            assert relerr(orc.fft(x, sign), ref) < 1e-13, (n, sign)
            assert relerr(orc.dft_naive(x, sign), ref) < 1e-13, (n, sign)


def pin_fft_library(orc):
    """Own FFT == numpy.fft on larger sizes, and known transforms."""
    rng = np.random.default_rng(8)
    for n in (64, 96, 128, 192, 384, 512, 768, 1024, 1536, 2048):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        assert relerr(orc.fft(x, -1), np.fft.fft(x)) < 1e-13, n
        assert relerr(orc.fft(x, +1), n * np.fft.ifft(x)) < 1e-13, n
    n = 48
    k0 = 5
    j = np.arange(n)
    plane = np.exp(2j * np.pi * k0 * j / n)
    X = orc.fft(plane, -1)
    expect = np.zeros(n, complex)
    expect[k0] = n
    assert np.abs(X - expect).max() < 1e-12       # forward sign: exp(-2 pi i jk/n)
    delta = np.zeros(n, complex)
    delta[0] = 1.0
    assert np.abs(orc.fft(delta) - 1.0).max() < 1e-15


def pin_fftn_library(orc):
    """Separable n-D transform == numpy.fft.fftn/ifftn; Parseval."""
    rng = np.random.default_rng(9)
    for shape in [(8,), (12, 8), (6, 16, 9), (24, 48), (3, 4, 2)]:
        x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        X = orc.fftn(x, -1)
        assert relerr(X, np.fft.fftn(x)) < 1e-13, shape
        assert relerr(orc.fftn(x, +1), np.fft.ifftn(x)) < 1e-13, shape
        assert relerr(orc.fftn(X, +1), x) < 1e-13, shape
        N = x.size
        assert abs(np.sum(np.abs(X) ** 2) / N - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)


# --------------------------------------------------------------------------
# Schroedinger (Sec. 2.2)
# --------------------------------------------------------------------------

def _free_exact(psi0, dims, spacing, t):
    """Free lattice evolution: psi~(t) = exp(-i |p|^2 t/2) psi~(0), p from
    numpy.fft.fftfreq (m = hbar = 1)."""
    P = np.meshgrid(*[wl.momenta(n, h) for n, h in zip(dims, spacing)][::-1], indexing="ij")
    p2 = sum(p * p for p in P)
    return np.fft.ifftn(np.exp(-0.5j * p2 * t) * np.fft.fftn(psi0))


def pin_free_schrodinger_exact(orc):
    """V = 0, no field: the split is exact, psi~(t) = exp(-i p^2 t/2) psi~(0),
    including the Nyquist column (random, unresolved state)."""
    for dims, sp in [((16,), (0.3,)), ((12, 8), (0.5, 0.25)), ((6, 8, 9), (0.4, 0.3, 0.7))]:
        shape = dims[::-1]
        psi0 = wl.random_state(shape, seed=11 + len(dims))
        dt, n = 0.037, 7
        out = orc.schrodinger_propagate(psi0, None, sp, dt, n)
        ref = _free_exact(psi0, dims, sp, dt * n)
        assert relerr(out, ref) < 1e-13, dims


def pin_free_gaussian_spreading(orc):
    """Continuum closed form of a free Gaussian, sigma^2 -> sigma^2 + i t
    (amplitude width, m = hbar = 1), while the packet stays inside the box:
    psi(x, t) = prod_a sqrt(s^2/z) exp(-(x_a - x0_a - p0_a t)^2/(2 z)
                                       + i p0_a x_a - i p0_a^2 t/2),  z = s^2 + i t."""
    dims, sp = (256, 256), (0.25, 0.25)
    x0, s, p0 = (-3.0, 2.0), 2.0, (1.5, -0.5)
    psi0 = wl.gaussian(dims, sp, x0, s, p0)
    t = 4.0
    out = orc.schrodinger_propagate(psi0, None, sp, 0.05, 80)
    X = wl.mesh(dims, sp)
    z = s * s + 1j * t

    def closed(tt, zz):
        g = np.ones(X[0].shape, complex)
        for a in range(2):
            g = g * np.sqrt(s * s / zz) * np.exp(-((X[a] - x0[a] - p0[a] * tt) ** 2) / (2 * zz)
                                                 + 1j * p0[a] * X[a] - 0.5j * p0[a] ** 2 * tt)
        return g

    g0 = closed(0.0, s * s + 0j)
    i = np.argmax(np.abs(psi0))
    scale = psi0.ravel()[i] / g0.ravel()[i]     # the normalisation workloads applied
    ref = scale * closed(t, z)
    assert relerr(out, ref) < 1e-9


def _coherent(x, t, omega, x0):
    """Harmonic-oscillator coherent state (m = hbar = 1, p0 = 0):
    (omega/pi)^{1/4} exp(-omega (x-xc)^2/2 + i pc x - i omega t/2 - i pc xc/2),
    xc = x0 cos(omega t), pc = -omega x0 sin(omega t)."""
    xc = x0 * np.cos(omega * t)
    pc = -omega * x0 * np.sin(omega * t)
    return (omega / np.pi) ** 0.25 * np.exp(-omega * (x - xc) ** 2 / 2 + 1j * pc * x
                                            - 0.5j * omega * t - 0.5j * pc * xc)


def pin_coherent_state_second_order(orc):
    """1D harmonic V = omega^2 x^2/2 with the coherent packet: error against
    the closed form at t = 100 is O(dt^2) (about 1.9e-4 at dt = 0.05 and a
    factor 4 smaller at dt/2), and the norm stays 1."""
    w = wl.config1()
    x = wl.lattice(w.dims[0], w.spacing[0])
    errs = []
    for dt, n in [(0.05, 2000), (0.025, 4000)]:
        out = orc.schrodinger_propagate(w.psi0, w.V, w.spacing, dt, n)
        errs.append(relerr(out, _coherent(x, dt * n, 0.1, -20.0)))
        assert abs(orc.norm(out, w.spacing) - 1.0) < 1e-12
    assert 1.0e-4 < errs[0] < 3.0e-4, errs
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


def pin_coherent_state_period(orc):
    """After one period 2 pi/omega the coherent state returns as -psi(0)
    (phase -i omega T/2 = -i pi), up to the O(dt^2) split error."""
    w = wl.config1()
    period = 2 * np.pi / 0.1
    n = 1256
    out = orc.schrodinger_propagate(w.psi0, w.V, w.spacing, period / n, n)
    assert relerr(out, -w.psi0) < 2.0e-4


def pin_schrodinger_norm_and_reversibility(orc):
    """Unitary: norm conserved to 1e-12.  Time-symmetric: n steps with dt then
    n steps with -dt and the field samples reversed return psi(0)."""
    dims, sp = (24, 16), (0.4, 0.5)
    shape = dims[::-1]
    psi0 = wl.random_state(shape, 21, sp)
    V = wl.random_potential(dims, 22, 2.0)
    F = wl.random_field(9, 2, 23, 0.3)
    out = orc.schrodinger_propagate(psi0, V, sp, 0.07, 9, F)
    assert abs(orc.norm(out, sp) - orc.norm(psi0, sp)) < 1e-12
    back = orc.schrodinger_propagate(out, V, sp, -0.07, 9, F[::-1].copy())
    assert relerr(back, psi0) < 1e-12


def pin_constant_potential_phase(orc):
    """A constant V0 only adds the global phase exp(-i V0 t)."""
    dims, sp = (32,), (0.3,)
    psi0 = wl.random_state((32,), 31)
    V0 = 0.73
    V = np.full((32,), V0)
    out = orc.schrodinger_propagate(psi0, V, sp, 0.05, 11)
    ref = np.exp(-1j * V0 * 0.55) * _free_exact(psi0, dims, sp, 0.55)
    assert relerr(out, ref) < 1e-13


def pin_shift_covariance(orc):
    """Shifting psi and V by one lattice cell commutes with the step (no field)."""
    dims, sp = (16, 12), (0.5, 0.5)
    psi0 = wl.random_state(dims[::-1], 41)
    V = wl.random_potential(dims, 42)
    a = orc.schrodinger_propagate(np.roll(psi0, 1, axis=1), np.roll(V, 1, axis=1), sp, 0.1, 5)
    b = np.roll(orc.schrodinger_propagate(psi0, V, sp, 0.1, 5), 1, axis=1)
    assert relerr(a, b) < 1e-13


def pin_field_kick_plane_wave(orc):
    """Length-gauge field on a lattice plane wave, V = 0.  With q = -1 the
    half-step factor exp(-i x E dt/2) is a lattice plane wave when
    E dt/2 = m 2 pi/L, so one step is known exactly:
    psi_j = exp(-i (p0 - E dt/2)^2 dt/2) exp(i (p0 - E dt) x_j), with x_j on
    [-L/2, L/2).  This fixes the field's sign, the half-step structure and the
    lattice origin."""
    n, h = 32, 0.25
    L = n * h
    dp = 2 * np.pi / L
    p0 = 5 * dp
    dt = 0.1
    E = 2 * dp / (dt / 2)               # kick of two lattice momenta per half step
    x = wl.lattice(n, h)
    psi0 = np.exp(1j * p0 * x)
    out = orc.schrodinger_propagate(psi0, None, (h,), dt, 1, np.array([[E]]))
    pm = p0 - E * dt / 2
    ref = np.exp(-0.5j * pm * pm * dt) * np.exp(1j * (p0 - E * dt) * x)
    assert np.abs(out - ref).max() < 1e-12


def pin_velocity_gauge_plane_waves(orc):
    """Velocity gauge (Eq. 13 with A), V = 0: the split is exact and each
    lattice plane wave only gains exp(-i sum_n tau |p - q A_n|^2 / (2 m)),
    so a random state evolves by that factor per momentum (NumPy FFT as the
    transform).  Fixes the sign of q A, the mass factor and the per-step A."""
    dims, sp = (16, 12), (0.3, 0.25)
    psi0 = wl.random_state(dims[::-1], 81)
    tau, n, m, q = 0.07, 5, 1.3, -1.0
    A = wl.random_field(n, 2, 82, 2.0)
    out = orc.schrodinger_propagate(psi0, None, sp, tau, n, A, mass=m, charge=q, gauge="velocity")
    px = wl.momenta(dims[0], sp[0])[None, :]
    py = wl.momenta(dims[1], sp[1])[:, None]
    ph = np.zeros(dims[::-1])
    for k in range(n):
        ph += tau * ((px - q * A[k, 0]) ** 2 + (py - q * A[k, 1]) ** 2) / (2 * m)
    ref = np.fft.ifft2(np.exp(-1j * ph) * np.fft.fft2(psi0))
    assert relerr(out, ref) < 1e-12


def pin_velocity_gauge_lattice_shift(orc):
    """A constant A with q A a lattice momentum (2 pi m_a / L_a): the
    velocity-gauge Hamiltonian is G H_0 G^dag with G = exp(i q A.x / hbar),
    and the lattice split steps are conjugate in the same way, so with a
    potential psi_vel(t) = G U_0(t) G^dag psi_vel(0), up to the weight that
    reaches the Nyquist momenta, where the lattice shift wraps: a Gaussian
    well and packet keep it near 1e-11 on this lattice (the wrong sign of G
    is off by order one)."""
    dims, sp = (48, 32), (0.3, 0.4)
    L = np.array(dims) * np.array(sp)
    q = -1.0
    A = (2 * np.pi * np.array([2.0, -1.0]) / L) / q
    X = wl.mesh(dims, sp)
    G = np.exp(1j * q * (A[0] * X[0] + A[1] * X[1]))
    V = -2.0 * np.exp(-(X[0] ** 2 + X[1] ** 2) / (2 * 1.5 ** 2))
    psi0 = wl.gaussian(dims, sp, (0.5, -0.4), 1.0)
    tau, n = 0.05, 12
    vel = orc.schrodinger_propagate(psi0, V, sp, tau, n, np.tile(A, (n, 1)), gauge="velocity")
    ref = G * orc.schrodinger_propagate(np.conj(G) * psi0, V, sp, tau, n, None)
    assert relerr(vel, ref) < 1e-10
    # A = 0 in the velocity gauge is the field-free step, bit for bit
    zero = orc.schrodinger_propagate(psi0, V, sp, tau, n, np.zeros((n, 2)), gauge="velocity")
    assert np.array_equal(zero, orc.schrodinger_propagate(psi0, V, sp, tau, n, None))


def pin_ehrenfest_field(orc):
    """V = 0 with a uniform field: <p> changes by q sum_n E_n dt (force qE),
    for a packet far from the box edge."""
    dims, sp = (256,), (0.2,)
    psi0 = wl.gaussian(dims, sp, (0.0,), 2.0, (0.7,))
    F = wl.random_field(20, 1, 51, 0.05)
    dt = 0.05
    out = orc.schrodinger_propagate(psi0, None, sp, dt, 20, F)
    p = wl.momenta(256, 0.2)
    pk = lambda s: np.sum(p * np.abs(np.fft.fft(s)) ** 2) / np.sum(np.abs(np.fft.fft(s)) ** 2)
    expect = pk(psi0) + (-1.0) * F[:, 0].sum() * dt
    assert abs(pk(out) - expect) < 1e-8


def pin_schrodinger_energy(orc):
    """Energy functional: plane wave -> p0^2/2 + V0; Gaussian ->
    p0^2/2 + d/(4 sigma^2); harmonic ground state -> omega/2; norm of the
    normalised Gaussian -> 1."""
    n, h = 64, 0.25
    L = n * h
    p0 = 3 * 2 * np.pi / L
    x = wl.lattice(n, h)
    pw = np.exp(1j * p0 * x) / np.sqrt(L)
    assert abs(orc.norm(pw, (h,)) - 1.0) < 1e-13
    assert abs(orc.energy(pw, np.full(n, 0.4), (h,)) - (0.5 * p0 * p0 + 0.4)) < 1e-12
    dims, sp = (256, 256), (0.1, 0.1)
    g = wl.gaussian(dims, sp, (0.5, -0.2), 1.5, (0.8, 0.3))
    assert abs(orc.norm(g, sp) - 1.0) < 1e-12
    e = orc.energy(g, None, sp)
    assert abs(e - (0.5 * (0.8 ** 2 + 0.3 ** 2) + 2 / (4 * 1.5 ** 2))) < 1e-9
    w = 0.5
    dims1, sp1 = (256,), (0.1,)
    gs = wl.gaussian(dims1, sp1, (0.0,), np.sqrt(1 / w))
    assert abs(orc.energy(gs, wl.harmonic(dims1, sp1, w), sp1) - w / 2) < 1e-9


# --------------------------------------------------------------------------
# Dirac (Sec. 2.3)
# --------------------------------------------------------------------------

_SX = np.array([[0, 1], [1, 0]], complex)
_SY = np.array([[0, -1j], [1j, 0]], complex)
_SZ = np.array([[1, 0], [0, -1]], complex)
_I2 = np.eye(2)
_Z2 = np.zeros((2, 2))


def textbook_dirac():
    """alpha_i = [[0, sigma_i], [sigma_i, 0]], beta = diag(1, 1, -1, -1)."""
    al = [np.block([[_Z2, s], [s, _Z2]]) for s in (_SX, _SY, _SZ)]
    be = np.block([[_I2, _Z2], [_Z2, -_I2]])
    return al, be


def textbook_h(p, mass=1.0, c=C):
    al, be = textbook_dirac()
    return sum(c * pi * al[i] for i, pi in enumerate(p)) + mass * c * c * be


def pin_dirac_algebra(orc):
    """alpha_i^2 = beta^2 = 1, {alpha_i, alpha_k} = 2 delta_ik,
    {alpha_i, beta} = 0 (Eq. 15); the matrices are the Dirac representation
    with Pauli blocks (Eq. 16)."""
    a1, a2, a3, b = orc.alpha_beta()
    al = [a1, a2, a3]
    I4 = np.eye(4)
    for i in range(3):
        assert np.allclose(al[i] @ al[i], I4, atol=0)
        assert np.allclose(al[i] @ b + b @ al[i], 0, atol=0)
        for k in range(3):
            if k != i:
                assert np.allclose(al[i] @ al[k] + al[k] @ al[i], 0, atol=0)
    assert np.allclose(b @ b, I4, atol=0)
    tal, tbe = textbook_dirac()
    for i in range(3):
        assert np.array_equal(al[i], tal[i]), i
    assert np.array_equal(b, tbe)


def pin_dirac_u_diagonalises(orc):
    """u(p) (Eqs. 29-30) is unitary and u H u^dagger = diag(E, E, -E, -E)
    (Eqs. 31-32), in 2D and 3D, with H the textbook free Hamiltonian."""
    for p in [(0.0, 0.0), (30.0, -12.0), (400.0, 250.0), (1e-3, 0.0), (10.0, 20.0, -5.0)]:
        u = orc.dirac_u(p)
        H = textbook_h(p)
        assert np.allclose(orc.dirac_h(p), H, rtol=0, atol=1e-9)
        assert np.abs(u @ u.conj().T - np.eye(4)).max() < 1e-14
        E = np.sqrt(C ** 4 + np.dot(p, p) * C * C)
        D = u @ H @ u.conj().T
        assert np.abs(D - np.diag([E, E, -E, -E])).max() < 1e-10 * E, p


def pin_dirac_kinetic_expm(orc):
    """Eq. 33 equals exp(-i tau (c alpha.p + m c^2 beta)) of Eq. 27
    (scipy.linalg.expm of the textbook Hamiltonian)."""
    for p, tau in [((3.0, -4.0), 1e-3), ((120.0, 45.0), 1e-4), ((0.0, 0.0), 2e-4),
                   ((7.0, 1.0, -2.0), 3e-4)]:
        M = orc.dirac_kinetic_matrix(p, tau)
        ref = scipy.linalg.expm(-1j * tau * textbook_h(p))
        assert np.abs(M - ref).max() < 1e-11, p


def pin_dirac_mixing_expm(orc):
    """Eq. 26 (via the exp-alpha identity, Eq. 23) equals
    exp(i delta q c alpha.Abar) with Abar = A tau and q = -1."""
    al, be = textbook_dirac()
    for A, tau, delta in [((20.0, 0.0), 1e-4, 0.5), ((3.0, -7.0), 2e-3, 0.5), ((0.0, 0.0), 1e-3, 0.5),
                          ((1.0, 2.0, 3.0), 1e-3, 1.0)]:
        R = orc.dirac_mixing_matrix(A, tau, delta)
        G = sum(A[i] * tau * al[i] for i in range(len(A)))
        ref = scipy.linalg.expm(1j * delta * (-1.0) * C * G)
        assert np.abs(R - ref).max() < 1e-13, A


def _free_dirac_exact(psi0, dims, sp, t):
    """Per momentum psi~(t) = [cos(E t) - i sin(E t) H/E] psi~(0) with the
    textbook H (H^2 = E^2)."""
    P = np.meshgrid(*[wl.momenta(m, h) for m, h in zip(dims, sp)][::-1], indexing="ij")[::-1]
    st = np.stack([np.fft.fft2(psi0[k]) for k in range(4)])
    res = np.empty_like(st)
    for iy in range(dims[1]):
        for ix in range(dims[0]):
            p = (P[0][iy, ix], P[1][iy, ix])
            H = textbook_h(p)
            E = np.sqrt(C ** 4 + (p[0] ** 2 + p[1] ** 2) * C * C)
            U = np.cos(E * t) * np.eye(4) - 1j * np.sin(E * t) * H / E
            res[:, iy, ix] = U @ st[:, iy, ix]
    return np.stack([np.fft.ifft2(res[k]) for k in range(4)])


def pin_free_dirac_exact(orc):
    """V = 0, A = 0: per momentum psi~(t) = [cos(E t) - i sin(E t) H/E] psi~(0),
    including the Nyquist rows (random, unresolved spinor)."""
    dims, sp = (16, 12), (0.05, 0.08)
    psi0 = wl.random_state((4,) + dims[::-1], 61)
    tau, n = 2e-4, 5
    out = orc.dirac_propagate(psi0, None, sp, tau, n)
    assert relerr(out, _free_dirac_exact(psi0, dims, sp, tau * n)) < 1e-12


def _per_momentum_3d(psi0, dims, sp, fn):
    """Apply the 4x4 matrix fn(p) to every momentum of a 3D spinor (NumPy FFT)."""
    st = np.stack([np.fft.fftn(psi0[k]) for k in range(4)])
    P = np.meshgrid(*[wl.momenta(m, h) for m, h in zip(dims, sp)][::-1], indexing="ij")[::-1]
    for idx in np.ndindex(*st.shape[1:]):
        p = np.array([P[0][idx], P[1][idx], P[2][idx]])
        st[(slice(None),) + idx] = fn(p) @ st[(slice(None),) + idx]
    return np.stack([np.fft.ifftn(st[k]) for k in range(4)])


def pin_free_dirac_exact_3d(orc):
    """3D, V = 0, A = 0: per momentum psi~(t) = expm(-i t H(p)) psi~(0) with the
    textbook H including alpha_3 (scipy expm), random spinor."""
    dims, sp = (8, 12, 8), (0.06, 0.05, 0.07)
    psi0 = wl.random_state((4,) + dims[::-1], 63)
    tau, n = 1.5e-4, 4
    out = orc.dirac_propagate(psi0, None, sp, tau, n)
    ref = _per_momentum_3d(psi0, dims, sp, lambda p: scipy.linalg.expm(-1j * tau * n * textbook_h(p)))
    assert relerr(out, ref) < 1e-12


def pin_dirac_uniform_A_second_order_3d(orc):
    """3D, constant A with all three components, V = 0: the split converges
    at second order to expm(-i t H(p - qA)) (q = -1)."""
    c = 10.0
    dims, sp = (8, 8, 12), (0.4, 0.4, 0.3)
    psi0 = wl.random_smooth_state(dims, sp, 64, comps=4)
    A = np.array([0.7, -0.5, 0.4])
    t = 0.15
    ref = _per_momentum_3d(psi0, dims, sp, lambda p: scipy.linalg.expm(-1j * t * textbook_h(p + A, 1.0, c)))
    errs = []
    for n in (16, 32):
        out = orc.dirac_propagate(psi0, None, sp, t / n, n, np.tile(A, (n, 1)), c=c)
        errs.append(relerr(out, ref))
    assert errs[0] < 5e-2, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def pin_dirac_energy_3d(orc):
    """<H> of a 3D spinor against (dV/N) sum_k psi~^dag H(p) psi~ + dV sum V |psi|^2."""
    dims, sp = (8, 12, 8), (0.1, 0.08, 0.12)
    psi = wl.random_state((4,) + dims[::-1], 65, sp)
    V = wl.random_potential(dims, 66, 2.0)
    st = np.stack([np.fft.fftn(psi[k]) for k in range(4)])
    P = np.meshgrid(*[wl.momenta(m, h) for m, h in zip(dims, sp)][::-1], indexing="ij")[::-1]
    t = 0.0
    for idx in np.ndindex(*st.shape[1:]):
        v = st[(slice(None),) + idx]
        t += np.vdot(v, textbook_h((P[0][idx], P[1][idx], P[2][idx])) @ v).real
    dV = float(np.prod(sp))
    N = int(np.prod(dims))
    ref = dV / N * t + dV * np.sum(V * np.sum(np.abs(psi) ** 2, axis=0))
    assert abs(orc.energy(psi, V, sp, 4) - ref) < 1e-10 * abs(ref)


def pin_dirac_profile_uniform(orc):
    """A vector potential that is the same in every column reproduces the
    uniform-A step exactly."""
    dims, sp = (12, 8), (0.05, 0.07)
    psi0 = wl.random_state((4,) + dims[::-1], 111, sp)
    V = wl.random_potential(dims, 112, 4.0)
    A = wl.random_field(3, 2, 113, 30.0)
    prof = np.repeat(A[:, None, :], dims[0], axis=1)
    out = orc.dirac_propagate_profile(psi0, V, sp, 1e-4, 3, prof)
    assert np.array_equal(out, orc.dirac_propagate(psi0, V, sp, 1e-4, 3, A))


def pin_dirac_profile_shift(orc):
    """Shifting the state, the potential and the profile A(x_1) by m columns
    shifts the result (translation covariance of the lattice step)."""
    dims, sp = (16, 8), (0.05, 0.06)
    psi0 = wl.random_state((4,) + dims[::-1], 114, sp)
    V = wl.random_potential(dims, 115, 4.0)
    prof = 40.0 * np.random.default_rng(116).standard_normal((3, dims[0], 2))
    m = 5
    out = orc.dirac_propagate_profile(psi0, V, sp, 1e-4, 3, prof)
    sh = orc.dirac_propagate_profile(np.roll(psi0, m, axis=-1), np.roll(V, m, axis=-1), sp, 1e-4, 3,
                                     np.roll(prof, m, axis=1))
    assert relerr(sh, np.roll(out, m, axis=-1)) < 1e-12


def pin_dirac_profile_two_steps_numpy(orc):
    """Two steps assembled in NumPy from the pinned pieces: the mixing of
    Eq. 26 per column (checked against expm), the kinetic matrix of Eq. 33
    per momentum (checked against expm), NumPy FFTs; fixes the column and
    step indexing of the profile."""
    dims, sp = (12, 8), (0.04, 0.05)
    psi = wl.random_state((4,) + dims[::-1], 117, sp)
    V = wl.random_potential(dims, 118, 3.0)
    prof = 30.0 * np.random.default_rng(119).standard_normal((2, dims[0], 2))
    tau = 1e-4
    P = np.meshgrid(*[wl.momenta(m, h) for m, h in zip(dims, sp)][::-1], indexing="ij")[::-1]
    K = {idx: orc.dirac_kinetic_matrix((P[0][idx], P[1][idx]), tau) for idx in np.ndindex(dims[1], dims[0])}
    ph = np.exp(-0.5j * tau * V)
    ref = psi.copy()
    for n in range(2):
        R = [orc.dirac_mixing_matrix(prof[n, i], tau, 0.5) for i in range(dims[0])]
        for half in range(2):
            for iy, ix in np.ndindex(dims[1], dims[0]):
                ref[:, iy, ix] = ph[iy, ix] * (R[ix] @ ref[:, iy, ix])
            if half == 1:
                break
            st = np.stack([np.fft.fft2(ref[k]) for k in range(4)])
            for idx in np.ndindex(dims[1], dims[0]):
                st[(slice(None),) + idx] = K[idx] @ st[(slice(None),) + idx]
            ref = np.stack([np.fft.ifft2(st[k]) for k in range(4)])
    out = orc.dirac_propagate_profile(psi, V, sp, tau, 2, prof)
    assert relerr(out, ref) < 1e-12


def pin_dirac_constant_potential_phase(orc):
    """A constant V0 with A = 0 only adds the global phase exp(-i V0 t) to the
    free Dirac evolution (Eqs. 21-22: the scalar factor commutes)."""
    dims, sp = (8, 12), (0.05, 0.08)
    psi0 = wl.random_state((4,) + dims[::-1], 62)
    V0, tau, n = 1234.5, 1e-4, 7
    out = orc.dirac_propagate(psi0, np.full(dims[::-1], V0), sp, tau, n)
    ref = np.exp(-1j * V0 * tau * n) * _free_dirac_exact(psi0, dims, sp, tau * n)
    assert relerr(out, ref) < 1e-12


def pin_dirac_norm_and_reversibility(orc):
    dims, sp = (16, 24), (0.05, 0.04)
    psi0 = wl.random_state((4,) + dims[::-1], 71, sp)
    V = wl.random_potential(dims, 72, 3.0)
    F = wl.random_field(6, 2, 73, 30.0)
    out = orc.dirac_propagate(psi0, V, sp, 1e-4, 6, F)
    assert abs(orc.norm(out, sp, 4) - orc.norm(psi0, sp, 4)) < 1e-12
    back = orc.dirac_propagate(out, V, sp, -1e-4, 6, F[::-1].copy())
    assert relerr(back, psi0) < 1e-12


def pin_dirac_uniform_A_second_order(orc):
    """Constant uniform A, V = 0: the exact evolution is
    exp(-i H(p - qA) t) per momentum (q = -1).  The split converges to it at
    second order (error ratio about 4 when dt halves)."""
    c = 10.0
    dims, sp = (16, 16), (0.3, 0.3)
    psi0 = wl.random_smooth_state(dims, sp, 81, comps=4)
    A = np.array([0.9, -0.4])
    t = 0.2
    P = np.meshgrid(*[wl.momenta(m, h) for m, h in zip(dims, sp)][::-1], indexing="ij")[::-1]
    st = np.stack([np.fft.fft2(psi0[k]) for k in range(4)])
    res = np.empty_like(st)
    for iy in range(dims[1]):
        for ix in range(dims[0]):
            p = np.array([P[0][iy, ix], P[1][iy, ix]]) + A     # p - qA with q = -1
            res[:, iy, ix] = scipy.linalg.expm(-1j * t * textbook_h(p, 1.0, c)) @ st[:, iy, ix]
    ref = np.stack([np.fft.ifft2(res[k]) for k in range(4)])
    errs = []
    for n in (20, 40):
        F = np.tile(A, (n, 1))
        out = orc.dirac_propagate(psi0, None, sp, t / n, n, F, c=c)
        errs.append(relerr(out, ref))
    assert errs[0] < 5e-2, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


SX = np.array([[0, 1], [1, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def _h1(p, m=1.0, c=C):
    """1D Dirac Hamiltonian c sigma_x p + m c^2 sigma_z, written here."""
    return c * p * SX + m * c * c * SZ


def pin_dirac1d_u_diagonalises(orc):
    """The 2x2 u(p) is unitary and u H u^dag = diag(E, -E) (the 1D form of
    Eqs. 29-32), including p = 0, both signs and |p| >> mc."""
    for p in (0.0, 0.7, -3.1, 250.0, -1.0e4):
        u = orc.dirac1d_u(p)
        H = orc.dirac1d_h(p)
        assert np.abs(H - _h1(p)).max() < 1e-9 * max(1.0, abs(p) * C)
        E = np.sqrt(C ** 4 + p * p * C * C)
        assert np.abs(u @ u.conj().T - np.eye(2)).max() < 1e-14
        assert np.abs(u @ _h1(p) @ u.conj().T - np.diag([E, -E])).max() < 1e-10 * E


def pin_dirac1d_free_exact(orc):
    """V = 0, A = 0: per momentum psi~(t) = expm(-i H(p) t) psi~(0) (scipy),
    for a random two-component spinor including the Nyquist index."""
    n, h = 24, 0.02
    psi0 = wl.random_state((2, n), 91)
    tau, steps = 3e-4, 6
    out = orc.dirac1d_propagate(psi0, None, (h,), tau, steps)
    st = np.fft.fft(psi0, axis=1)
    for k, p in enumerate(wl.momenta(n, h)):
        st[:, k] = scipy.linalg.expm(-1j * tau * steps * _h1(p)) @ st[:, k]
    assert relerr(out, np.fft.ifft(st, axis=1)) < 1e-12


def pin_dirac1d_constant_potential_phase(orc):
    n, h = 32, 0.05
    psi0 = wl.random_state((2, n), 92)
    V0, tau, steps = 321.5, 2e-4, 5
    out = orc.dirac1d_propagate(psi0, np.full(n, V0), (h,), tau, steps)
    ref = np.exp(-1j * V0 * tau * steps) * orc.dirac1d_propagate(psi0, None, (h,), tau, steps)
    assert relerr(out, ref) < 1e-12


def pin_dirac1d_norm_and_reversibility(orc):
    n, h = 48, 0.04
    psi0 = wl.random_state((2, n), 93, (h,))
    V = wl.random_potential((n,), 94, 5.0)
    A = wl.random_field(7, 1, 95, 40.0)[:, 0]
    out = orc.dirac1d_propagate(psi0, V, (h,), 1e-4, 7, A)
    assert abs(orc.norm(out, (h,), 2) - orc.norm(psi0, (h,), 2)) < 1e-12
    back = orc.dirac1d_propagate(out, V, (h,), -1e-4, 7, A[::-1].copy())
    assert relerr(back, psi0) < 1e-12


def pin_dirac1d_equals_2d_pair(orc):
    """The two-component 1D equation is the (1,4) component pair of the
    four-component 2D code on a state constant along y (p_y = 0), with the
    same V(x) and A = (A_x, 0): two independent oracle paths (4x4 u(p) of
    Eq. 30 and the mixing of Eq. 26 against their 2x2 forms)."""
    nx, ny, h = 32, 8, (0.05, 0.1)
    psi1 = wl.random_state((2, nx), 96, (h[0],))
    V = wl.random_potential((nx,), 97, 20.0)
    A = wl.random_field(5, 1, 98, 60.0)[:, 0]
    tau = 2e-4
    one = orc.dirac1d_propagate(psi1, V, (h[0],), tau, 5, A)
    psi2 = np.zeros((4, ny, nx), dtype=complex)
    psi2[0] = psi1[0][None, :]
    psi2[3] = psi1[1][None, :]
    F = np.stack([A, np.zeros_like(A)], axis=1)
    two = orc.dirac_propagate(psi2, np.tile(V, (ny, 1)), h, tau, 5, F)
    assert np.abs(two[1]).max() < 1e-13 and np.abs(two[2]).max() < 1e-13
    assert relerr(two[0][0], one[0]) < 1e-12 and relerr(two[3][3], one[1]) < 1e-12


def pin_dirac1d_uniform_A_second_order(orc):
    """Constant A, V = 0: exact evolution expm(-i H(p - qA) t) per momentum
    (q = -1); the split converges at second order."""
    c = 10.0
    n, h = 32, 0.3
    psi0 = wl.random_smooth_state((n,), (h,), 99, comps=2)
    A, t = 0.8, 0.2
    st = np.fft.fft(psi0, axis=1)
    for k, p in enumerate(wl.momenta(n, h)):
        st[:, k] = scipy.linalg.expm(-1j * t * _h1(p + A, 1.0, c)) @ st[:, k]
    ref = np.fft.ifft(st, axis=1)
    errs = [relerr(orc.dirac1d_propagate(psi0, None, (h,), t / m, m, np.full(m, A), c=c), ref) for m in (20, 40)]
    assert errs[0] < 5e-2, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def pin_dirac1d_energy(orc):
    """<H> of a 1D spinor: (dV/N) sum_k psi~^dag H(p) psi~ + dV sum V |psi|^2,
    written here with NumPy's FFT."""
    n, h = 64, 0.05
    psi = wl.random_state((2, n), 100, (h,))
    V = wl.random_potential((n,), 101, 3.0)
    st = np.fft.fft(psi, axis=1)
    t = sum(np.vdot(st[:, k], _h1(p) @ st[:, k]).real for k, p in enumerate(wl.momenta(n, h)))
    ref = h / n * t + h * np.sum(V * np.sum(np.abs(psi) ** 2, axis=0))
    assert abs(orc.energy(psi, V, (h,), 2) - ref) < 1e-10 * abs(ref)


def pin_dirac_velocity(orc):
    """Sec. 5.1: a positive-energy packet with mean momentum (40, 0) moves
    at |p|/(m sqrt(1 + p^2/(mc)^2)) = 38.398 a.u."""
    dims, sp = (512, 32), (1.0 / 32, 0.5)
    scal = wl.gaussian(dims, sp, (-4.0, 0.0), 1.0, (40.0, 0.0))
    psi0 = wl.dirac_positive_spin_up(scal, dims, sp)
    t, n = 0.05, 10
    out = orc.dirac_propagate(psi0, None, sp, t / n, n)
    X = wl.mesh(dims, sp)
    dV = sp[0] * sp[1]
    mean_x = lambda s: dV * np.sum(X[0] * np.sum(np.abs(s) ** 2, axis=0))
    v = (mean_x(out) - mean_x(psi0)) / t
    assert abs(v - 40.0 / np.sqrt(1 + (40.0 / C) ** 2)) < 0.05, v
    gold = json.load(open(os.path.join(GOLDEN, "sec5_1_free_dirac_packet.json")))
    assert abs(v - gold["printed_velocity_au"]) < gold["printed_precision_au"], v


def pin_dirac_energy(orc):
    """Energy of a lattice plane-wave spinor with the textbook positive- or
    negative-energy eigenvector is +-E(p) (+ V0)."""
    dims, sp = (16, 8), (0.1, 0.2)
    L = [n * h for n, h in zip(dims, sp)]
    p = (3 * 2 * np.pi / L[0], -1 * 2 * np.pi / L[1])
    H = textbook_h(p)
    w, vecs = np.linalg.eigh(H)
    X = wl.mesh(dims, sp)
    phase = np.exp(1j * (p[0] * X[0] + p[1] * X[1]))
    vol = L[0] * L[1]
    for idx in (0, 3):
        psi = np.stack([vecs[k, idx] * phase for k in range(4)]) / np.sqrt(vol)
        assert abs(orc.norm(psi, sp, 4) - 1.0) < 1e-13
        e = orc.energy(psi, np.full(dims[::-1], -0.3), sp, comps=4)
        assert abs(e - (w[idx] - 0.3)) < 1e-9 * abs(w[idx]), (e, w[idx])


ALL_PINS = [
    pin_fft_brute_force, pin_fft_library, pin_fftn_library,
    pin_free_schrodinger_exact, pin_free_gaussian_spreading, pin_coherent_state_second_order,
    pin_coherent_state_period, pin_schrodinger_norm_and_reversibility, pin_constant_potential_phase,
    pin_shift_covariance, pin_field_kick_plane_wave, pin_velocity_gauge_plane_waves,
    pin_velocity_gauge_lattice_shift, pin_dirac1d_u_diagonalises, pin_dirac1d_free_exact,
    pin_dirac1d_constant_potential_phase, pin_dirac1d_norm_and_reversibility, pin_dirac1d_equals_2d_pair,
    pin_dirac1d_uniform_A_second_order, pin_dirac1d_energy, pin_free_dirac_exact_3d,
    pin_dirac_uniform_A_second_order_3d, pin_dirac_energy_3d, pin_dirac_profile_uniform,
    pin_dirac_profile_shift, pin_dirac_profile_two_steps_numpy, pin_ehrenfest_field, pin_schrodinger_energy,
    pin_dirac_algebra, pin_dirac_u_diagonalises, pin_dirac_kinetic_expm, pin_dirac_mixing_expm,
    pin_free_dirac_exact, pin_dirac_constant_potential_phase, pin_dirac_norm_and_reversibility, pin_dirac_uniform_A_second_order,
    pin_dirac_velocity, pin_dirac_energy,
]
