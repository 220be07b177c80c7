"""Seeded synthetic inputs for the Fourier split-operator step.

This module only builds inputs (lattices, potentials, initial wave functions,
laser-field samples).  It holds none of the split-step arithmetic, so both the
CUDA path and the FP64 oracle can consume its arrays without sharing code.

Workloads follow the paper's applications (Bauke & Keitel, arXiv:1012.3911,
Secs. 4.2 and 5): Gaussian packets, soft-core Coulomb potentials (Eq. 44 with
the soft-core parameter given directly as a^2), sin^2-enveloped laser pulses
in the dipole approximation, and a positive-energy spin-up Dirac packet built
from plane waves (Sec. 5.1).

Conventions shared by every array here:
  * NumPy C order with x fastest: shape (ny, nx) in 2D, (nz, ny, nx) in 3D,
    a Dirac spinor (4, ny, nx);  ``dims`` lists sides in axis order (nx, ny, nz);
  * lattice x_{a,j} = -n_a h_a/2 + j h_a on the periodic box [-L/2, L/2);
  * field samples are taken at step midpoints t_n + dt/2, shape (n_steps, ndim),
    components in axis order (x, y, z);
  * seeds are NumPy PCG64 ``default_rng(1000 + config_index)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field
from typing import Optional, Tuple

import numpy as np

C_LIGHT = 137.036  # speed of light in atomic units


@dataclass
class Workload:
    """One propagation problem: initial state, potential, field, step size."""
    name: str
    dims: Tuple[int, ...]            # (nx, ny, nz) axis order
    spacing: Tuple[float, ...]       # (h_x, h_y, h_z)
    comps: int                       # 1 Schroedinger, 4 Dirac
    psi0: np.ndarray                 # complex128, (…, ny, nx) or (4, …, ny, nx)
    V: Optional[np.ndarray]          # float64 spatial shape, potential energy
    dt: float
    n_steps: int
    field: Optional[np.ndarray]      # (n_steps, ndim) float64, E (Schr) or A (Dirac)
    mass: float = 1.0
    charge: float = -1.0
    hbar: float = 1.0
    c: float = C_LIGHT
    meta: dict = dc_field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return len(self.dims)

    @property
    def npoints(self) -> int:
        return int(np.prod(self.dims))

    @property
    def shape(self) -> Tuple[int, ...]:
        return tuple(self.dims[::-1])


def lattice(n: int, h: float) -> np.ndarray:
    """x_j = -n h/2 + j h, j = 0..n-1."""
    return -0.5 * n * h + h * np.arange(n, dtype=np.float64)


def mesh(dims, spacing):
    """Coordinate arrays in NumPy order: returns [x, y, z][:ndim], each of the
    spatial shape (…, ny, nx)."""
    axes = [lattice(n, h) for n, h in zip(dims, spacing)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # (z, y, x) order
    return grids[::-1]


def momenta(n: int, h: float, hbar: float = 1.0) -> np.ndarray:
    """p_k = hbar 2 pi kappa_k/(n h) with kappa from numpy.fft.fftfreq
    (the Nyquist index maps to -n/2)."""
    return hbar * 2.0 * np.pi * np.fft.fftfreq(n, d=h)


def normalise(psi: np.ndarray, spacing, comps: int = 1) -> np.ndarray:
    dV = float(np.prod(spacing))
    nrm = np.sqrt(dV * np.sum(np.abs(psi) ** 2))
    return psi / nrm


def gaussian(dims, spacing, center, sigma: float, p0=None) -> np.ndarray:
    """exp(-|x - x0|^2/(2 sigma^2) + i p0.x), normalised to dV sum |psi|^2 = 1.
    sigma is the amplitude width, so sigma = sqrt(1/omega) is the harmonic
    ground-state width."""
    X = mesh(dims, spacing)
    arg = np.zeros(X[0].shape, dtype=np.complex128)
    for a in range(len(dims)):
        arg += -((X[a] - center[a]) ** 2) / (2.0 * sigma * sigma)
        if p0 is not None:
            arg += 1j * p0[a] * X[a]
    return normalise(np.exp(arg), spacing)


def soft_core(dims, spacing, a2: float, Z: float = 1.0) -> np.ndarray:
    """V = -Z / sqrt(r^2 + a2) (the soft-core form of Eq. 44 with a2 given)."""
    X = mesh(dims, spacing)
    r2 = sum(x * x for x in X)
    return -Z / np.sqrt(r2 + a2)


def harmonic(dims, spacing, omega: float) -> np.ndarray:
    """V = omega^2 |x|^2 / 2 (m = 1)."""
    X = mesh(dims, spacing)
    return 0.5 * omega * omega * sum(x * x for x in X)


def sin2_pulse(n_steps: int, dt: float, amp: float, omega: float, T: float) -> np.ndarray:
    """f(t_n + dt/2) for f(t) = amp sin^2(pi t/T) cos(omega t)."""
    t = (np.arange(n_steps, dtype=np.float64) + 0.5) * dt
    return amp * np.sin(np.pi * t / T) ** 2 * np.cos(omega * t)


def dirac_positive_spin_up(psi_scalar: np.ndarray, dims, spacing, mass: float = 1.0,
                           c: float = C_LIGHT, hbar: float = 1.0) -> np.ndarray:
    """Project a scalar packet onto positive-energy spin-up plane-wave spinors
    per momentum (Sec. 5.1): psi~_s(p) times the textbook free-particle spinor
    sqrt((E+mc^2)/(2E)) (1, 0, c p_z/(E+mc^2), c (p_x + i p_y)/(E+mc^2)),
    E = sqrt(m^2 c^4 + p^2 c^2), then back to real space and normalised."""
    ndim = len(dims)
    P = np.meshgrid(*[momenta(n, h, hbar) for n, h in zip(dims, spacing)][::-1], indexing="ij")[::-1]
    px = P[0]
    py = P[1] if ndim > 1 else np.zeros_like(px)
    pz = P[2] if ndim > 2 else np.zeros_like(px)
    mc2 = mass * c * c
    E = np.sqrt(mc2 * mc2 + (px * px + py * py + pz * pz) * c * c)
    nrm = np.sqrt((E + mc2) / (2.0 * E))
    st = np.fft.fftn(psi_scalar)
    comps = np.stack([
        nrm * st,
        np.zeros_like(st),
        nrm * c * pz / (E + mc2) * st,
        nrm * c * (px + 1j * py) / (E + mc2) * st,
    ])
    out = np.stack([np.fft.ifftn(comps[k]) for k in range(4)])
    return normalise(out, spacing)


def random_state(shape, seed: int, spacing=None) -> np.ndarray:
    """Complex normal samples, normalised (for generic parity cases)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if spacing is None:
        return z / np.sqrt(np.sum(np.abs(z) ** 2))
    return normalise(z, spacing)


def random_smooth_state(dims, spacing, seed: int, n_packets: int = 3, comps: int = 1) -> np.ndarray:
    """Sum of a few seeded Gaussian packets with random centres/momenta, so the
    state is resolved on the lattice (used for longer runs at FP32)."""
    rng = np.random.default_rng(seed)
    L = [n * h for n, h in zip(dims, spacing)]
    parts = []
    for _ in range(comps):
        acc = 0
        for _ in range(n_packets):
            ctr = [rng.uniform(-0.2, 0.2) * l for l in L]
            sig = rng.uniform(0.05, 0.1) * min(L)
            p0 = [rng.uniform(-0.2, 0.2) * np.pi / h for h in spacing]
            acc = acc + (rng.standard_normal() + 1j * rng.standard_normal()) * gaussian(dims, spacing, ctr, sig, p0)
        parts.append(acc)
    psi = np.stack(parts) if comps > 1 else parts[0]
    return normalise(psi, spacing)


def random_potential(dims, seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(tuple(dims[::-1]))


def random_field(n_steps: int, ndim: int, seed: int, scale: float = 0.05) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((n_steps, ndim))


# ---------------------------------------------------------------------------
# The paper-shaped configurations.  Sizes can be overridden to build the
# reduced cases the oracle finishes in seconds.
# ---------------------------------------------------------------------------

def config1(n: int = 1024, L: float = 200.0, omega: float = 0.1, x0: float = -20.0,
            dt: float = 0.05, n_steps: int = 2000) -> Workload:
    """1D Schroedinger, harmonic V = omega^2 x^2/2, coherent packet
    sigma = sqrt(1/omega) at x0, p0 = 0; the FP64 plain-path workload."""
    dims = (n,)
    sp = (L / n,)
    psi0 = gaussian(dims, sp, (x0,), np.sqrt(1.0 / omega))
    return Workload("1d_schrodinger_harmonic", dims, sp, 1, psi0, harmonic(dims, sp, omega),
                    dt, n_steps, None, meta=dict(omega=omega, x0=x0, L=L))


def config2(n: int = 2048, L: float = 400.0, dt: float = 0.02, n_steps: int = 5000,
            E0: float = 0.05, omega: float = 0.057, sigma: float = 2.0,
            seed: int = 1002, T: Optional[float] = None) -> Workload:
    """2D Schroedinger on [-L/2, L/2)^2: soft-core V = -1/sqrt(r^2 + 1), dipole
    field along x with E(t) = E0 sin^2(pi t/T) cos(omega t), T = n_steps dt,
    Gaussian sigma = 2 at a seeded offset in [-5, 5]^2."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(-5.0, 5.0, size=2)
    dims = (n, n)
    sp = (L / n, L / n)
    T = n_steps * dt if T is None else T
    Ex = sin2_pulse(n_steps, dt, E0, omega, T)
    field = np.stack([Ex, np.zeros_like(Ex)], axis=1)
    psi0 = gaussian(dims, sp, off, sigma)
    return Workload("2d_schrodinger_softcore_laser", dims, sp, 1, psi0, soft_core(dims, sp, 1.0),
                    dt, n_steps, field, meta=dict(offset=off.tolist(), E0=E0, omega=omega, T=T, L=L))


def config3(n: int = 512, L: float = 128.0, dt: float = 0.02, n_steps: int = 200,
            E0: float = 0.03, omega: float = 0.057, sigma: float = 1.5,
            seed: int = 1003, T: Optional[float] = None) -> Workload:
    """3D Schroedinger on [-L/2, L/2)^3: V = -1/sqrt(r^2 + 0.5), field along z
    with a sin^2 envelope over T = n_steps dt, Gaussian sigma = 1.5 at a seeded
    offset in [-5, 5]^3."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(-5.0, 5.0, size=3)
    dims = (n, n, n)
    sp = (L / n,) * 3
    T = n_steps * dt if T is None else T
    Ez = sin2_pulse(n_steps, dt, E0, omega, T)
    field = np.stack([np.zeros_like(Ez), np.zeros_like(Ez), Ez], axis=1)
    psi0 = gaussian(dims, sp, off, sigma)
    return Workload("3d_schrodinger_softcore_laser", dims, sp, 1, psi0, soft_core(dims, sp, 0.5),
                    dt, n_steps, field, meta=dict(offset=off.tolist(), E0=E0, omega=omega, T=T, L=L))


def config4(n: int = 1024, L: float = 8.0, dt: float = 1e-4, n_steps: int = 1000,
            A0: float = 20.0, omega: float = 2.0, sigma: float = 0.5, p0=(50.0, 0.0),
            Z: float = 1.0, seed: int = 1004, T: Optional[float] = None) -> Workload:
    """2D Dirac, four components, on [-L/2, L/2)^2, c = 137.036:
    V = -Z/sqrt(r^2 + 0.01), vector potential along x with
    A(t) = A0 sin^2(pi t/T) cos(omega t), T = n_steps dt, Gaussian sigma = 0.5,
    p0 = (50, 0), projected per momentum onto positive-energy spin-up spinors.
    The seed is drawn for the record; the packet starts at the origin."""
    rng = np.random.default_rng(seed)
    _ = rng.uniform()
    dims = (n, n)
    sp = (L / n, L / n)
    T = n_steps * dt if T is None else T
    Ax = sin2_pulse(n_steps, dt, A0, omega, T)
    field = np.stack([Ax, np.zeros_like(Ax)], axis=1)
    scal = gaussian(dims, sp, (0.0, 0.0), sigma, p0)
    psi0 = dirac_positive_spin_up(scal, dims, sp)
    return Workload("2d_dirac_softcore_laser", dims, sp, 4, psi0, soft_core(dims, sp, 0.01, Z),
                    dt, n_steps, field, meta=dict(A0=A0, omega=omega, T=T, L=L, p0=list(p0)))


def dirac3d_packet(n: int = 128, n_steps: int = 50, dt: float = 1e-4) -> Workload:
    """3D four-component Dirac on [-4, 4)^3: soft core V = -1/sqrt(r^2 + 0.01),
    uniform A(t) = (20 cos 2t, 5 sin 2t, 2) at the step midpoints, and a
    positive-energy spin-up packet (Gaussian sigma 0.5, p0 = (50, 0, 0)) at the
    origin."""
    h = 8.0 / n
    dims, sp = (n, n, n), (h, h, h)
    X = mesh(dims, sp)
    t = (np.arange(n_steps) + 0.5) * dt
    A = np.stack([20.0 * np.cos(2.0 * t), 5.0 * np.sin(2.0 * t), 2.0 * np.ones_like(t)], axis=1)
    psi0 = dirac_positive_spin_up(gaussian(dims, sp, (0.0, 0.0, 0.0), 0.5, (50.0, 0.0, 0.0)), dims, sp)
    V = -1.0 / np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2 + 0.01)
    return Workload("3d_dirac_packet", dims, sp, 4, psi0, V, dt, n_steps, A)


def dirac_pulse(n_steps: int = 200) -> Workload:
    """The 2D Dirac lattice, potential and packet of config 4 in a pulse
    travelling along x: A_y(x, t) = 20 sin(eta) sin^2(eta/2) with
    eta = k x - c k t, k = 2 pi / L, sampled at the step midpoints on every
    lattice column; field shape (n_steps, n_x, 2) (meta['profile'] = True)."""
    w = config4(n_steps=n_steps)
    n = w.dims[0]
    x = lattice(n, w.spacing[0])
    k = 2 * np.pi / (n * w.spacing[0])
    t = (np.arange(n_steps) + 0.5) * w.dt
    eta = k * x[None, :] - 137.036 * k * t[:, None]
    A = np.zeros((n_steps, n, 2))
    A[:, :, 1] = 20.0 * np.sin(eta) * np.sin(0.5 * eta) ** 2
    return Workload("2d_dirac_pulse", w.dims, w.spacing, 4, w.psi0, w.V, w.dt, n_steps, A, meta=dict(profile=True))


def velocity_gauge_benchmark() -> Workload:
    """The benchmark workload (config 2) in the velocity gauge: the field
    samples become the vector potential A_n = -dt sum_{m <= n} E_m (so that
    E = -dA/dt), entering the momentum-space factor (meta['gauge'])."""
    w = config2()
    A = -np.cumsum(w.field, axis=0) * w.dt
    return Workload("2d_schrodinger_velocity_gauge", w.dims, w.spacing, 1, w.psi0, w.V, w.dt, w.n_steps, A,
                    meta=dict(w.meta, gauge="velocity"))


CONFIG5_SIDES = (256, 384, 512, 768, 1024, 1536, 2048)


def config5_instance(k: int, seed: int = 1005, n_steps: int = 400, dt: float = 0.05, h: float = 0.2,
                     sides=None) -> Workload:
    """Instance k of the batched + adjoint workload: 2D Schroedinger, sides
    n_x, n_y drawn independently from 256 ... 2048 (radix 2 and 3), spacing
    0.2, soft-core V = -1/sqrt(r^2 + 1), field along x with 400 samples
    E_k ~ N(0, 0.02^2), dt = 0.05, Gaussian psi_0 (sigma = 2) and a Gaussian
    target phi (sigma = 2, p = 0) at independent offsets in [-5, 5]^2
    (meta['phi']).  `sides` overrides the drawn (n_x, n_y)."""
    rng = np.random.default_rng([seed, k])
    nx, ny = (int(rng.choice(CONFIG5_SIDES)), int(rng.choice(CONFIG5_SIDES)))
    if sides is not None:
        nx, ny = sides
    dims = (nx, ny)
    sp = (h, h)
    off = rng.uniform(-5.0, 5.0, size=2)
    offt = rng.uniform(-5.0, 5.0, size=2)
    ex = rng.normal(0.0, 0.02, size=n_steps)
    field = np.stack([ex, np.zeros_like(ex)], axis=1)
    psi0 = gaussian(dims, sp, tuple(off), 2.0)
    phi = gaussian(dims, sp, tuple(offt), 2.0)
    return Workload(f"5_batch_{k}", dims, sp, 1, psi0, soft_core(dims, sp, 1.0), dt, n_steps, field,
                    meta=dict(phi=phi, offset=list(off), target_offset=list(offt), sides=[nx, ny]))


def config5(n_instances: int = 64, seed: int = 1005, n_steps: int = 400):
    """The 64 instances of the batched + adjoint workload."""
    return [config5_instance(k, seed, n_steps) for k in range(n_instances)]


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}
