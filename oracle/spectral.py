"""FP64 spectral method (test infrastructure): autocorrelation, windowed
spectrum and eigenfunctions of the eigenstates subsection of Bauke & Keitel.

Test infrastructure, not product code: only ``tests/`` import this module.

Propagating a trial state psi in a time-independent potential from t = 0 to
T = N dt with the split step (the oracle's own step, one at a time):

    chi(t_n)   = dV sum conj(psi_0) psi_n                       (autocorrelation)
    chi~(E)    = dt sum_n chi(t_n) (1 - cos(2 pi t_n / T)) exp(i t_n E / hbar)
    Psi_E(x)   = dt sum_n psi_n(x) (1 - cos(2 pi t_n / T)) exp(i E t_n / hbar)

with t_n = n dt, n = 0..N; the window vanishes at both ends, so this sum is
the trapezoid and the rectangle rule of the integrals alike.
"""
from __future__ import annotations

import numpy as np

from . import schrodinger_propagate


def spectral(psi0, V, spacing, dt, n_steps, energies, mass=1.0, hbar=1.0, propagate=None):
    """Returns (chi [N+1], spectrum [K], psi_E [K, ...shape]) for the energies E_k.
    propagate(psi, dt) -> psi advances one step (default: the oracle's
    Schroedinger step); for a spinor the sums run over all components and
    dV is the product of the spatial spacings."""
    psi0 = np.asarray(psi0, dtype=np.complex128)
    E = np.atleast_1d(np.asarray(energies, dtype=np.float64))
    N = int(n_steps)
    T = N * dt
    dV = float(np.prod(spacing))
    chi = np.zeros(N + 1, dtype=np.complex128)
    acc = np.zeros((len(E),) + psi0.shape, dtype=np.complex128)
    psi = psi0
    for n in range(N + 1):
        if n > 0:
            psi = (propagate(psi, dt) if propagate is not None
                   else schrodinger_propagate(psi, V, spacing, dt, 1, None, mass=mass, hbar=hbar))
        t = n * dt
        chi[n] = dV * np.vdot(psi0, psi)
        w = 1.0 - np.cos(2.0 * np.pi * t / T)
        for k, e in enumerate(E):
            acc[k] += w * np.exp(1j * t * e / hbar) * psi
    t = dt * np.arange(N + 1)
    win = 1.0 - np.cos(2.0 * np.pi * t / T)
    spec = dt * np.array([np.sum(chi * win * np.exp(1j * t * e / hbar)) for e in E])
    return chi, spec, dt * acc


def peak(energies, values):
    """Energy of the largest |value| on a grid, refined by the parabola
    through it and its two neighbours."""
    a = np.abs(np.asarray(values))
    i = int(np.argmax(a))
    if i == 0 or i == len(a) - 1:
        return float(energies[i])
    y0, y1, y2 = a[i - 1], a[i], a[i + 1]
    d = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return float(energies[i] + d * (energies[1] - energies[0]))
