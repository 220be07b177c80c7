"""FP64 adjoint gradient of a final-state overlap (test infrastructure).

Test infrastructure, not product code: only ``tests/`` import this module.

Objective (a follow-on of the paper's method, not in the paper): for the
Schroedinger split step of Eqs. 6-8 / 10a-b, psi_{n+1} = U_n psi_n with
U_n = A_n B A_n, A_n = exp(-i tau W_n / (2 hbar)), W_n = V - q x.E_n, and
B = F^-1 exp(-i tau p^2 / (2 m hbar)) F, the target overlap is
c = <phi|psi_N> = dV sum conj(phi) psi_N and J = |c|^2.

Costates: lambda_N = phi, lambda_n = U_n^dagger lambda_{n+1}; U_n^dagger is
the same step with tau -> -tau (A_n and B are unitary and A_n is diagonal).
Differentiating U_n (A_n appears twice, and the position operator X_a
commutes with A_n):

    dc/dE_{n,a} = k_E ( <lambda_{n+1}|X_a|psi_{n+1}> + <lambda_n|X_a|psi_n> ),
    k_E = (-i tau / (2 hbar)) (-q)
    dc/dV_j     = k_V dV sum_n w_n conj(lambda_{n,j}) psi_{n,j},
    k_V = -i tau / (2 hbar),  w_n = 1 for n = 0, N and 2 otherwise,
    dJ/dx = 2 Re( conj(c) dc/dx ).

Everything below is a direct transcription of these formulas with the
oracle's own FP64 step (sop_oracle.c), one step at a time, all states kept.
"""
from __future__ import annotations

import numpy as np

from . import schrodinger_propagate


def _coords(shape, spacing):
    """Lattice coordinate arrays x_a (a in axis order x, y, z) broadcast to
    the NumPy shape (…, ny, nx); x_{a,j} = -n_a h_a / 2 + j h_a."""
    nd = len(shape)
    out = []
    for a in range(nd):
        n = shape[nd - 1 - a]
        h = spacing[a]
        x = -0.5 * n * h + h * np.arange(n)
        sh = [1] * nd
        sh[nd - 1 - a] = n
        out.append(np.broadcast_to(x.reshape(sh), shape))
    return out


def schrodinger_adjoint(psi0, V, spacing, dt, n_steps, field, phi, mass=1.0, charge=-1.0, hbar=1.0):
    """Returns (J, dJ/dfield with shape (n_steps, ndim), dJ/dV with the shape
    of psi0).  field: (n_steps, ndim) samples (midpoint of each step)."""
    psi0 = np.asarray(psi0, dtype=np.complex128)
    phi = np.asarray(phi, dtype=np.complex128)
    nd = psi0.ndim
    N = int(n_steps)
    F = np.asarray(field, dtype=np.float64).reshape(N, nd)
    dV = float(np.prod(spacing[:nd]))
    kw = dict(mass=mass, charge=charge, hbar=hbar)

    psis = [psi0]
    for n in range(N):
        psis.append(schrodinger_propagate(psis[-1], V, spacing, dt, 1, F[n:n + 1], **kw))
    lams = [None] * (N + 1)
    lams[N] = phi
    for n in range(N - 1, -1, -1):
        lams[n] = schrodinger_propagate(lams[n + 1], V, spacing, -dt, 1, F[n:n + 1], **kw)

    c = dV * np.vdot(phi, psis[N])
    X = _coords(psi0.shape, spacing)
    s = np.array([[dV * np.vdot(lams[m], X[a] * psis[m]) for a in range(nd)] for m in range(N + 1)])
    kE = (-1j * dt / (2.0 * hbar)) * (-charge)
    dc_dE = kE * (s[1:] + s[:-1])
    acc = np.zeros(psi0.shape, dtype=np.complex128)
    for m in range(N + 1):
        w = 1.0 if m in (0, N) else 2.0
        acc += w * np.conj(lams[m]) * psis[m]
    kV = -1j * dt / (2.0 * hbar)
    dc_dV = kV * dV * acc
    J = float(abs(c) ** 2)
    return J, 2.0 * np.real(np.conj(c) * dc_dE), 2.0 * np.real(np.conj(c) * dc_dV)


def objective(psi0, V, spacing, dt, n_steps, field, phi, mass=1.0, charge=-1.0, hbar=1.0):
    """J = |<phi|psi_N>|^2 by forward propagation only (for finite differences)."""
    psiN = schrodinger_propagate(psi0, V, spacing, dt, n_steps, field, mass=mass, charge=charge, hbar=hbar)
    dV = float(np.prod(spacing[:np.asarray(psi0).ndim]))
    return float(abs(dV * np.vdot(np.asarray(phi, dtype=np.complex128), psiN)) ** 2)
