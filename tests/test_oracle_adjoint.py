"""The FP64 adjoint of the oracle against central finite differences of the
oracle's own forward propagation (CPU)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint
from paper_1012_3911_gb300 import workloads as wl


def _case(dims, spacing, n_steps, seed):
    rng = np.random.default_rng(seed)
    psi0 = wl.gaussian(dims, spacing, [0.8] + [0.0] * (len(dims) - 1), 1.2, [0.5] + [0.0] * (len(dims) - 1))
    phi = wl.gaussian(dims, spacing, [-0.6] + [0.3] * (len(dims) - 1), 1.4, [0.0] * len(dims))
    V = wl.random_potential(dims, seed, 1.5)
    F = rng.normal(0.0, 0.3, size=(n_steps, len(dims)))
    return psi0, phi, V, F


@pytest.mark.parametrize("dims,spacing,n_steps,dt", [((24, 16), (0.5, 0.4), 10, 0.05), ((64,), (0.25,), 16, 0.04)])
def test_field_gradient_matches_central_differences(dims, spacing, n_steps, dt):
    psi0, phi, V, F = _case(dims, spacing, n_steps, 11)
    J, gE, gV = adjoint.schrodinger_adjoint(psi0, V, spacing, dt, n_steps, F, phi)
    assert J == pytest.approx(adjoint.objective(psi0, V, spacing, dt, n_steps, F, phi), rel=1e-12)
    h = 1e-5
    fd = np.zeros_like(F)
    for n in range(n_steps):
        for a in range(len(dims)):
            Fp, Fm = F.copy(), F.copy()
            Fp[n, a] += h
            Fm[n, a] -= h
            fd[n, a] = (adjoint.objective(psi0, V, spacing, dt, n_steps, Fp, phi)
                        - adjoint.objective(psi0, V, spacing, dt, n_steps, Fm, phi)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 1e-6                       # a case where the field matters
    assert np.abs(gE - fd).max() < 1e-6 * scale


def test_potential_gradient_matches_central_differences():
    dims, spacing, n_steps, dt = (24, 16), (0.5, 0.4), 8, 0.05
    psi0, phi, V, F = _case(dims, spacing, n_steps, 12)
    J, gE, gV = adjoint.schrodinger_adjoint(psi0, V, spacing, dt, n_steps, F, phi)
    rng = np.random.default_rng(5)
    h = 1e-5
    scale = np.abs(gV).max()
    assert scale > 1e-8
    for _ in range(8):
        j = tuple(int(rng.integers(0, s)) for s in V.shape)
        Vp, Vm = V.copy(), V.copy()
        Vp[j] += h
        Vm[j] -= h
        fd = (adjoint.objective(psi0, Vp, spacing, dt, n_steps, F, phi)
              - adjoint.objective(psi0, Vm, spacing, dt, n_steps, F, phi)) / (2 * h)
        assert abs(gV[j] - fd) < 1e-6 * scale


def test_field_free_target_equal_to_propagated_state():
    """phi = psi_N itself: J = |<psi_N|psi_N>|^2 = 1 is stationary in every
    parameter (unitarity), so the gradient vanishes."""
    dims, spacing, n_steps, dt = (16, 12), (0.5, 0.5), 6, 0.05
    psi0, _, V, F = _case(dims, spacing, n_steps, 13)
    psi0 = psi0 / np.sqrt(oracle.norm(psi0, spacing))
    phi = oracle.schrodinger_propagate(psi0, V, spacing, dt, n_steps, F)
    J, gE, gV = adjoint.schrodinger_adjoint(psi0, V, spacing, dt, n_steps, F, phi)
    assert J == pytest.approx(1.0, abs=1e-12)
    assert np.abs(gE).max() < 1e-10
    assert np.abs(gV).max() < 1e-10


def _fd_field(psi0, phi, V, F, spacing, dt, n_steps):
    h = 1e-5
    fd = np.zeros_like(F)
    for n in range(n_steps):
        for a in range(F.shape[1]):
            Fp, Fm = F.copy(), F.copy()
            Fp[n, a] += h
            Fm[n, a] -= h
            fd[n, a] = (adjoint.objective(psi0, V, spacing, dt, n_steps, Fp, phi)
                        - adjoint.objective(psi0, V, spacing, dt, n_steps, Fm, phi)) / (2 * h)
    return fd


@pytest.mark.parametrize("mutant", ["position_sign", "costate_direction", "end_weights"])
def test_planted_adjoint_mistakes_are_caught(monkeypatch, mutant):
    """A plausible mistake in the adjoint (the sign of the position operator,
    the direction of the costate step, the weights of the end points) moves
    the gradient by far more than the 1e-6 tolerance of the finite-difference
    checks above.  (A constant shift of the lattice origin is not such a
    mistake: <lambda_m|psi_m> = c for every m, so it adds an imaginary term
    that drops out of Re(conj(c) dc).)"""
    dims, spacing, n_steps, dt = (24, 16), (0.5, 0.4), 6, 0.05
    psi0, phi, V, F = _case(dims, spacing, n_steps, 14)
    fd = _fd_field(psi0, phi, V, F, spacing, dt, n_steps)
    if mutant == "position_sign":
        real = adjoint._coords
        monkeypatch.setattr(adjoint, "_coords", lambda shape, sp: [-x for x in real(shape, sp)])
        J, gE, gV = adjoint.schrodinger_adjoint(psi0, V, spacing, dt, n_steps, F, phi)
        bad = np.abs(gE - fd).max()
    elif mutant == "costate_direction":
        real = adjoint.schrodinger_propagate
        monkeypatch.setattr(adjoint, "schrodinger_propagate",
                            lambda psi, V, sp, dt_, n, f, **kw: real(psi, V, sp, abs(dt_), n, f, **kw))
        J, gE, gV = adjoint.schrodinger_adjoint(psi0, V, spacing, dt, n_steps, F, phi)
        bad = np.abs(gE - fd).max()
    else:
        # all weights 2: compare the potential gradient at one point with FD
        J, gE, gV = adjoint.schrodinger_adjoint(psi0, V, spacing, dt, n_steps, F, phi)
        psis = [psi0]
        for n in range(n_steps):
            psis.append(oracle.schrodinger_propagate(psis[-1], V, spacing, dt, 1, F[n:n + 1]))
        lams = [phi]
        for n in range(n_steps - 1, -1, -1):
            lams.insert(0, oracle.schrodinger_propagate(lams[0], V, spacing, -dt, 1, F[n:n + 1]))
        dV = float(np.prod(spacing))
        c = dV * np.vdot(phi, psis[-1])
        acc = sum(2.0 * np.conj(l) * p for l, p in zip(lams, psis))
        g_wrong = 2.0 * np.real(np.conj(c) * (-0.5j * dt) * dV * acc)
        j = (5, 7)
        h = 1e-5
        Vp, Vm = V.copy(), V.copy()
        Vp[j] += h
        Vm[j] -= h
        fdv = (adjoint.objective(psi0, Vp, spacing, dt, n_steps, F, phi)
               - adjoint.objective(psi0, Vm, spacing, dt, n_steps, F, phi)) / (2 * h)
        assert abs(gV[j] - fdv) < 1e-6 * np.abs(gV).max()
        bad = abs(g_wrong[j] - fdv) / np.abs(gV).max()
        assert bad > 1e-4
        return
    assert bad > 1e-4 * np.abs(fd).max()
