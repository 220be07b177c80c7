"""The adjoint gradient on the GPU against the oracle's FP64 adjoint (which
the CPU tests pin to central finite differences)."""
import numpy as np
import pytest

import gpu_cases as gc
from oracle import adjoint as oadj
from paper_1012_3911_gb300 import sop, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def _small_case(dims, n_steps, seed):
    w = gc.random_workload(dims, 1, seed=seed, n_steps=n_steps, dt=0.05, field_scale=0.3, v_scale=1.0)
    phi = wl.gaussian(dims, w.spacing, [-0.5] + [0.2] * (len(dims) - 1), 1.0)
    return w, phi


def _gpu_adjoint(w, phi, dtype, every):
    import torch
    p = sop.Propagator(w.dims, w.spacing, 1, dtype)
    p.set_state(torch.from_numpy(w.psi0))
    if w.V is not None:
        p.set_potential(w.V)
    gV = torch.zeros(w.psi0.shape, dtype=torch.float64, device="cuda")
    J, gE = p.adjoint_gradient(phi, w.n_steps, w.dt, w.field, every, gV)
    psi_after = p.state.cpu().numpy()
    p.close()
    return J, gE, gV.cpu().numpy(), psi_after


def _check(J, gE, gV, ref, tol):
    Jr, gEr, gVr = ref
    assert abs(J - Jr) <= tol * abs(Jr), (J, Jr)
    assert np.abs(gE - gEr).max() <= tol * np.abs(gEr).max(), np.abs(gE - gEr).max() / np.abs(gEr).max()
    assert np.abs(gV - gVr).max() <= tol * np.abs(gVr).max(), np.abs(gV - gVr).max() / np.abs(gVr).max()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("dims,n_steps,every", [((64, 48), 30, 7), ((32, 24, 16), 9, 4), ((96, 64), 5, 20),
                                                ((64, 32), 6, 1)])
def test_adjoint_matches_oracle(dtype, dims, n_steps, every):
    w, phi = _small_case(dims, n_steps, 21)
    ref = oadj.schrodinger_adjoint(w.psi0, w.V, w.spacing, w.dt, n_steps, w.field, phi)
    J, gE, gV, psi_after = _gpu_adjoint(w, phi, dtype, every)
    _check(J, gE, gV, ref, 1e-9 if dtype == "c128" else 1e-4)
    # the bound state is left as it was
    assert np.array_equal(psi_after, w.psi0.astype(np.complex64 if dtype == "c64" else np.complex128))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_adjoint_config5_instance(dtype):
    """One instance of the batched + adjoint workload at its own size (mixed
    radix sides), 400 steps, checkpoints every 20, against the oracle."""
    w = wl.config5_instance(3, sides=(384, 256))
    phi = w.meta["phi"]
    ref = oadj.schrodinger_adjoint(w.psi0, w.V, w.spacing, w.dt, w.n_steps, w.field, phi)
    J, gE, gV, _ = _gpu_adjoint(w, phi, dtype, 20)
    _check(J, gE, gV, ref, 1e-9 if dtype == "c128" else 1e-4)


def test_autograd_function():
    import torch
    from paper_1012_3911_gb300.adjoint import overlap_objective
    w, phi = _small_case((48, 32), 12, 23)
    p = sop.Propagator(w.dims, w.spacing, 1, "c128")
    field = torch.tensor(w.field, dtype=torch.float64, requires_grad=True)
    V = torch.tensor(w.V, dtype=torch.float64, device="cuda", requires_grad=True)
    psi0 = torch.from_numpy(w.psi0).cuda()
    phi_t = torch.from_numpy(phi).cuda()
    J = overlap_objective(p, psi0, phi_t, field, V, w.dt, every=5)
    J.backward()
    Jr, gEr, gVr = oadj.schrodinger_adjoint(w.psi0, w.V, w.spacing, w.dt, w.n_steps, w.field, phi)
    assert float(J.detach()) == pytest.approx(Jr, rel=1e-10)
    assert np.abs(field.grad.numpy() - gEr).max() <= 1e-9 * np.abs(gEr).max()
    assert np.abs(V.grad.cpu().numpy() - gVr).max() <= 1e-9 * np.abs(gVr).max()
    p.close()


def test_adjoint_rejects_dirac_and_bad_arguments():
    import torch
    p = sop.Propagator((32, 16), (0.2, 0.2), 4, "c64")
    phi = torch.zeros_like(p.state)
    with pytest.raises(sop.SopError):
        sop.sop_adjoint_gradient(p.plan, phi, 4, 0.01, None, 2, 2)
    p.close()
    q = sop.Propagator((32, 16), (0.2, 0.2), 1, "c64")
    phi = torch.zeros_like(q.state)
    for n, dt, every in [(0, 0.01, 2), (4, 0.0, 2), (4, 0.01, 0), (4, float("nan"), 2)]:
        with pytest.raises(sop.SopError):
            sop.sop_adjoint_gradient(q.plan, phi, n, dt, None, every, 2)
    q.close()


def test_adjoint_reuses_its_buffers_and_follows_the_potential():
    """Repeated calls on one plan (the checkpoint block kept between calls,
    grown for a longer run, reused for a shorter one) give exactly the
    results of a fresh plan, and a new potential reaches the -dt plan."""
    import torch
    w, phi = _small_case((64, 48), 30, 33)
    p = sop.Propagator(w.dims, w.spacing, 1, "c64")
    p.set_state(torch.from_numpy(w.psi0))
    p.set_potential(w.V)
    p.set_pass_shape(1, 3)   # a tuned shape: the -dt plan must take it too (bitwise the same)
    gV = torch.zeros(w.psi0.shape, dtype=torch.float64, device="cuda")
    short = p.adjoint_gradient(phi, 12, w.dt, w.field[:12], 5, gV)
    gV_short = gV.clone()
    long_ = p.adjoint_gradient(phi, 30, w.dt, w.field, 7, gV)
    gV_long = gV.clone()
    again = p.adjoint_gradient(phi, 12, w.dt, w.field[:12], 5, gV)
    assert again[0] == short[0] and np.array_equal(again[1], short[1]) and torch.equal(gV, gV_short)
    V2 = w.V * 0.5
    p.set_potential(V2)
    moved = p.adjoint_gradient(phi, 30, w.dt, w.field, 7, gV)
    p.close()
    fresh = sop.Propagator(w.dims, w.spacing, 1, "c64")
    fresh.set_state(torch.from_numpy(w.psi0))
    fresh.set_potential(V2)
    gV2 = torch.zeros_like(gV)
    ref = fresh.adjoint_gradient(phi, 30, w.dt, w.field, 7, gV2)
    fresh.close()
    assert moved[0] == ref[0] and np.array_equal(moved[1], ref[1]) and torch.equal(gV, gV2)
    assert moved[0] != long_[0]
    ref_long = oadj.schrodinger_adjoint(w.psi0, w.V, w.spacing, w.dt, 30, w.field, phi)
    _check(long_[0], long_[1], gV_long.cpu().numpy(), ref_long, 1e-4)
