"""Shared helpers of the GPU parity tests: run one workload through the C ABI
(libsop.so via the ctypes binding) and through the FP64 oracle on the same
seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1012_3911_gb300 import workloads as wl

# Parity bars.  FP64: the stated 1e-10 relative L2.  FP32: 2e-4 after a full
# step count; for a handful of steps the FP32 rounding floor (a few 1e-7 per
# transform) allows a tighter 2e-5.
TOL_F64 = 1e-10
TOL_F32_FULL = 2e-4
TOL_F32_SHORT = 2e-5


def relerr(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1012_3911_gb300 import build
    build.build()


def run_gpu(w: wl.Workload, dtype: str, n_steps=None, field="default", chunks=None, stream=None):
    """Propagate w.psi0 on the GPU; returns (psi as complex128 numpy, propagator)."""
    import torch
    from paper_1012_3911_gb300.sop import Propagator
    n = w.n_steps if n_steps is None else n_steps
    F = w.field if isinstance(field, str) else field
    if F is not None:
        F = np.asarray(F)[:n]
    prop = Propagator(w.dims, w.spacing, w.comps, dtype,
                      params=dict(mass=w.mass, charge=w.charge, hbar=w.hbar, c=w.c), stream=stream)
    prop.set_state(torch.from_numpy(w.psi0))
    if w.V is not None:
        prop.set_potential(w.V)
    if chunks is None:
        prop.step(n, w.dt, F)
    else:
        done = 0
        for c in chunks:
            prop.step(c, w.dt, None if F is None else F[done:done + c])
            done += c
        assert done == n
    torch.cuda.synchronize()
    return prop.state.cpu().numpy().astype(np.complex128), prop


_ORACLE_CACHE = {}


def run_oracle(w: wl.Workload, n_steps=None, field="default"):
    """Oracle result for the workload; cached within the session so the two
    precisions of a parametrised test share one oracle run."""
    n = w.n_steps if n_steps is None else n_steps
    key = (w.name, w.dims, w.spacing, w.dt, n, isinstance(field, str),
           hash(w.psi0.tobytes()), None if w.V is None else hash(w.V.tobytes()),
           None if w.field is None else hash(np.asarray(w.field).tobytes()))
    if isinstance(field, str) and key in _ORACLE_CACHE:
        return _ORACLE_CACHE[key]
    out = _run_oracle(w, n, field)
    if isinstance(field, str):
        while len(_ORACLE_CACHE) >= 6:
            _ORACLE_CACHE.pop(next(iter(_ORACLE_CACHE)))
        _ORACLE_CACHE[key] = out
    return out


def _run_oracle(w: wl.Workload, n, field):
    F = w.field if isinstance(field, str) else field
    if F is not None:
        F = np.asarray(F)[:n]
    if w.comps == 1:
        return oracle.schrodinger_propagate(w.psi0, w.V, w.spacing, w.dt, n, F, w.mass, w.charge, w.hbar)
    return oracle.dirac_propagate(w.psi0, w.V, w.spacing, w.dt, n, F, w.mass, w.charge, w.hbar, w.c)


def random_workload(dims, comps, seed, n_steps, dt, field_scale, v_scale=1.0, spacing=None):
    """Seeded generic case: smooth random state, random potential and field."""
    if spacing is None:
        spacing = tuple(0.1 + 0.05 * a for a in range(len(dims)))
    if comps == 1:
        psi0 = wl.random_smooth_state(dims, spacing, seed)
    else:
        psi0 = wl.random_smooth_state(dims, spacing, seed, comps=4)
    V = wl.random_potential(dims, seed + 1, v_scale) if v_scale else None
    F = wl.random_field(n_steps, len(dims), seed + 2, field_scale) if field_scale else None
    return wl.Workload(f"random{dims}", tuple(dims), tuple(spacing), comps, psi0, V, dt, n_steps, F)
