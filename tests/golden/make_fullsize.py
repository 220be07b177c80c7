"""Write the full-size, full-length oracle fixtures ``fullsize_config{2,3,4}.npz``
and ``fullsize_{dirac3d,pulse,velocity}.npz``.

Each fixture holds the FP64 oracle's final state of one workload
(``paper_1012_3911_gb300.workloads.config2/3/4`` at their full lattice and full
step count: 2048^2 x 5000 steps, 512^3 x 200 steps, 1024^2 Dirac x 1000 steps;
and the benchmark's follow-on Dirac workloads ``dirac3d_packet``, 128^3 x 50
steps, ``dirac_pulse``, 1024^2 x 200 steps with A varying along x, and
``velocity_gauge_benchmark``, config 2 in the velocity gauge) on a
seeded sample of lattice values, plus the oracle's norm and field-free energy
of that final state and a few checksums of the inputs.  The GPU parity tests
(``tests/test_gpu_fullsize_oracle.py``) propagate the same inputs at full size
and compare the sampled values element by element.

The sample is the union of 8192 indices drawn uniformly over the whole array
(every component, every residue class of the lattice) and 8192 drawn with
probability proportional to |psi_N|^2 (where the wave function lives), from
``default_rng(2000 + config index)``.

Only the oracle and the seeded input generators run here; nothing of the CUDA
path.  Run from the repository root (it takes about 75 minutes on 8 cores):

    python tests/golden/make_fullsize.py [2 3 4 dirac3d pulse velocity]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1012_3911_gb300 import workloads as wl  # noqa: E402

N_UNIFORM = 8192
N_WEIGHTED = 8192


def input_checksums(w: wl.Workload) -> dict:
    """Sums of the inputs, to notice a changed generator (compared with a
    relative tolerance: NumPy's exp/sin may round differently per platform)."""
    out = dict(psi0_sum=complex(w.psi0.sum()), psi0_abs2=float(np.sum(np.abs(w.psi0) ** 2)),
               V_sum=float(w.V.sum()) if w.V is not None else 0.0,
               field_sum=float(np.asarray(w.field).sum()) if w.field is not None else 0.0)
    return out


def sample_indices(psi: np.ndarray, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    flat = np.abs(psi.ravel()) ** 2
    uni = rng.choice(flat.size, size=N_UNIFORM, replace=False)
    wgt = rng.choice(flat.size, size=N_WEIGHTED, replace=False, p=flat / flat.sum())
    return np.unique(np.concatenate([uni, wgt])).astype(np.int64)


# follow-on workloads: generator and sample seed
EXTRA = {"dirac3d": (wl.dirac3d_packet, 2005), "pulse": (wl.dirac_pulse, 2006),
         "velocity": (wl.velocity_gauge_benchmark, 2007)}


def workload(cfg) -> wl.Workload:
    return EXTRA[cfg][0]() if cfg in EXTRA else wl.CONFIGS[cfg]()


def fixture_name(cfg) -> str:
    return f"fullsize_{cfg}.npz" if cfg in EXTRA else f"fullsize_config{cfg}.npz"


def run(cfg) -> str:
    w = workload(cfg)
    t0 = time.time()
    if w.comps == 1:
        out = oracle.schrodinger_propagate(w.psi0, w.V, w.spacing, w.dt, w.n_steps, w.field,
                                           w.mass, w.charge, w.hbar, gauge=w.meta.get("gauge", "length"))
    elif w.meta.get("profile"):
        out = oracle.dirac_propagate_profile(w.psi0, w.V, w.spacing, w.dt, w.n_steps, w.field,
                                             w.mass, w.charge, w.hbar, w.c)
    else:
        out = oracle.dirac_propagate(w.psi0, w.V, w.spacing, w.dt, w.n_steps, w.field,
                                     w.mass, w.charge, w.hbar, w.c)
    secs = time.time() - t0
    idx = sample_indices(out, EXTRA[cfg][1] if cfg in EXTRA else 2000 + cfg)
    nrm = oracle.norm(out, w.spacing, w.comps)
    en = oracle.energy(out, w.V, w.spacing, w.comps, w.mass, w.hbar, w.c)
    cs = input_checksums(w)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), fixture_name(cfg))
    np.savez_compressed(
        path, workload=w.name, dims=np.asarray(w.dims), n_steps=w.n_steps, dt=w.dt,
        comps=w.comps, idx=idx, values=out.ravel()[idx], norm=nrm, energy=en,
        psi0_sum=cs["psi0_sum"], psi0_abs2=cs["psi0_abs2"], V_sum=cs["V_sum"],
        field_sum=cs["field_sum"], oracle_seconds=secs, oracle_threads=oracle.get_threads())
    print(f"{cfg}: {w.dims} x {w.n_steps} steps in {secs:.0f} s on "
          f"{oracle.get_threads()} threads; norm {nrm:.15f} energy {en:.12f}; "
          f"{idx.size} samples -> {path}", flush=True)
    return path


def main(argv):
    oracle.set_threads(oracle.max_threads())
    cfgs = [a if a in EXTRA else int(a) for a in argv] or [4, 2, 3, "dirac3d", "pulse", "velocity"]
    for c in cfgs:
        run(c)


if __name__ == "__main__":
    main(sys.argv[1:])
