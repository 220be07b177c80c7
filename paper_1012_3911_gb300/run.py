"""Propagate one of the paper-shaped workloads from the command line.

    python -m paper_1012_3911_gb300.run --config 2 --n 2048 --dtype c64 --steps 3,2

runs ``sop_step`` on the seeded workload of the given configuration (1: 1D
harmonic, 2: 2D laser-driven soft core, 3: 3D, 4: 2D Dirac), in the listed
chunks of steps, and prints norm and energy after each chunk.  Used as a
small driver for profilers as well.
"""
from __future__ import annotations

import argparse
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--n", type=int, default=None, help="lattice side (default: the configuration's)")
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--steps", default="3,2", help="comma-separated chunks of split steps")
    ap.add_argument("--no-energy", action="store_true")
    args = ap.parse_args(argv)

    import torch
    from . import build, workloads as wl
    from .sop import Propagator

    build.build()
    chunks = [int(s) for s in args.steps.split(",") if s]
    kw = {} if args.n is None else {"n": args.n}
    w = wl.CONFIGS[args.config](n_steps=max(1, sum(chunks)), **kw)
    p = Propagator(w.dims, w.spacing, w.comps, args.dtype)
    p.set_state(torch.from_numpy(w.psi0))
    if w.V is not None:
        p.set_potential(w.V)
    done = 0
    for c in chunks:
        t0 = time.perf_counter()
        p.step(c, w.dt, None if w.field is None else w.field[done:done + c])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        done += c
        e = float("nan") if args.no_energy else p.energy()
        print(f"{w.name} {'x'.join(map(str, w.dims))} {args.dtype}: steps {done} ({c} in {dt * 1e3:.2f} ms) "
              f"norm {p.norm():.12f} energy {e:.9f}", flush=True)
    p.close()


if __name__ == "__main__":
    main()
