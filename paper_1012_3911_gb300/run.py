"""Propagate one of the paper-shaped workloads from the command line.

    python -m paper_1012_3911_gb300.run --config 2 --n 2048 --dtype c64 --steps 3,2

runs ``sop_step`` on the seeded workload of the given configuration (1: 1D
harmonic, 2: 2D laser-driven soft core, 3: 3D, 4: 2D Dirac), in the listed
chunks of steps, and prints norm and energy after each chunk.

    python -m paper_1012_3911_gb300.run --spectral 4 --n 2048 --steps 24

runs ``sop_spectral`` instead: a Gaussian trial state in the 2D soft-core
well of the eigenstates subsection (zeta = 0.791, spacing 0.2, dt = 0.05) for
the given number of steps, the spectrum and the eigenfunctions at that many
energies in [-0.6, -0.4].

    python -m paper_1012_3911_gb300.run --dirac3d --n 128 --steps 10
    python -m paper_1012_3911_gb300.run --pulse --n 1024 --steps 10

step a 3D four-component Dirac packet (n^3 on [-4, 4)^3, soft core, A with
three components) or the 2D Dirac workload in a pulse travelling along x
(A_y(x, t), per-column mixing).  Used as small drivers for profilers as well.
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
    ap.add_argument("--shape", default=None,
                    help="launch shapes 'C,S' of the contiguous and strided passes (default: shape 0)")
    ap.add_argument("--spectral", type=int, default=0,
                    help="run the spectral method with eigenfunctions at this many energies (<= 16)")
    ap.add_argument("--dirac3d", action="store_true", help="3D four-component Dirac packet")
    ap.add_argument("--pulse", action="store_true", help="2D Dirac in a pulse travelling along x")
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    from . import build, workloads as wl
    from .sop import Propagator

    build.build()
    chunks = [int(s) for s in args.steps.split(",") if s]
    if args.dirac3d or args.pulse:
        steps = max(1, sum(chunks))
        if args.dirac3d:
            n = args.n or 128
            h = 8.0 / n
            dims, sp = (n, n, n), (h, h, h)
            X = wl.mesh(dims, sp)
            V = -1.0 / np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2 + 0.01)
            psi0 = wl.dirac_positive_spin_up(wl.gaussian(dims, sp, (0.0, 0.0, 0.0), 0.5, (50.0, 0.0, 0.0)), dims, sp)
            t = (np.arange(steps) + 0.5) * 1e-4
            field = np.stack([20.0 * np.cos(2.0 * t), 5.0 * np.sin(2.0 * t), 2.0 * np.ones_like(t)], axis=1)
            p = Propagator(dims, sp, 4, args.dtype)
        else:
            w = wl.config4(n=args.n or 1024, n_steps=steps)
            dims, sp, V, psi0 = w.dims, w.spacing, w.V, w.psi0
            x = wl.lattice(dims[0], sp[0])
            k = 2 * np.pi / (dims[0] * sp[0])
            eta = k * x[None, :] - 137.036 * k * ((np.arange(steps) + 0.5) * w.dt)[:, None]
            field = np.zeros((steps, dims[0], 2))
            field[:, :, 1] = 20.0 * np.sin(eta) * np.sin(0.5 * eta) ** 2
            p = Propagator(dims, sp, 4, args.dtype)
            p.set_field_profile(True)
        p.set_state(torch.from_numpy(psi0))
        p.set_potential(V)
        t0 = time.perf_counter()
        p.step(steps, 1e-4, field)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"{'dirac3d' if args.dirac3d else 'pulse'} {'x'.join(map(str, dims))} {args.dtype}: {steps} steps in "
              f"{dt * 1e3:.2f} ms, norm {p.norm():.12f}", flush=True)
        p.close()
        return
    if args.spectral:
        n, h = args.n or 2048, 0.2
        steps = max(1, sum(chunks))
        p = Propagator((n, n), (h, h), 1, args.dtype)
        p.set_state(torch.from_numpy(wl.gaussian((n, n), (h, h), (0.5, -0.3), 1.2)))
        p.set_potential(wl.soft_core((n, n), (h, h), 0.791 ** 2))
        E = np.linspace(-0.6, -0.4, args.spectral)
        t0 = time.perf_counter()
        chi, spec, _ = p.spectral(steps, 0.05, E, True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        k = int(np.argmax(np.abs(spec)))
        print(f"spectral {n}x{n} {args.dtype}: {steps} steps in {dt * 1e3:.2f} ms, |chi_N| {abs(chi[-1]):.9f}, "
              f"largest |spectrum| at E = {E[k]:.4f}", flush=True)
        p.close()
        return
    kw = {} if args.n is None else {"n": args.n}
    w = wl.CONFIGS[args.config](n_steps=max(1, sum(chunks)), **kw)
    p = Propagator(w.dims, w.spacing, w.comps, args.dtype)
    if args.shape:
        sc, ss = (int(v) for v in args.shape.split(","))
        p.set_pass_shape(0, sc)
        p.set_pass_shape(1, ss)
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
