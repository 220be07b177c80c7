"""Runs one small case of every pass kind through whichever library the
environment selects (SOP_CHECK=1: the check build) and saves the final
states to the .npz file named on the command line; prints one JSON line with
the number of overwritten canaries (-1 in a normal build).  Driven by
tests/test_gpu_check_build.py, which runs it once per build."""
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import gpu_cases as gc  # noqa: E402
from paper_1012_3911_gb300 import sop, workloads as wl  # noqa: E402


def run(dims, comps, dtype, steps, seed, shapes=None, field_scale=0.05, profile=False):
    w = gc.random_workload(dims, comps, seed=seed, n_steps=steps, dt=0.01, field_scale=field_scale)
    p = sop.Propagator(w.dims, w.spacing, comps, dtype)
    if shapes is not None:
        p.set_pass_shape(0, shapes[0])
        p.set_pass_shape(1, shapes[1])
    F = w.field
    if profile:
        p.set_field_profile(True)
        rng = np.random.default_rng(seed)
        F = 20.0 * rng.standard_normal((steps, dims[0], len(dims)))
    p.set_state(torch.from_numpy(w.psi0))
    p.set_potential(w.V)
    p.step(steps, w.dt, F)
    p.norm()   # synchronises; raises if a kernel recorded a failed check
    out = p.state.cpu().numpy()
    p.close()
    return out


def main(path):
    out = {}
    out["s2d"] = run((384, 256), 1, "c64", 3, 11)
    out["s2d_shapes"] = run((384, 256), 1, "c64", 3, 11, shapes=(3, 5))
    out["s2d_big"] = run((1024, 768), 1, "c64", 2, 12, shapes=(7, 2))
    out["s2d_c128"] = run((256, 192), 1, "c128", 2, 13)
    out["s3d"] = run((64, 48, 32), 1, "c64", 2, 14)
    out["s3d_c128"] = run((32, 32, 16), 1, "c128", 2, 15)
    out["d2d"] = run((256, 256), 4, "c64", 2, 16, field_scale=20.0)
    out["d2d_c128"] = run((128, 96), 4, "c128", 2, 17, field_scale=20.0)
    out["d3d"] = run((32, 32, 32), 4, "c64", 2, 18, field_scale=20.0)
    out["pulse"] = run((256, 128), 4, "c64", 3, 19, profile=True)
    # batch of uneven lattices (multi-instance passes)
    ws = [wl.config5_instance(k, sides=s, n_steps=4) for k, s in enumerate([(256, 192), (192, 256)])]
    props = []
    for w in ws:
        q = sop.Propagator(w.dims, w.spacing, 1, "c64")
        q.set_state(torch.from_numpy(w.psi0))
        q.set_potential(w.V)
        props.append(q)
    b = sop.Batch(props)
    b.step(4, ws[0].dt, [w.field for w in ws])
    for k, q in enumerate(props):
        q.norm()
        out[f"batch{k}"] = q.state.cpu().numpy()
    b.close()
    for q in props:
        q.close()
    # adjoint (materialising passes, the -dt plan, segment reductions)
    w = gc.random_workload((64, 48), 1, seed=20, n_steps=9, dt=0.05, field_scale=0.3)
    phi = wl.gaussian((64, 48), w.spacing, (-0.5, 0.2), 1.0)
    q = sop.Propagator(w.dims, w.spacing, 1, "c64")
    q.set_state(torch.from_numpy(w.psi0))
    q.set_potential(w.V)
    gV = torch.zeros(w.psi0.shape, dtype=torch.float64, device="cuda")
    J, gE = q.adjoint_gradient(phi, w.n_steps, w.dt, w.field, 4, gV)
    out["adj_J"] = np.array([J])
    out["adj_gE"] = np.asarray(gE)
    out["adj_gV"] = gV.cpu().numpy()
    q.close()
    torch.cuda.synchronize()
    np.savez(path, **out)
    try:
        bad = sop.sop_debug_check_canaries()
    except sop.SopError:
        bad = -1
    print(json.dumps({"canaries_bad": bad, "cases": sorted(out)}))


if __name__ == "__main__":
    main(sys.argv[1])
