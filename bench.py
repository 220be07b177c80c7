#!/usr/bin/env python
"""Throughput of the Fourier split-operator step on GB300.

One benchmark step is one full propagation of the 2D Schroedinger workload
(2048 x 2048 lattice on [-200, 200)^2, complex64, soft-core Coulomb potential,
sin^2 laser pulse, 5000 split steps of dt = 0.02) through ``sop_step``, with
psi and V resident in HBM.  The metric is grid-point-steps per second
(lattice points x split steps / device time), whole job over all GPUs.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

Under torchrun each rank propagates its own replica (independent problems;
the split step has no cross-GPU exchange), ranks are timed between barriers
and the maximum time is used.  ``--impl reference`` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1012_3911_gb300 import replicas  # noqa: E402  (no torch import at module load)

METRIC = "grid-pt-steps/s and HBM-roofline % per split step, FP32 vs FP64 at stated err"
UNIT = "grid-pt-steps/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10, help="timed benchmark steps")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--split-steps", type=int, default=5000, help="split steps per benchmark step")
    ap.add_argument("--n", type=int, default=2048, help="lattice side")
    ap.add_argument("--fp64-steps", type=int, default=500, help="split steps of the FP64 sample (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="benchmark steps of the end-to-end leg (0: skip)")
    ap.add_argument("--cpu-steps", type=int, default=200,
                    help="oracle split steps of the CPU baseline, about 10-30 s on 16 cores (0: skip)")
    ap.add_argument("--cpu-one-core-steps", type=int, default=8,
                    help="oracle split steps timed on one core beside the all-core baseline (0: skip)")
    ap.add_argument("--ref-split-steps", type=int, default=2, help="oracle split steps per reference step")
    ap.add_argument("--profile-every", type=int, default=64,
                    help="time the passes of one split step in this many (per-class roofline)")
    ap.add_argument("--batched", type=int, default=1, help="also time the batched, adjoint and spectral forms (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=400, help="split steps of the batched / adjoint / spectral sample")
    ap.add_argument("--configs", type=int, default=1,
                    help="also time configs 1, 3, 4 and config 2 in FP64 at full size and length (0: skip)")
    ap.add_argument("--pass-shapes", default=None, help="'C,S': fixed launch shapes instead of sop_autotune")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1012_3911_gb300", "csrc")
    for name in sorted(os.listdir(cs)):
        with open(os.path.join(cs, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


# The sources the pencil-pass kernels are compiled from (device code and the
# argument structures); host-side driver files do not change them.
PASS_KERNEL_FILES = ("sop_async.cuh", "sop_fft.cuh", "sop_kernels.cuh", "sop_internal.h", "sop_pass_inst.cu",
                     "sop_pass_var.cu", "sop_dirac4.cuh")


def pass_kernel_hash() -> str:
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1012_3911_gb300", "csrc")
    for name in PASS_KERNEL_FILES:
        with open(os.path.join(cs, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class: str):
    """Per-launch DRAM bytes of a pass class from the committed ncu summary,
    or None when the pass kernels' sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("pass_kernel_hash") != pass_kernel_hash():
        return None
    ent = d.get("per_launch_dram_bytes", {}).get(kernel_class)
    return None if ent is None else float(ent)


def golden_sample(cfg: int):
    """The FP64 oracle's final state of a paper-shaped configuration at full
    size and full step count, on a seeded sample of lattice values, written by
    tests/golden/make_fullsize.py (oracle and input generators only)."""
    path = os.path.join(ROOT, "tests", "golden", f"fullsize_config{cfg}.npz")
    if not os.path.exists(path):
        return None
    return np.load(path)


def fp64_flop_counts():
    """FP64 operations per lattice point of the complex128 split step, counted
    by ncu (profiles/fp64_flops.json), or None."""
    path = os.path.join(ROOT, "profiles", "fp64_flops.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def config_legs(args, sop, wl, torch, stream, flush, peak):
    """Each paper-shaped configuration in its own right: configs 1 (1D, FP64),
    3 (3D 512^3) and 4 (2D Dirac 1024^2) timed over their full step counts,
    config 2 in FP64 over its full 5000 steps; every run compared with the
    FP64 oracle (config 1 in full, the others on the stored oracle sample)."""
    out = {}

    def run(w, dtype, n_steps=None, tune=True):
        n = w.n_steps if n_steps is None else n_steps
        q = sop.Propagator(w.dims, w.spacing, w.comps, dtype,
                           params=dict(mass=w.mass, charge=w.charge, hbar=w.hbar, c=w.c))
        if w.V is not None:
            q.set_potential(w.V)
        q.set_state(torch.from_numpy(w.psi0))
        shapes = q.autotune(w.dt, 32 if w.npoints < (1 << 24) else 4) if tune else [0, 0]
        F = None if w.field is None else np.asarray(w.field)[:n]
        q.step(min(4, n), w.dt, None if F is None else F[:min(4, n)])   # warm-up
        q.set_state(torch.from_numpy(w.psi0))
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        q.step(n, w.dt, F)
        b.record(stream)
        torch.cuda.synchronize()
        return q, a.elapsed_time(b) * 1e-3, shapes

    def sampled_err(q, g):
        idx = torch.from_numpy(g["idx"]).cuda()
        got = q.state.reshape(-1)[idx].to(torch.complex128).cpu().numpy()
        ref = g["values"]
        return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    # config 1: 1D harmonic coherent state, plain FP64 path, whole line on chip
    import oracle
    w1 = wl.config1()
    q, t, _ = run(w1, "c128", tune=False)
    ref1 = oracle.schrodinger_propagate(w1.psi0, w1.V, w1.spacing, w1.dt, w1.n_steps)
    got1 = q.state.cpu().numpy()
    out["1"] = {"value": w1.npoints * w1.n_steps / t, "unit": UNIT, "dtype": "f64",
                "workload": "1D Schroedinger N=1024 on [-100,100), harmonic V (omega 0.1), coherent packet "
                            "x0=-20, dt 0.05, 2000 steps", "us_per_step": t / w1.n_steps * 1e6,
                "roofline": "n/a: the whole line stays on chip across steps (latency-bound, one CTA)",
                "err_vs_oracle": {"f64": float(np.linalg.norm(got1 - ref1) / np.linalg.norm(ref1)),
                                  "compared": "full state after 2000 steps"}}
    q.close()

    flops = fp64_flop_counts()
    # B_min per point and step (two round trips of psi plus FP32 V) and the
    # bytes the pass design moves (every pass reads and writes psi; the
    # real-space pass reads the 8-byte complex phase table)
    design_pt = {4: 2 * 2 * 32 + 8, 3: 4 * 2 * 8 + 8, 2: 2 * 2 * 8 + 8}
    for cfg, make, b_per_pt in ((4, wl.config4, 4 * 32 + 4), (3, wl.config3, 4 * 8 + 4), (2, wl.config2, 4 * 8 + 4)):
        w = make()
        g = golden_sample(cfg)
        leg = {"workload": w.name, "lattice": list(w.dims), "components": w.comps, "split_steps": w.n_steps}
        for dtype in (("c128",) if cfg == 2 else ("c64", "c128")):
            q, t, shapes = run(w, dtype)
            key = {"c64": "f32", "c128": "f64"}[dtype]
            ent = {"value": w.npoints * w.n_steps / t, "unit": UNIT, "us_per_step": t / w.n_steps * 1e6,
                   "pass_shapes": shapes}
            if dtype == "c64":
                bmin = b_per_pt * w.npoints
                dsg = design_pt[cfg] * w.npoints
                ent["roofline"] = {"bound": "hbm", "step_b_min_bytes": bmin,
                                   "achieved": bmin / (t / w.n_steps) / 1e9, "peak": peak, "unit": "GB/s",
                                   "frac": bmin / (t / w.n_steps) / 1e9 / peak,
                                   "design_bytes_per_step": dsg,
                                   "design_frac": dsg / (t / w.n_steps) / 1e9 / peak}
            elif flops is not None and cfg in (2, 4):
                key_f = {2: "schrodinger_2d", 4: "dirac_2d"}[cfg]
                fpp = flops.get("flops_per_point_step", {}).get(key_f)
                ipp = flops.get("fp64_instructions_per_point_step", {}).get(key_f)
                if fpp:
                    ach = fpp * w.npoints / (t / w.n_steps) / 1e12
                    ent["roofline"] = {"bound": "alu", "achieved": ach, "unit": "TFLOP/s",
                                       "flops_per_point_step": fpp, "peak": None, "frac": None,
                                       "fp64_instr_per_point_step": ipp,
                                       "fp64_instr_per_s": ipp * w.npoints / (t / w.n_steps),
                                       "peak_source": "sop_fma_peak (FP64 FMA chains, measured in this run)"}
            if g is not None:
                ent["err_vs_oracle"] = sampled_err(q, g)
                ent["norm"] = q.norm()
                ent["oracle_norm"] = float(g["norm"])
            leg[key] = ent
            q.close()
            torch.cuda.empty_cache()
        out[str(cfg)] = leg
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    import oracle
    from paper_1012_3911_gb300 import workloads as wl
    oracle.build()
    cores = oracle.max_threads()
    oracle.set_threads(cores)
    w = wl.config2(n=args.n, n_steps=args.split_steps)
    S = args.ref_split_steps
    F = w.field[:S]
    psi = w.psi0
    for _ in range(args.warmup):
        oracle.schrodinger_propagate(psi, w.V, w.spacing, w.dt, S, F)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.schrodinger_propagate(psi, w.V, w.spacing, w.dt, S, F)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = w.npoints * S * args.steps / total
    sample = (f"{S} of {w.n_steps} split steps per benchmark step on the full {args.n}x{args.n} lattice, "
              f"FP64 oracle, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded, paper-shaped)",
        "config": {"workload": f"2D Schroedinger {args.n}x{args.n}, soft-core V, sin^2 laser along x, dt=0.02",
                   "split_steps_per_step": S, "parallelism": "host cores (OpenMP over pencils)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = replicas.dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1012_3911_gb300 import build as sop_build
    sop_build.build()
    from paper_1012_3911_gb300 import sop, workloads as wl

    w = wl.config2(n=args.n, n_steps=args.split_steps)
    S = args.split_steps
    stream = torch.cuda.current_stream()
    prop = sop.Propagator(w.dims, w.spacing, 1, "c64")
    psi0 = torch.from_numpy(w.psi0.astype(np.complex64)).cuda()
    prop.set_potential(w.V)
    prop.state.copy_(psi0)
    if args.pass_shapes:   # fixed shapes (profiling runs), else the autotuner's choice
        pass_shapes = [int(v) for v in args.pass_shapes.split(",")]
        prop.set_pass_shape(0, pass_shapes[0])
        prop.set_pass_shape(1, pass_shapes[1])
    else:
        pass_shapes = prop.autotune(w.dt, 64)   # launch shapes of the x and y passes (untimed)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(ev=None):
        prop.state.copy_(psi0)          # same input every benchmark step (untimed)
        flush.fill_(1.0)                # evict L2 (untimed)
        if ev is not None:
            ev[0].record(stream)
        prop.step(S, w.dt, w.field)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one_step()
    barrier()

    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id  # type: ignore[attr-defined]
    except Exception:
        bus = None
    sampler = ClockSampler(bus)
    sop.sop_profile_enable(prop.plan, args.profile_every)
    sop.sop_profile_read(prop.plan)
    launches0 = sop.sop_launch_counter(prop.plan)
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    sampler.start()
    barrier()
    for k in range(args.steps):
        one_step(events[k])
    barrier()
    clocks = sampler.stop()
    launches = sop.sop_launch_counter(prop.plan) - launches0
    # the state after the last benchmark step is the full 5000-step run: its
    # error against the oracle's stored full-length sample (untimed)
    full_err = None
    g2 = golden_sample(2) if (args.n == 2048 and S == 5000) else None
    if g2 is not None:
        got = prop.state.reshape(-1)[torch.from_numpy(g2["idx"]).cuda()].to(torch.complex128).cpu().numpy()
        full_err = {"f32": float(np.linalg.norm(got - g2["values"]) / np.linalg.norm(g2["values"])),
                    "split_steps": S, "compared": f"{g2['idx'].size} sampled lattice values of the oracle's "
                                                  "final state (tests/golden/fullsize_config2.npz)"}
    cls_ms, cls_n = sop.sop_profile_read(prop.plan)
    sop.sop_profile_enable(prop.plan, 0)
    total_ms = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in events), dist, "cuda")
    value = replicas.job_throughput(w.npoints, S, args.steps, world, total_ms)

    # ---- roofline of the dominant kernel -----------------------------------
    names = sop.PASS_CLASS_NAMES
    dom = int(np.argmax(cls_ms[:2]))
    bytes_per_pt = {0: 2 * 8 + 4, 1: 2 * 8}[dom]   # psi read+write (+ FP32 V on the real-space side)
    alg_bytes = w.npoints * bytes_per_pt
    avg_ms = cls_ms[dom] / max(1, cls_n[dom])
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic(names[dom]), "kernel": names[dom], "peak_source": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
                "profile_every": args.profile_every,
                "source_hash": kernel_source_hash(), "pass_kernel_hash": pass_kernel_hash(),
                "pass_avg_ms": {names[i]: cls_ms[i] / cls_n[i] for i in range(len(cls_ms)) if cls_n[i]},
                "pass_timed_launches": {names[i]: cls_n[i] for i in range(len(cls_ms)) if cls_n[i]}}
    # whole split step against the byte model: B_min = two psi round trips + FP32 V;
    # the pass design moves exactly that in 2D (one x pass, one y pass per step)
    t_split = total_ms / args.steps / S * 1e-3
    b_min = 2 * 2 * 8 * w.npoints + 4 * w.npoints
    roofline["step_b_min_bytes"] = b_min
    roofline["step_b_min_frac"] = b_min / t_split / 1e9 / peak
    # share of the step per class: sampled average x launches per benchmark step
    per_step = {0: S + 1, 1: S, 4: -(-(S + 1) // 512)}
    est = {names[c]: cls_ms[c] / cls_n[c] * k for c, k in per_step.items() if cls_n[c]}
    roofline["pass_ms_share"] = {k: v / sum(est.values()) for k, v in est.items()}

    # ---- batched and adjoint forms (the config-5 workload), complex64 -------
    batched = None
    adjoint = None
    spectral = None
    velocity = None
    dirac1d = None
    dirac3d = None
    dirac_profile = None
    if args.batched and rank == 0:
        ws = wl.config5(64, n_steps=args.batch_steps)
        npts5 = sum(x.npoints for x in ws)
        props = []
        for x in ws:
            q = sop.Propagator(x.dims, x.spacing, 1, "c64")
            q.set_state(torch.from_numpy(x.psi0))
            q.set_potential(x.V)
            q.autotune(x.dt, 8)   # launch shapes per lattice shape (cached); each size group uses its first member's
            props.append(q)
        bat = sop.Batch(props)
        fields = [x.field for x in ws]
        bat.step(2, ws[0].dt, [f[:2] for f in fields])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        bat.step(args.batch_steps, ws[0].dt, fields)
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) * 1e-3
        # the same batch with every step launched directly (no replayed graph)
        os.environ["SOP_BATCH_GRAPH"] = "0"
        bat_d = sop.Batch(props)
        os.environ.pop("SOP_BATCH_GRAPH")
        bat_d.step(2, ws[0].dt, [f[:2] for f in fields])
        flush.fill_(1.0)
        e0.record(stream)
        bat_d.step(args.batch_steps, ws[0].dt, fields)
        e1.record(stream)
        torch.cuda.synchronize()
        td = e0.elapsed_time(e1) * 1e-3
        bat_d.close()
        flush.fill_(1.0)
        e0.record(stream)
        for q, x in zip(props, ws):
            q.step(args.batch_steps, x.dt, x.field)
        e1.record(stream)
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1) * 1e-3
        batched = {"value": npts5 * args.batch_steps / tb, "unit": UNIT, "dtype": "f32",
                   "workload": f"64 independent 2D Schroedinger lattices, sides from 256..2048 (radix 2 and 3), "
                               f"{npts5} points in all, {args.batch_steps} lockstep split steps (sop_batch_step)",
                   "one_plan_at_a_time": npts5 * args.batch_steps / ts,
                   "direct_launches": npts5 * args.batch_steps / td,
                   "time_loop": "middle steps replayed as one captured CUDA graph per step (size groups on "
                                "concurrent streams); first and last step launched directly"}
        # adjoint gradient of |<phi|psi_N>|^2 on one instance of that workload
        x = ws[0]
        q = props[0]
        q.set_state(torch.from_numpy(x.psi0))
        phi = torch.from_numpy(x.meta["phi"]).to(q.state.dtype).cuda()
        gV = torch.zeros(x.psi0.shape, dtype=torch.float64, device="cuda")
        q.adjoint_gradient(phi, args.batch_steps, x.dt, x.field, 20, gV)   # warm-up: buffers, -dt tables
        torch.cuda.synchronize()
        ta = tf = float("inf")
        for _ in range(3):   # best of three, each form; the forward run advances the state copy
            t0 = time.perf_counter()
            q.adjoint_gradient(phi, args.batch_steps, x.dt, x.field, 20, gV)
            torch.cuda.synchronize()
            ta = min(ta, time.perf_counter() - t0)
            q.set_state(torch.from_numpy(x.psi0))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q.step(args.batch_steps, x.dt, x.field)
            torch.cuda.synchronize()
            tf = min(tf, time.perf_counter() - t0)
            q.set_state(torch.from_numpy(x.psi0))
        adjoint = {"value": x.npoints * args.batch_steps / ta, "unit": UNIT, "dtype": "f32",
                   "workload": f"J = |<phi|psi_N>|^2 and its gradient in all {args.batch_steps} field samples and "
                               f"the potential grid, {x.dims[0]}x{x.dims[1]} lattice, checkpoints every 20 steps",
                   "ratio_to_forward": ta / tf,
                   "timing": "best of 3 host-timed calls each (adjoint, then a forward run of the same steps); at this "
                             "lattice both are bound by launch issue (the adjoint issues about 3.3x the forward's "
                             "kernels and copies: forward sweep, recomputed segments, costate sweep, reductions)"}
        bat.close()
        for q in props:
            q.close()
        torch.cuda.empty_cache()
        # spectral method for eigenstates: 2D soft core (zeta = 0.791), trial
        # Gaussian, chi_n every step, the windowed spectrum on 201 energies and
        # the eigenfunctions at 4 of them
        ns, hs = 2048, 0.2
        Vs = wl.soft_core((ns, ns), (hs, hs), 0.791 ** 2)
        psis = wl.gaussian((ns, ns), (hs, hs), (0.5, -0.3), 1.2)
        q = sop.Propagator((ns, ns), (hs, hs), 1, "c64")
        q.set_potential(Vs)
        Es = np.linspace(-0.6, -0.4, 201)
        q.set_state(torch.from_numpy(psis))
        q.spectral(20, 0.05, Es[:4], True)
        torch.cuda.synchronize()
        q.set_state(torch.from_numpy(psis))
        t0 = time.perf_counter()
        q.spectral(args.batch_steps, 0.05, Es, False)
        torch.cuda.synchronize()
        tsp = time.perf_counter() - t0
        q.set_state(torch.from_numpy(psis))
        t0 = time.perf_counter()
        _, _, psiE = q.spectral(args.batch_steps, 0.05, Es[:4], True)
        torch.cuda.synchronize()
        tse = time.perf_counter() - t0
        del psiE
        q.set_state(torch.from_numpy(psis))
        t0 = time.perf_counter()
        q.step(args.batch_steps, 0.05)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        spectral = {"value": ns * ns * args.batch_steps / tse, "unit": UNIT, "dtype": "f32",
                    "workload": f"spectral eigenstates: {ns}x{ns} 2D soft core (zeta 0.791), {args.batch_steps} "
                                f"steps, chi every step, spectrum on 201 energies, eigenfunctions at 4",
                    "spectrum_only": ns * ns * args.batch_steps / tsp,
                    "ratio_to_forward": tse / tf}
        q.close()
        torch.cuda.empty_cache()
        # velocity gauge on the benchmark lattice: A = -integral of E (so that
        # E = -dA/dt), the same split steps with per-step kinetic rows
        qv = sop.Propagator(w.dims, w.spacing, 1, "c64")
        qv.set_gauge("velocity")
        qv.set_potential(w.V)
        Avel = -np.cumsum(w.field, axis=0) * w.dt
        qv.state.copy_(psi0)
        qv.step(4, w.dt, Avel[:4])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qv.state.copy_(psi0)
        flush.fill_(1.0)
        e0.record(stream)
        qv.step(S, w.dt, Avel)
        e1.record(stream)
        torch.cuda.synchronize()
        tv = e0.elapsed_time(e1) * 1e-3
        velocity = {"value": w.npoints * S / tv, "unit": UNIT, "dtype": "f32",
                    "workload": f"benchmark lattice and potential, vector potential A = -int E dt in the "
                                f"momentum-space factor (Eq. 13), {S} split steps",
                    "ratio_to_length_gauge": tv / (total_ms * 1e-3 / args.steps)}
        qv.close()
        torch.cuda.empty_cache()
        # one-dimensional two-component Dirac equation (whole steps on chip):
        # 4096 points on [-4, 4), soft core Z = 1, a^2 = 0.01, A_1 = 20 sin^2 cos 2t
        n1, T1 = 4096, 2000
        h1 = 8.0 / n1
        x1 = wl.lattice(n1, h1)
        t1 = (np.arange(T1) + 0.5) * 1e-4
        A1 = (20.0 * np.sin(np.pi * t1 / (T1 * 1e-4)) ** 2 * np.cos(2.0 * t1)).reshape(T1, 1)
        psi1 = wl.dirac_positive_spin_up(wl.gaussian((n1, 1), (h1, 1.0), (0.0, 0.0), 0.5, (50.0, 0.0)),
                                         (n1, 1), (h1, 1.0))[[0, 3], 0, :]
        qd = sop.Propagator((n1,), (h1,), 2, "c64")
        qd.set_potential(-1.0 / np.sqrt(x1 * x1 + 0.01))
        qd.set_state(torch.from_numpy(psi1))
        qd.step(20, 1e-4, A1[:20])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qd.step(T1, 1e-4, A1)
        e1.record(stream)
        torch.cuda.synchronize()
        td = e0.elapsed_time(e1) * 1e-3
        dirac1d = {"value": n1 * T1 / td, "unit": UNIT, "dtype": "f32",
                   "workload": f"1D two-component Dirac, {n1} points on [-4,4), soft core Z=1 (a^2 0.01), "
                               f"A_1 = 20 sin^2 cos 2t, dt 1e-4, {T1} steps, one CTA keeps the line on chip",
                   "us_per_step": td / T1 * 1e6}
        qd.close()
        # three-dimensional four-component Dirac: 128^3 on [-4,4)^3, soft core,
        # A with three components; 4x4 factors inside four-component x and z
        # passes, the y transforms of the four components as a batch
        w3 = wl.dirac3d_packet(128, 50)
        n3, T3, A3 = w3.dims[0], w3.n_steps, w3.field
        q3 = sop.Propagator(w3.dims, w3.spacing, 4, "c64")
        q3.set_potential(w3.V)
        q3.set_state(torch.from_numpy(w3.psi0))
        del w3
        q3.step(3, 1e-4, A3[:3])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q3.step(T3, 1e-4, A3)
        e1.record(stream)
        torch.cuda.synchronize()
        t3d = e0.elapsed_time(e1) * 1e-3
        npt3 = n3 ** 3
        # streamed bytes per step of the fused design: 4 passes over the 4 components
        # (read + write, 8 B each), the per-momentum table (32 B) and the V phase (8 B);
        # B_min: two round trips of the spinor plus FP32 V
        design3 = 4 * 2 * 4 * 8 * npt3 + 32 * npt3 + 8 * npt3
        bmin3 = 2 * 2 * 4 * 8 * npt3 + 4 * npt3
        dirac3d = {"value": npt3 * T3 / t3d, "unit": UNIT, "dtype": "f32",
                   "workload": f"3D four-component Dirac, {n3}^3 on [-4,4)^3, soft core (a^2 0.01), "
                               f"A = (20 cos 2t, 5 sin 2t, 2), dt 1e-4, {T3} steps",
                   "us_per_step": t3d / T3 * 1e6,
                   "design_bytes_per_step": design3,
                   "design_frac_of_peak": design3 / (t3d / T3) / 1e9 / measured_peaks()[0],
                   "b_min_bytes_per_step": bmin3,
                   "b_min_frac": bmin3 / (t3d / T3) / 1e9 / measured_peaks()[0]}
        q3.close()
        torch.cuda.empty_cache()
        # 2D Dirac in a pulse travelling along x (A_y(x, t), the paper's
        # scattering geometry) on the 1024^2 Dirac lattice, against the same
        # plan with the uniform field of that workload
        w4 = wl.dirac_pulse(200)
        n4, T4, A4 = w4.dims[0], w4.n_steps, w4.field
        w4.field = wl.config4(n_steps=200).field   # the uniform field of the same workload
        qp = sop.Propagator(w4.dims, w4.spacing, 4, "c64")
        qp.set_potential(w4.V)
        qp.set_state(torch.from_numpy(w4.psi0))
        qp.step(4, w4.dt, w4.field[:4])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qp.step(T4, w4.dt, w4.field)
        e1.record(stream)
        torch.cuda.synchronize()
        tu = e0.elapsed_time(e1) * 1e-3
        qp.set_field_profile(True)
        qp.set_state(torch.from_numpy(w4.psi0))
        qp.step(4, w4.dt, A4[:4])
        e0.record(stream)
        qp.step(T4, w4.dt, A4)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) * 1e-3
        dirac_profile = {"value": n4 * n4 * T4 / tp, "unit": UNIT, "dtype": "f32",
                         "workload": f"2D Dirac {n4}^2 (config-4 lattice and potential), A_y(x, t) of a pulse "
                                     f"travelling along x, {T4} steps, per-column mixing inside the x pass of the "
                                     f"component pairs",
                         "us_per_step": tp / T4 * 1e6, "uniform_A_us_per_step": tu / T4 * 1e6}
        qp.close()
        torch.cuda.empty_cache()

    # ---- every configuration at full size and full step count ---------------
    configs = None
    fma_peaks = None
    if args.configs and rank == 0:
        fma_peaks = {"f64_tflops": sop.sop_fma_peak(True) / 1e12, "f32_tflops": sop.sop_fma_peak(False) / 1e12,
                     "how": "sop_fma_peak: 8 independent FMA chains per thread, 8 CTAs x 256 threads per SM, "
                            "best of 3 launches (CUDA events)"}
        configs = config_legs(args, sop, wl, torch, stream, flush, measured_peaks()[0])
        for leg in configs.values():
            r = leg.get("f64", {}).get("roofline") if isinstance(leg, dict) else None
            if r and r.get("bound") == "alu":
                r["peak"] = fma_peaks["f64_tflops"]
                r["frac"] = r["achieved"] / r["peak"]
                # the FP64 pipe issues one DADD, DMUL or DFMA per slot: its
                # occupancy against the measured FMA issue rate (peak / 2)
                r["pipe_frac"] = r.pop("fp64_instr_per_s") / (r["peak"] * 1e12 / 2)

    # ---- FP64 sample, same lattice -----------------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        p64 = sop.Propagator(w.dims, w.spacing, 1, "c128")
        p64.set_potential(w.V)
        psi64 = torch.from_numpy(w.psi0).cuda()
        S64 = args.fp64_steps
        ts = []
        for k in range(3):
            p64.state.copy_(psi64)
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p64.step(S64, w.dt, w.field[:S64])
            b.record(stream)
            torch.cuda.synchronize()
            if k > 0:
                ts.append(a.elapsed_time(b))
        ms = sum(ts) / len(ts)
        fp64 = {"value": w.npoints * S64 / (ms * 1e-3), "unit": UNIT, "split_steps": S64,
                "ms_per_split_step": ms / S64, "dtype": "f64"}
        p64.close()

    # ---- end to end through the C ABI with host buffers ------------------------
    e2e = None
    if args.e2e_steps > 0:
        host = torch.from_numpy(w.psi0.astype(np.complex64)).pin_memory()
        src = host.clone()
        ts = []
        # same per-pass event sampling as the device-timed region, so the two compare
        sop.sop_profile_enable(prop.plan, args.profile_every)
        for k in range(args.e2e_steps + 1):
            host.copy_(src)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            prop.step_host(host, S, w.dt, w.field)
            t1 = time.perf_counter()
            if k > 0:
                ts.append(t1 - t0)
        sop.sop_profile_read(prop.plan)
        sop.sop_profile_enable(prop.plan, 0)
        nbytes = host.numel() * host.element_size()
        e2e = {"value": world * w.npoints * S / (sum(ts) / len(ts)), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # ---- oracle on the host cores (rank 0) and accuracy on that sample -------
    cpu = None
    err = None
    if rank == 0 and args.cpu_steps > 0:
        import oracle
        oracle.build()
        cores = oracle.max_threads()
        oracle.set_threads(cores)
        nc = args.cpu_steps
        t0 = time.perf_counter()
        ref = oracle.schrodinger_propagate(w.psi0, w.V, w.spacing, w.dt, nc, w.field[:nc])
        tcpu = time.perf_counter() - t0
        cpu = {"value": w.npoints * nc / tcpu, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nc} of {S} split steps on the full {args.n}x{args.n} lattice (FP64, {tcpu:.1f} s)"}
        if args.cpu_one_core_steps > 0:
            n1 = args.cpu_one_core_steps
            oracle.set_threads(1)
            t0 = time.perf_counter()
            oracle.schrodinger_propagate(w.psi0, w.V, w.spacing, w.dt, n1, w.field[:n1])
            t1c = time.perf_counter() - t0
            oracle.set_threads(cores)
            cpu["one_core"] = {"value": w.npoints * n1 / t1c, "unit": UNIT, "cores": 1,
                               "sample": f"{n1} split steps, same lattice ({t1c:.1f} s)"}
        err = {"split_steps": nc}
        for dt_name in ("c64", "c128"):
            p = sop.Propagator(w.dims, w.spacing, 1, dt_name)
            p.set_potential(w.V)
            p.set_state(torch.from_numpy(w.psi0))
            p.step(nc, w.dt, w.field[:nc])
            out = p.state.cpu().numpy().astype(np.complex128)
            err[{"c64": "f32", "c128": "f64"}[dt_name]] = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
            p.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded, shaped like the paper's 2D laser-driven soft-core workload)",
            "config": {"workload": f"2D Schroedinger {args.n}x{args.n} on [-200,200)^2, complex64, soft-core V, "
                                   f"sin^2 laser along x, {S} split steps of dt=0.02 per benchmark step",
                       "lattice": [args.n, args.n], "split_steps_per_step": S,
                       "ms_per_split_step": total_ms / args.steps / S,
                       "pass_shapes": {"x": pass_shapes[0], "y": pass_shapes[1],
                                       "chosen_by": "--pass-shapes" if args.pass_shapes else "sop_autotune"},
                       "l2": "flushed (256 MiB write) before every timed step; psi + V tables stay L2-resident "
                             "within a step",
                       "parallelism": f"replicas x{world} (independent problems, no data-path collective)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "err_vs_oracle_full_length": full_err, "configs": configs, "fma_peaks": fma_peaks,
            "fp64": fp64, "batched": batched, "adjoint": adjoint, "spectral": spectral, "velocity_gauge": velocity, "dirac1d": dirac1d, "dirac3d": dirac3d, "dirac_profile": dirac_profile, "err_vs_oracle": err, "clocks": clocks,
        }
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(s + "\n")
    prop.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
