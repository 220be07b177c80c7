"""In-tree build of libsop.so (hand-written CUDA for sm_103a, no cmake).

``build()`` compiles the kernel and driver translation units in parallel with
nvcc for ``-gencode arch=compute_103a,code=sm_103a`` and links
``_build/libsop.so`` next to this file.  It is a no-op when the sources and
flags are unchanged since the last build.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
# SOP_CHECK=1 in the environment: the check build (index and alignment tests in
# the pass kernels, canary bytes after every device buffer) in _build_check/
CHECK = os.environ.get("SOP_CHECK", "") == "1"
OUT_DIR = os.path.join(HERE, "_build_check" if CHECK else "_build")
LIB = os.path.join(OUT_DIR, "libsop.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-std=c++17", "-O3", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
          "-Xcompiler", "-O2", f"-I{INCLUDE}", f"-I{CSRC}"] + (["-DSOP_CHECK=1"] if CHECK else [])

# (object name, source, extra defines)
UNITS = [
    ("pass_f32_contig", "sop_pass_inst.cu", ["-DSOP_REAL=float", "-DSOP_CONTIG=1"]),
    ("pass_f32_strided", "sop_pass_inst.cu", ["-DSOP_REAL=float", "-DSOP_CONTIG=0"]),
    ("pass_f64_contig", "sop_pass_inst.cu", ["-DSOP_REAL=double", "-DSOP_CONTIG=1"]),
    ("pass_f64_strided", "sop_pass_inst.cu", ["-DSOP_REAL=double", "-DSOP_CONTIG=0"]),
    ("pass4_f32_contig", "sop_pass4_inst.cu", ["-DSOP_REAL=float", "-DSOP_CONTIG=1"]),
    ("pass4_f32_strided", "sop_pass4_inst.cu", ["-DSOP_REAL=float", "-DSOP_CONTIG=0"]),
    ("pass4_f64_contig", "sop_pass4_inst.cu", ["-DSOP_REAL=double", "-DSOP_CONTIG=1"]),
    ("pass4_f64_strided", "sop_pass4_inst.cu", ["-DSOP_REAL=double", "-DSOP_CONTIG=0"]),
    ("fso1d_f32", "sop_1d_inst.cu", ["-DSOP_REAL=float", "-DSOP_IS_DOUBLE=0"]),
    ("fso1d_f64", "sop_1d_inst.cu", ["-DSOP_REAL=double", "-DSOP_IS_DOUBLE=1"]),
] + [
    (f"pass_var{v}_f32_{'contig' if c else 'strided'}", "sop_pass_var.cu",
     ["-DSOP_REAL=float", f"-DSOP_CONTIG={c}", f"-DSOP_VAR={v}"])
    for v in (1, 2, 3, 4, 5, 6, 7) for c in (1, 0)
] + [
    ("peak", "sop_peak.cu", []),
    ("tables", "sop_tables.cu", []),
    ("reduce", "sop_reduce.cu", []),
    ("api", "sop_api.cu", []),
    ("noalloc", "sop_noalloc.cu", []),
    ("adjoint", "sop_adjoint.cu", []),
    ("dirac3d", "sop_dirac3d.cu", []),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsop.so")


def _stamp() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            path = os.path.join(d, name)
            if os.path.isfile(path):
                h.update(name.encode())
                with open(path, "rb") as f:
                    h.update(f.read())
    h.update(" ".join(ARCH + CFLAGS).encode())
    h.update(repr(UNITS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every translation unit and link libsop.so; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp_path = os.path.join(OUT_DIR, "stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_path):
        if open(stamp_path).read().strip() == stamp:
            return LIB
    cc = nvcc()

    def compile_unit(unit):
        name, src, defs = unit
        obj = os.path.join(OUT_DIR, name + ".o")
        cmd = [cc] + ARCH + CFLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{r.stderr}")
        if verbose:
            with open(os.path.join(OUT_DIR, name + ".ptxas.txt"), "w") as f:
                f.write(r.stderr)
        return obj

    jobs = jobs or min(len(UNITS), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
