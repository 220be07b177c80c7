"""GPU path (libsop.so through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs: relative L2 error within 1e-10 on the FP64
path and within 2e-4 (full step counts) or 2e-5 (a few steps) on the FP32
path.  Sizes span several CTAs and ragged tails (pencil counts that are not a
multiple of the pencils per CTA), radix-3 sides, every supported rank, and the
Dirac spinor."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


DT_SCHR = 0.05

# (dims, steps): 1D, 2D and 3D Schroedinger shapes with radix-3 sides and
# pencil counts that leave partial CTAs.
SCHR_CASES = [
    ((8,), 3), ((12,), 2), ((16,), 5), ((24,), 3), ((48,), 4), ((96,), 2), ((384,), 3), ((1024,), 6),
    ((3072,), 2), ((4096,), 2),
    ((16, 8), 3), ((12, 24), 2), ((64, 48), 3), ((96, 8), 2), ((384, 24), 2), ((8, 768), 2),
    ((256, 12), 3), ((2048, 12), 2), ((12, 1536), 2),
    ((16, 12, 8), 2), ((8, 8, 8), 3), ((24, 32, 48), 2), ((64, 8, 12), 2), ((12, 96, 16), 2),
]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims,steps", SCHR_CASES, ids=[f"{'x'.join(map(str, d))}-{s}" for d, s in SCHR_CASES])
def test_schrodinger_random(dims, steps, dtype):
    w = gc.random_workload(dims, 1, seed=100 + sum(dims), n_steps=steps, dt=DT_SCHR, field_scale=0.2)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    err = gc.relerr(out, ref)
    tol = gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT
    assert err < tol, (dims, dtype, err)


DIRAC_CASES = [((8, 8), 2), ((16, 12), 3), ((32, 24), 2), ((64, 64), 3), ((24, 96), 2), ((256, 16), 2),
               ((12, 384), 2)]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims,steps", DIRAC_CASES, ids=[f"{'x'.join(map(str, d))}-{s}" for d, s in DIRAC_CASES])
def test_dirac_random(dims, steps, dtype):
    w = gc.random_workload(dims, 4, seed=200 + sum(dims), n_steps=steps, dt=2e-4, field_scale=30.0,
                           v_scale=50.0, spacing=(0.02, 0.03))
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    err = gc.relerr(out, ref)
    tol = gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT
    assert err < tol, (dims, dtype, err)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_no_potential_no_field(dtype):
    w = gc.random_workload((32, 24), 1, seed=5, n_steps=4, dt=0.1, field_scale=0.0, v_scale=0.0)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    assert gc.relerr(out, ref) < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_field_chunking_and_split_calls(dtype):
    """More steps than one field-table chunk, and the same run split over
    several sop_step calls (the merged boundary half steps are exact algebra)."""
    w = gc.random_workload((16, 24), 1, seed=9, n_steps=700, dt=0.02, field_scale=0.3)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    tol = gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL
    assert gc.relerr(out, ref) < tol
    out2, _ = gc.run_gpu(w, dtype, chunks=[1, 299, 400])
    assert gc.relerr(out2, ref) < tol


def test_one_dimensional_field_chunking():
    w = gc.random_workload((64,), 1, seed=11, n_steps=1100, dt=0.02, field_scale=0.3)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, "c128")
    assert gc.relerr(out, ref) < gc.TOL_F64


# ---------------------------------------------------------------------------
# Paper-shaped workloads at their full step counts (reduced lattices where the
# oracle would take minutes), both precisions.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config1_harmonic_full(dtype):
    w = wl.config1()
    ref = gc.run_oracle(w)
    out, prop = gc.run_gpu(w, dtype)
    err = gc.relerr(out, ref)
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL), err
    assert abs(prop.norm() - 1.0) < (1e-12 if dtype == "c128" else 1e-4)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config2_reduced_lattice_full_steps(dtype):
    w = wl.config2(n=256, L=50.0)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    err = gc.relerr(out, ref)
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL), err


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config3_reduced_lattice_full_steps(dtype):
    w = wl.config3(n=48, L=12.0)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    err = gc.relerr(out, ref)
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL), err


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config4_reduced_lattice_full_steps(dtype):
    w = wl.config4(n=128, L=4.0)
    ref = gc.run_oracle(w)
    out, _ = gc.run_gpu(w, dtype)
    err = gc.relerr(out, ref)
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_FULL), err


# ---------------------------------------------------------------------------
# Reductions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims,comps", [((1024,), 1), ((48, 32), 1), ((16, 12, 24), 1), ((32, 48), 4)])
def test_norm_and_energy(orc, dims, comps, dtype):
    sp = tuple(0.05 + 0.02 * a for a in range(len(dims)))
    w = gc.random_workload(dims, comps, seed=300 + sum(dims), n_steps=1, dt=1e-3, field_scale=0.0,
                           v_scale=3.0, spacing=sp)
    _, prop = gc.run_gpu(w, dtype, n_steps=0)
    psi = prop.state.cpu().numpy().astype(np.complex128)
    n_ref = orc.norm(psi, sp, comps)
    e_ref = orc.energy(psi, w.V, sp, comps, w.mass, w.hbar, w.c)
    tol = 1e-12 if dtype == "c128" else 1e-6
    assert abs(prop.norm() - n_ref) < tol * abs(n_ref)
    assert abs(prop.energy() - e_ref) < tol * max(1.0, abs(e_ref))
