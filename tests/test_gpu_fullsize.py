"""Parity at the full lattice sizes of the paper-shaped workloads, in the
launch configuration the benchmark times: full arrays against the oracle for
a few steps (the oracle needs seconds per step there), and properties that
hold at any size for the full step count."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1012_3911_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_config2_full_lattice_vs_oracle(dtype):
    w = wl.config2()
    ref = gc.run_oracle(w, n_steps=2)
    out, _ = gc.run_gpu(w, dtype, n_steps=2)
    err = gc.relerr(out, ref)
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT), err


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_config4_full_lattice_vs_oracle(dtype):
    w = wl.config4()
    ref = gc.run_oracle(w, n_steps=2)
    out, _ = gc.run_gpu(w, dtype, n_steps=2)
    err = gc.relerr(out, ref)
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT), err


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_config3_full_lattice_vs_oracle(dtype):
    """512^3 (1 GiB of complex64 psi): the streaming 3D passes, element by
    element against the oracle over two split steps (every pass kind)."""
    w = wl.config3()
    ref = gc.run_oracle(w, n_steps=2)
    out, prop = gc.run_gpu(w, dtype, n_steps=2)
    err = gc.relerr(out, ref)
    prop.close()
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT), err


def test_config2_full_run_invariants():
    """The benchmarked workload end to end (2048^2, 5000 steps): the FP32 run
    keeps its norm, and the FP64 run reverses to the initial state."""
    import torch
    w = wl.config2()
    out32, p32 = gc.run_gpu(w, "c64")
    assert abs(p32.norm() - 1.0) < 2e-4
    out64, p64 = gc.run_gpu(w, "c128")
    assert abs(p64.norm() - 1.0) < 1e-11
    # FP32 against FP64 at the full step count (reported accuracy, both GPU)
    assert gc.relerr(out32, out64) < gc.TOL_F32_FULL
    p64.step(w.n_steps, -w.dt, w.field[::-1].copy())
    torch.cuda.synchronize()
    assert gc.relerr(p64.state.cpu().numpy(), w.psi0) < 1e-9
