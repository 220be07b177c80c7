"""Launch shapes of the pencil passes (pencils per CTA, tile buffers, table
placement, register budget): every shape gives bit-identical states, on the
paper-shaped sides and on ragged ones, and the autotuner keeps the state and
picks a shape whose run still matches the oracle."""
import numpy as np
import pytest
import torch

import gpu_cases as gc
from paper_1012_3911_gb300 import sop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(orc):
    gc.require_gpu()


def run_shape(w, shape_c, shape_s, n_steps, dtype="c64"):
    prop = sop.Propagator(w.dims, w.spacing, w.comps, dtype,
                          params=dict(mass=w.mass, charge=w.charge, hbar=w.hbar, c=w.c))
    prop.set_pass_shape(0, shape_c)
    prop.set_pass_shape(1, shape_s)
    prop.set_state(torch.from_numpy(w.psi0))
    if w.V is not None:
        prop.set_potential(w.V)
    F = None if w.field is None else np.asarray(w.field)[:n_steps]
    prop.step(n_steps, w.dt, F)
    torch.cuda.synchronize()
    out = prop.state.clone()
    prop.close()
    return out


CASES = [
    ((2048, 2048), 1, 3),     # the benchmark lattice
    ((384, 256), 1, 5),       # radix-3 x, ragged
    ((1024, 768), 4, 4),      # Dirac pairs, radix-3 y
    ((256, 384, 512), 1, 3),  # 3D: every pass kind
]


@pytest.mark.parametrize("dims,comps,n_steps", CASES)
def test_every_shape_is_bitwise_the_default(dims, comps, n_steps):
    w = gc.random_workload(dims, comps, seed=len(dims) * 17 + dims[0], n_steps=n_steps, dt=0.01,
                           field_scale=0.05 if comps == 1 else 20.0)
    ref = run_shape(w, 0, 0, n_steps)
    for shape in range(1, sop.SOP_PASS_SHAPES):
        out = run_shape(w, shape, shape, n_steps)
        assert torch.equal(out, ref), f"shape {shape} differs from the default shape"


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotune_keeps_the_state_and_matches_the_oracle(dtype):
    w = gc.random_workload((512, 384), 1, seed=91, n_steps=6, dt=0.01, field_scale=0.05)
    prop = sop.Propagator(w.dims, w.spacing, 1, dtype)
    prop.set_state(torch.from_numpy(w.psi0))
    prop.set_potential(w.V)
    before = prop.state.clone()
    chosen = prop.autotune(w.dt, 4)
    assert all(0 <= c < sop.SOP_PASS_SHAPES for c in chosen)
    assert torch.equal(prop.state, before)
    # cached for the shape: a second plan takes the same choice without timing
    prop2 = sop.Propagator(w.dims, w.spacing, 1, dtype)
    prop2.set_state(torch.from_numpy(w.psi0))
    assert prop2.autotune(w.dt, 4) == chosen
    prop2.close()
    prop.step(w.n_steps, w.dt, w.field)
    torch.cuda.synchronize()
    ref = gc.run_oracle(w)
    err = gc.relerr(prop.state.cpu().numpy(), ref)
    prop.close()
    assert err < (gc.TOL_F64 if dtype == "c128" else gc.TOL_F32_SHORT), err


def test_autotune_cache_file_is_read_and_appended(tmp_path, monkeypatch):
    """SOP_AUTOTUNE_CACHE: a line for this device model and lattice shape is
    taken without timing; a shape tuned afresh is appended to the file."""
    model = torch.cuda.get_device_name(0).replace(" ", "_")
    path = tmp_path / "shapes.txt"
    # 2D 192 x 96 complex64 (sides no other test tunes) -> shapes 3 and 5;
    # a complex128 line with shapes other than 0 is ignored, so are malformed
    # lines and other models' lines
    path.write_text(f"a malformed line\n{model} 2 192 96 1 1 0 3 5\n{model} 2 192 96 1 1 1 4 4\n"
                    f"other_gpu 2 96 192 1 1 0 2 2\n")
    monkeypatch.setenv("SOP_AUTOTUNE_CACHE", str(path))
    w = gc.random_workload((192, 96), 1, seed=5, n_steps=2, dt=0.01, field_scale=0.05)
    prop = sop.Propagator(w.dims, w.spacing, 1, "c64")
    prop.set_state(torch.from_numpy(w.psi0))
    assert prop.autotune(w.dt, 2) == [3, 5]
    prop.close()
    prop = sop.Propagator(w.dims, w.spacing, 1, "c128")
    prop.set_state(torch.from_numpy(w.psi0))
    assert prop.autotune(w.dt, 2) == [0, 0]   # tuned: the bad line was not taken
    prop.close()
    w2 = gc.random_workload((96, 192), 1, seed=6, n_steps=2, dt=0.01, field_scale=0.05)
    prop = sop.Propagator(w2.dims, w2.spacing, 1, "c64")
    prop.set_state(torch.from_numpy(w2.psi0))
    chosen = prop.autotune(w2.dt, 2)
    prop.close()
    lines = path.read_text().split("\n")
    assert f"{model} 2 96 192 1 1 0 {chosen[0]} {chosen[1]}" in lines
    assert f"{model} 2 192 96 1 1 1 0 0" in lines
