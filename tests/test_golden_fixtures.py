"""The stored full-size oracle fixtures (tests/golden/fullsize_*.npz, written
by tests/golden/make_fullsize.py from the oracle and the seeded generators)
still belong to the generators' inputs: lattice, step count, dt and
checksums of psi_0, V and the field match, and the sample indices are valid.
CPU only; the 512^3 configuration is left to its GPU test (its inputs alone
take 2 GB)."""
import os

import numpy as np
import pytest

from paper_1012_3911_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

CASES = {
    "config2": wl.config2,
    "config4": wl.config4,
    "dirac3d": wl.dirac3d_packet,
    "pulse": wl.dirac_pulse,
    "velocity": wl.velocity_gauge_benchmark,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fixture_matches_its_inputs(name):
    path = os.path.join(GOLDEN, f"fullsize_{name}.npz")
    if not os.path.exists(path):
        pytest.fail(f"{path} is missing: run tests/golden/make_fullsize.py")
    g = np.load(path)
    w = CASES[name]()
    assert tuple(g["dims"]) == w.dims and int(g["n_steps"]) == w.n_steps and float(g["dt"]) == w.dt
    assert int(g["comps"]) == w.comps
    assert abs(float(g["psi0_abs2"]) - float(np.sum(np.abs(w.psi0) ** 2))) <= 1e-9 * float(g["psi0_abs2"])
    assert abs(float(g["V_sum"]) - float(w.V.sum())) <= 1e-9 * abs(float(g["V_sum"]))
    fs = float(np.asarray(w.field).sum())
    assert abs(float(g["field_sum"]) - fs) <= 1e-9 * max(1.0, abs(float(g["field_sum"])))
    idx = g["idx"]
    assert idx.ndim == 1 and idx.size >= 8192 and np.all(np.diff(idx) > 0)
    assert idx[0] >= 0 and idx[-1] < w.comps * w.npoints
    vals = g["values"]
    assert vals.shape == idx.shape and np.all(np.isfinite(vals))
    # a unitary scheme: the oracle's final norm stays that of psi_0 (Eq. 8)
    norm0 = float(g["psi0_abs2"]) * float(np.prod(w.spacing))
    assert abs(float(g["norm"]) - norm0) < 1e-6 * norm0
