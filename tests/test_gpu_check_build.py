"""The check build (-DSOP_CHECK=1: every pass kernel tests its global
indices against the lattice, its shared-memory offsets against the tile
buffer and every TMA x coordinate for 16-byte alignment, and each device
buffer carries canary bytes) runs one case of every pass kind -- 2D and 3D
Schroedinger in both dtypes and several launch shapes, Dirac pairs, the
four-component 3D Dirac passes, the per-column pulse mixing, multi-instance
batch passes and the adjoint -- with no failed test, no overwritten canary,
and final states bit-identical to the normal build's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import gpu_cases as gc

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
WORKER = os.path.join(HERE, "check_build_worker.py")


def _worker(env, path):
    r = subprocess.run([sys.executable, WORKER, str(path)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_check_build_passes_and_matches_the_normal_build(tmp_path):
    gc.require_gpu()
    env_check = dict(os.environ, SOP_CHECK="1")
    env_norm = {k: v for k, v in os.environ.items() if k != "SOP_CHECK"}
    b = subprocess.run([sys.executable, "-c", "from paper_1012_3911_gb300 import build; build.build()"], cwd=ROOT,
                       env=env_check, capture_output=True, text=True, timeout=1200)
    assert b.returncode == 0, b.stderr[-3000:]
    info = _worker(env_check, tmp_path / "check.npz")
    assert info["canaries_bad"] == 0, info
    info_n = _worker(env_norm, tmp_path / "normal.npz")
    assert info_n["canaries_bad"] == -1   # the normal build has no canaries
    a = np.load(tmp_path / "check.npz")
    n = np.load(tmp_path / "normal.npz")
    assert sorted(a.files) == sorted(n.files)
    for k in n.files:
        assert np.array_equal(a[k], n[k]), k
