"""The launch-shape autotuner (HBS_AUTOTUNE=1): it times every candidate of the tuned launches
(the per-node inversion: persistent Gauss-Jordan or blocked Gauss-Jordan on clusters of 1, 2,
4 or 8 CTAs; the Schur factorization's CTAs per group) on the live problem, keeps the fastest,
writes its choices to HBS_TUNE_FILE, and every variant gives the same Bragg amplitudes as the
default launches to rounding."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import require_lib

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from paper_1301_1247_gb300 import hbs, inputs
x, y, dx, dy = inputs.wiggly(0, 0.35, 20, 0.03).sample(6000)
th = inputs.bloch_grouped_angles(3, 30.0, 1.0, 40, 3).ravel()
out = []
for _ in range(int(sys.argv[3])):
    h = hbs.Handle(x, y, dx, dy, 1.0, 30.0, 1e-12, hbs.default_options(precision=1))
    r = h.solve(th)
    out.append(np.concatenate([np.concatenate(r.bragg(i)[1:3]) for i in range(len(th))]))
np.save(sys.argv[1], np.array(out))
"""


def _run(tmp_path, tag, env_extra, reps):
    out = tmp_path / f"{tag}.npy"
    env = dict(os.environ, **env_extra)
    subprocess.run([sys.executable, "-c", CODE, str(out), ROOT, str(reps)], check=True, env=env, timeout=600)
    return np.load(out)


def test_autotuner_explores_persists_and_keeps_results(tmp_path):
    require_lib()
    tune = tmp_path / "tune.txt"
    base = _run(tmp_path, "base", {"HBS_AUTOTUNE": "0", "HBS_TUNE_FILE": ""}, 1)[0]
    tuned = _run(tmp_path, "tuned", {"HBS_AUTOTUNE": "1", "HBS_TUNE_FILE": str(tune)}, 5)
    keys = {}
    for line in tune.read_text().splitlines():
        k, v, ms = line.split()
        keys[k] = (int(v), float(ms))
    assert any(k.startswith("inverse/") for k in keys) and any(k.startswith("schur/") for k in keys), keys
    assert all(ms > 0 for _, ms in keys.values())
    for row in tuned:  # exploring builds (each a different shape) and the tuned ones
        assert np.linalg.norm(row - base) / np.linalg.norm(base) < 1e-11
    # a new process with tuning off starts from the stored choices
    again = _run(tmp_path, "again", {"HBS_AUTOTUNE": "0", "HBS_TUNE_FILE": str(tune)}, 1)[0]
    assert np.linalg.norm(again - base) / np.linalg.norm(base) < 1e-11
