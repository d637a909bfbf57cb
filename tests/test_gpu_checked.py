"""GPU test of the bounds-checked build (tests/checked_paths.py in a fresh
process with VECKM_LIBRARY=checked): the main paths (embeddings, the plain
and tensor-core heads for D = 64 and 128, explicit requests, a stream, a
batch, the direct window form) agree with the FP64 oracle, and no index that
a kernel derived from data would have left its buffer."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_the_main_paths_without_a_bad_index():
    env = dict(os.environ, VECKM_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_paths.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("CHECKS ")]
    assert line, r.stdout[-2000:]
    _, n, where = line[-1].split()
    assert int(n) == 0, f"{n} out-of-buffer indices, the first at {where}"
