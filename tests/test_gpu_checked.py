"""The bounds-checked build (libhram_checked.so, -DHRAM_CHECKED): every
cell-list row, candidate range, sort slot, padded predicate read and ghost
index is checked before use, and a failed check makes the case's status
HR_ECHECK instead of touching memory out of range.  The parity cases run
against that build in a child process (impact, perturbed and closed-box
neighbour sets, a shuffled upload over several scan tiles, the disk rings
with particles inside the disk, stencil rows over 32 candidates, the probe
window, a batch, and the tangent and adjoint sweeps); every check must hold
(any HR_ECHECK raises in the binding and fails the case)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_cases_pass_every_bounds_check():
    from paper_2609_05494_b300 import build
    build.build()
    env = dict(os.environ, HRAM_CHECKED="1")
    cases = ["tests/test_gpu_parity.py", "-k", "not all_wall_probes",
             "tests/test_gpu_batch.py::test_batch_equals_cases_run_alone",
             "tests/test_gpu_adjoint.py::test_adjoint_equals_tangent"]
    probe = subprocess.run([sys.executable, "-c",
                            "from paper_2609_05494_b300 import _lib; print(_lib.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert probe.stdout.strip().endswith("libhram_checked.so"), probe.stdout + probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider"]
                       + cases, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    print(r.stdout[-3000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
