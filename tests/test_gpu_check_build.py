"""The bounded-index debug build (libfdph_check.so, -DFDPH_CHECK) on the small parity cases.

In that build every ring, state, partial-sum and near-slice index of the step kernels is checked
against the extent of its array (a failure records an error word that the next synchronising call
reports as FDPH_E_CHECK; the access is skipped, no trap), and every plan allocation ends in a
canary compared on each synchronisation.  The parity tests of the FP64, FP32 and FP16 paths
(tensor cores included) run in a child process that loads the checked library: they must pass
unchanged, i.e. no check fires and the results still match the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_parity_cases_pass_under_index_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build
    build.build(check=True)
    env = dict(os.environ, FDPH_LIB="check")
    which = subprocess.run([sys.executable, "-c", "from paper_1903_02118_gb300 import fdph; fdph.lib(); print(fdph.LIB_PATH)"],
                           env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert which.returncode == 0 and which.stdout.strip().endswith("libfdph_check.so"), which.stdout + which.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
                        "tests/test_gpu_parity.py", "tests/test_gpu_tensor_cores.py", "tests/test_gpu_batch.py",
                        "-k", "not full_size"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
