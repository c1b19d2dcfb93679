"""The parity matrix once more on the debug build of the library (libaerafold_debug.so, built by
__graft_entry__.build() with AR_DEBUG_BOUNDS): every station, walk, spectrum, output, corner
slab and frequency-cell index of the kernels is checked on the device, and a failed check sets
an error bit that ar_sync turns into AR_ERR_DEVICE (the access is skipped, nothing traps). The
tests below call ar_sync after their launches, so they fail on any such bit; the guard bands
around every output (tests/guard_util.py) stay on. A stand-in for a memory checker, which this
GPU pool does not offer.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG_LIB = os.path.join(ROOT, "paper_1507_07733_gb300", "lib", "libaerafold_debug.so")
MATRIX = ["tests/test_gpu_parity.py", "tests/test_gpu_patterns.py", "tests/test_gpu_batch.py",
          "tests/test_gpu_peak_fine.py", "tests/test_gpu_snr.py", "tests/test_gpu_reconstruct.py"]


def test_parity_matrix_on_the_debug_build():
    if not os.path.exists(DEBUG_LIB):
        pytest.fail(f"{DEBUG_LIB} not built: run __graft_entry__.build()")
    env = dict(os.environ, AERAFOLD_LIB=DEBUG_LIB)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *MATRIX],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-25:])
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
