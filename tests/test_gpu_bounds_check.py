"""Bounds-checked build: the small parity cases of every kernel family, run on
libac_check.so (built with -DAC_CHECK: every index the kernels compute is checked, a
violation is recorded and reported as AC_ERR_STATE, never trapped) in a subprocess, must be
bit-exact against the oracle with no violation reported.  compute-sanitizer is not used on
this hardware; this build stands in for its memcheck of the kernels' own indices."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build_runs_every_kernel_family_exactly():
    lib = os.path.join(ROOT, "paper_cs_0502039_gb300", "libac_check.so")
    assert os.path.exists(lib), "libac_check.so is built by __graft_entry__.build()"
    env = dict(os.environ, AC_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-m", "tests.bounds_check_cases"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "batch, transfers, static entry ok" in r.stdout
