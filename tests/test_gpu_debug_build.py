"""The debug build's bounds checks (GBMC_DEBUG; mc_debug_status).  The
device sanitizer is closed on this machine, so the library has a build whose
kernels check the index of every access to a caller buffer or checkpoint
against the buffer's extent, skip an access outside it and record it
without trapping.  A child process loads that build (GBMC_LIBRARY) and runs
GPU tests that materialise paths of every model, run the Heston adjoint
with checkpoints, evaluate the network, draw labels and write the random
stream; afterwards no access may have been skipped.  The release build
reports that it has no checks."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, sys
import pytest
rc = pytest.main(sys.argv[1:])
from paper_1906_02818_gb300 import native
L = native.lib()
v, site, idx = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
st = L.mc_debug_status(ctypes.byref(v), ctypes.byref(site), ctypes.byref(idx))
print(f"DEBUG-STATUS rc={st} violations={v.value} site={site.value} index={idx.value}", flush=True)
sys.exit(rc if rc else (0 if st == 0 and v.value == 0 else 3))
"""


def test_release_build_has_no_checks():
    import ctypes
    from paper_1906_02818_gb300 import native
    L = native.lib()
    v, s, i = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
    assert L.mc_debug_status(ctypes.byref(v), ctypes.byref(s), ctypes.byref(i)) == native.MC_EUNSUPPORTED


def test_gpu_tests_under_the_bounds_checked_build():
    from paper_1906_02818_gb300 import build
    lib = build.build(debug=True)
    tests = ["tests/test_gpu_simulate.py", "tests/test_gpu_greeks.py", "tests/test_gpu_rng.py",
             "tests/test_gpu_mlp.py::test_forward_bf16_matches_emulation",
             "tests/test_gpu_risk.py::test_labels_match_oracle", "tests/test_gpu_risk.py::test_label_greeks_match_oracle"]
    env = dict(os.environ, GBMC_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, *tests, "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    out = r.stdout + r.stderr
    print(out[-1500:])
    assert "DEBUG-STATUS rc=0 violations=0" in out, out[-3000:]
    assert r.returncode == 0, out[-3000:]
