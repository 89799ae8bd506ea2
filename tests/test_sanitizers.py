"""Host-side memory and undefined-behaviour checks with the compilers'
sanitizers (AddressSanitizer + UndefinedBehaviorSanitizer), standing in on
the host for a device sanitizer:
  * the FP64 oracle built with both sanitizers runs its own pin tests;
  * the library's host code (argument checks, marshalling, the moments and
    combination of sharded runs) built with both sanitizers runs the ABI
    tests, which need no device.
Each run is a child process with the sanitizer runtimes preloaded; a report
from either sanitizer fails the test."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.slow

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtimes():
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            pytest.skip(f"{name} not available")
        libs.append(p)
    return ":".join(libs)


def _run(args, env_extra):
    env = dict(os.environ, LD_PRELOAD=_runtimes(), ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", **env_extra)
    r = subprocess.run([sys.executable, "-m", "pytest", *args, "-q", "-x", "-p", "no:cacheprovider",
                        "-m", "not gpu and not slow"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    out = r.stdout + r.stderr
    assert "ERROR: AddressSanitizer" not in out, out[-4000:]
    assert "runtime error:" not in out, out[-4000:]
    assert r.returncode == 0, out[-4000:]
    return out


def test_oracle_under_address_and_ub_sanitizers():
    import oracle  # noqa: F401  (the sanitizer build is made by the child)
    env = {"GBMC_ORACLE_SANITIZE": "1", "OMP_NUM_THREADS": "4"}
    subprocess.run([sys.executable, "-c", "import oracle; oracle.build()"], cwd=ROOT, env=dict(os.environ, **env),
                   check=True)
    tests = sorted(f"tests/{f}" for f in os.listdir(os.path.join(ROOT, "tests"))
                   if f.startswith("test_oracle_") and f.endswith(".py"))
    out = _run(tests, env)
    assert "passed" in out


def test_library_host_code_under_address_and_ub_sanitizers():
    from paper_1906_02818_gb300 import build
    lib = build.build(sanitize=True)
    out = _run(["tests/test_abi.py", "tests/test_shard_gloo.py::test_moments_and_combine_through_the_library"],
               {"GBMC_LIBRARY": lib})
    assert "passed" in out
