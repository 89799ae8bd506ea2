"""The oracle and the CUDA path share no code, and the product has no CPU
fallback: the package and its kernels never import, include, link or load
anything under oracle/; the oracle never reaches into the package; the input
generators import neither; a call without the CUDA library raises instead
of computing."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1906_02818_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_product_never_reaches_the_oracle():
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        text = open(path, errors="replace").read()
        assert not re.search(r"\boracle\b|liboracle|orc_", text), path
    for path in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in open(path).read(), path


def test_oracle_never_reaches_the_product():
    for path in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(path).read()
        assert not re.search(r"paper_1906_02818_gb300|libgbmc|mc\.h|csrc|\bgbmc\b", text), path


def test_input_generators_import_neither():
    text = open(os.path.join(ROOT, "workloads.py")).read()
    imports = re.findall(r"^\s*(?:from|import)\s+([\w.]+)", text, flags=re.M)
    assert not any(m.split(".")[0] in ("oracle", "paper_1906_02818_gb300") for m in imports), imports


def test_missing_library_raises_instead_of_computing():
    """With the library pointed at a file that does not exist, importing the
    package works (it loads no CUDA) and the first call raises; the oracle is
    never imported."""
    code = ("import sys\n"
            "import paper_1906_02818_gb300 as gb\n"
            "try:\n"
            "    gb.price(dict(kind='gbm', s0=[100.0], sigma=[0.2], r=0.05), dict(steps=4, T=1.0, paths=16),\n"
            "             [dict(kind='call', strike=100.0)])\n"
            "except (ImportError, OSError) as e:\n"
            "    print('raised', type(e).__name__)\n"
            "print('oracle loaded' if 'oracle' in sys.modules else 'oracle absent')\n")
    env = dict(os.environ, GBMC_LIBRARY=os.path.join(ROOT, "no_such_dir", "libgbmc.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "raised" in r.stdout and "oracle absent" in r.stdout, r.stdout

