"""Pins of the oracle's random stream (Sec. IV.A Philox, Sec. VI.D Box-Muller).

The Philox pin runs PyTorch's own header-only Philox4x32-10 engine (an
implementation independent of the oracle's) as a compiled program and requires
bit equality over the whole counter/key space.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

TORCH_PHILOX_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cinttypes>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    try:
        import torch
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) else None


@pytest.fixture(scope="module")
def torch_philox():
    inc = _torch_include()
    if inc is None:
        pytest.skip("PyTorch's Philox header is not installed")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "p.cpp"), os.path.join(d, "p")
    with open(src, "w") as f:
        f.write(TORCH_PHILOX_PROG)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)

    def run(triples):
        inp = "\n".join(f"{a} {b} {c}" for a, b, c in triples) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(t) for t in line.split()] for line in out.strip().splitlines()], dtype=np.uint64)
    return run


def test_philox_bit_exact_vs_torch_engine(orc, torch_philox):
    rng = np.random.default_rng(7)
    triples = [(0, 0, 0), (42, 0, 0), (42, 1, 0), (42, 0, 1), (2**64 - 1, 2**64 - 1, 2**64 - 1)]
    def u64():
        return (int(rng.integers(0, 2**32)) << 32) | int(rng.integers(0, 2**32))
    for _ in range(300):
        triples.append((u64(), u64(), u64()))
    ref = torch_philox(triples)
    for (seed, sub, off), want in zip(triples, ref):
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = orc.philox(ctr, key)
        assert [int(v) for v in got] == [int(v) for v in want], (seed, sub, off)


def test_uniform_map_exact_and_open(orc):
    assert orc.uniform(0) == 2.0 ** -24
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2**32, size=2000, dtype=np.uint64):
        u = orc.uniform(int(x))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exact in binary32 as well
        assert u == ((int(x) >> 9) + 0.5) / 2**23


@pytest.mark.parametrize("seed,stream", [(42, 12345), ((7 << 40) | 42, 12345), (42, (2 << 56) | 9),
                                         ((1 << 63) | 5, (1 << 35) | 3)])
def test_box_muller_pairs(orc, seed, stream):
    """Normals 4q..4q+3 of stream s under key seed come from the block at
    counter (q lo, q hi, s lo, s hi), key (seed lo, seed hi):
    z0^2 + z1^2 = -2 ln u(x0) and atan2(z1, z0) = 2 pi u(x1) (mod 2 pi); same
    for lanes 2, 3 (both words of the key, the stream and the counter used)."""
    for q in [0, 1, 7, 1000, 2**33 + 5]:
        x = orc.philox([q & 0xFFFFFFFF, q >> 32, stream & 0xFFFFFFFF, stream >> 32],
                       [seed & 0xFFFFFFFF, seed >> 32])
        z = orc.normals(seed, stream, 4 * q, 4)
        for pair in range(2):
            ua, ub = orc.uniform(int(x[2 * pair])), orc.uniform(int(x[2 * pair + 1]))
            z0, z1 = z[2 * pair], z[2 * pair + 1]
            assert np.isclose(z0 * z0 + z1 * z1, -2.0 * np.log(ua), rtol=1e-13, atol=1e-15)
            ang = np.arctan2(z1, z0) % (2 * np.pi)
            assert np.isclose(ang, (2 * np.pi * ub) % (2 * np.pi), rtol=0, atol=1e-10)


def test_normal_moments(orc):
    """Mean 0, variance 1, skewness 0, excess kurtosis 0 within 5 standard
    errors over 2^21 draws spread over many streams."""
    z = np.concatenate([orc.normals(42, s, 0, 1 << 14) for s in range(128)])
    n = z.size
    m = z.mean()
    v = z.var()
    skew = np.mean((z - m) ** 3) / v ** 1.5
    kurt = np.mean((z - m) ** 4) / v ** 2 - 3.0
    assert abs(m) < 5 / np.sqrt(n)
    assert abs(v - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(skew) < 5 * np.sqrt(6.0 / n)
    assert abs(kurt) < 5 * np.sqrt(24.0 / n)
    assert np.max(np.abs(z)) <= np.sqrt(-2 * np.log(2.0 ** -24)) + 1e-12


def test_streams_are_uncorrelated(orc):
    a = orc.normals(42, 0, 0, 1 << 16)
    b = orc.normals(42, 1, 0, 1 << 16)
    c = orc.normals(43, 0, 0, 1 << 16)
    for x, y in [(a, b), (a, c), (a[:-1], a[1:])]:
        assert abs(np.corrcoef(x, y)[0, 1]) < 5 / np.sqrt(x.size)


def test_uniform_equidistribution(orc):
    """Chi-square over 256 bins of the 2^16 uniforms of 2^14 Philox blocks."""
    u = []
    for q in range(1 << 8):
        for s in range(64):
            u.extend(orc.uniform(int(w)) for w in orc.philox([q, 0, s, 0], [42, 0]))
    u = np.array(u)
    counts, _ = np.histogram(u, bins=256, range=(0.0, 1.0))
    e = u.size / 256
    chi2 = np.sum((counts - e) ** 2 / e)
    # 255 degrees of freedom: mean 255, sd ~22.6; 5-sigma band
    assert 255 - 5 * 22.6 < chi2 < 255 + 5 * 22.6
