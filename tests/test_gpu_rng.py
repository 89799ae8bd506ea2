"""The GPU's random stream against the FP64 oracle's, through the C ABI
(Sec. IV.A: Philox4x32-10; Sec. VI.D: Box-Muller): the raw 32-bit words of
mc_philox_words bit for bit, for keys with both words in use, stream indices
and block counters above 2^32 (and across the 2^32 boundary of the counter's
low word), and the normals of mc_normals within the SFU error window."""
import numpy as np
import pytest

from test_gpu_tc import normal_error_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


@pytest.mark.parametrize("seed", [42, (7 << 32) | 0x1234, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("stream_index", [0, 12345, (1 << 32) + 7, (1 << 56) + 3, (5 << 56) + (1 << 40) + 9])
@pytest.mark.parametrize("q0", [0, (1 << 32) - 300, (1 << 40) + 17])
def test_philox_words_bit_exact(gb, orc, seed, stream_index, q0):
    n = 601  # a ragged count (not a multiple of the 256-thread block)
    got = gb.philox_words(seed, stream_index, q0, n).cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n):
        q = q0 + i
        want = orc.philox([q & 0xFFFFFFFF, q >> 32, stream_index & 0xFFFFFFFF, stream_index >> 32], key)
        assert np.array_equal(got[i], want), (i, got[i], want)


def test_philox_words_large_launch_matches_sampled_oracle(gb, orc):
    """A launch of 2^22 blocks (a grid-stride loop over many waves): 4096
    sampled blocks bit for bit, and every word's byte histogram near uniform."""
    n, seed, s = 1 << 22, 42, (1 << 33) + 5
    got = gb.philox_words(seed, s, (1 << 32) - 1000, n).cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(0)
    for i in rng.choice(n, 4096, replace=False):
        q = (1 << 32) - 1000 + int(i)
        want = orc.philox([q & 0xFFFFFFFF, q >> 32, s & 0xFFFFFFFF, s >> 32], [seed, 0])
        assert np.array_equal(got[i], want), i
    top = np.bincount((got.ravel() >> 24).astype(np.int64), minlength=256)
    exp = got.size / 256
    chi2 = float(((top - exp) ** 2 / exp).sum())
    assert chi2 < 255 + 6 * np.sqrt(2 * 255), chi2  # 255 degrees of freedom, ~6 sigma


@pytest.mark.parametrize("stream_index,j0,count", [(0, 0, 1 << 20), ((1 << 32) + 5, (1 << 33) + 1, 100003),
                                                   ((2 << 56) + 77, 3, 1)])
def test_normals_against_oracle(gb, orc, stream_index, j0, count):
    got = gb.normals(42, stream_index, j0, count).double().cpu().numpy()
    want = orc.normals(42, stream_index, j0, count)
    # the window pairs lanes (2m, 2m + 1) of one block: align to the block start
    pad = j0 % 2
    zf = np.concatenate([orc.normals(42, stream_index, j0 - pad, pad), want,
                         orc.normals(42, stream_index, j0 + count, (pad + count) % 2)])[None, :]
    eps = normal_error_bound(zf)[0, pad:pad + count]
    err = np.abs(got - want)
    assert np.all(err <= eps), float(np.max(err / eps))
    assert float(np.max(err)) < 1e-3
