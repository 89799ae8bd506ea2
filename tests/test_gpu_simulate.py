"""GPU parity of materialised paths (mc_simulate) with the oracle, path by
path, on tiny and ragged path counts (brute force) and on the d = 64 basket."""
import numpy as np
import pytest

import workloads
from gpu_util import BAND, cfg_of, gbm_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


@pytest.mark.parametrize("paths", [1, 2, 3, 7, 32, 1000])
@pytest.mark.parametrize("scheme", ["log_euler", "euler"])
def test_gbm1d_paths_brute_force(gb, orc, paths, scheme):
    w = workloads.gbm_1d(paths=paths, steps=65)
    got = gb.simulate(gbm_model(w), cfg_of(w, scheme=scheme, path_offset=11), save_every=5).cpu().numpy()
    ref = orc.gbm_paths(w["s0"], w["sigma"], w["r"], w["T"], 65, paths, scheme=scheme, save_every=5,
                        path_offset=11)
    assert got.shape == ref.shape
    assert rel_err(got, ref) <= BAND


@pytest.mark.parametrize("d,scheme", [(3, "log_euler"), (12, "euler"), (64, "log_euler")])
def test_basket_paths(gb, orc, d, scheme):
    s0, sg, corr = workloads.basket_market(d, 3, seed=9)
    model = dict(kind="gbm", s0=s0, sigma=sg, corr=corr, r=0.05)
    got = gb.simulate(model, dict(steps=36, T=1.0, paths=129, scheme=scheme), save_every=6).cpu().numpy()
    ref = orc.gbm_paths(s0, sg, 0.05, 1.0, 36, 129, corr=corr, scheme=scheme, save_every=6)
    assert got.shape == ref.shape
    assert rel_err(got, ref) <= BAND


def test_basket_d64_config_paths(gb, orc):
    w = workloads.basket_d64(paths=64)
    got = gb.simulate(gbm_model(w), cfg_of(w), save_every=63).cpu().numpy()
    ref = orc.gbm_paths(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], 64, corr=w["corr"], save_every=63)
    assert rel_err(got, ref) <= BAND


@pytest.mark.parametrize("paths", [1, 5, 300])
def test_heston_paths(gb, orc, paths):
    m = dict(workloads.HESTON_PARAMS)
    got = gb.simulate(dict(kind="heston", **m), dict(steps=64, T=1.0, paths=paths), save_every=8).cpu().numpy()
    ref = orc.heston_paths(m, 1.0, 64, paths, save_every=8)
    assert rel_err(got[:, 0], ref[:, 0]) <= BAND
    # the variance is O(0.04) and crosses zero: compare on an absolute scale
    assert np.max(np.abs(got[:, 1] - ref[:, 1])) <= BAND * 0.04 * 10


def test_normals_within_error_model(gb, orc):
    """The kernels' normals against the oracle's, read through the 1-D Euler
    path with r = 0 and sigma sqrt(dt) = 1: each step is the single rounding
    S_{i+1} = fl(S_i + S_i z_i), so (S_{i+1} - S_i) / S_i recovers the GPU's
    z_i to within 2^-24 |S_{i+1} / S_i|.  2^18 paths x 8 steps cover all four
    lanes of two Philox blocks per path; every normal lies within
    normal_error_bound, the window that the reduced-precision emulation tests
    grant each normal, plus that resolution."""
    from test_gpu_tc import normal_error_bound
    N, M = 1 << 18, 8
    model = dict(kind="gbm", s0=[1.0], sigma=[1.0], r=0.0)
    cfg = dict(steps=M, T=float(M), paths=N, scheme="euler", seed=42)
    S = gb.simulate(model, cfg, save_every=1)[:, 0].double().cpu().numpy()          # [M + 1, N]
    So = orc.gbm_paths([1.0], [1.0], 0.0, float(M), M, N, scheme="euler", seed=42)[:, 0]
    zg = (S[1:] - S[:-1]) / S[:-1]
    zo = So[1:] / So[:-1] - 1.0
    res = 2.0 ** -24 * np.abs(S[1:] / S[:-1]) * 1.01
    eps = normal_error_bound(zo.T).T
    err = np.abs(zg - zo)
    r = np.hypot(zo[0::2], zo[1::2]).repeat(2, axis=0)
    for lo, hi in [(0, 0.01), (0.01, 0.5), (0.5, 2), (2, 4), (4, 6)]:
        m = (r >= lo) & (r < hi)
        if m.any():
            print(f"r in [{lo}, {hi}): {m.sum():8d} normals, max |err| {err[m].max():.2e}, "
                  f"max |err| / bound {np.max((err / (eps + res))[m]):.3f}")
    assert np.all(err <= eps + res), np.max(err / (eps + res))


@pytest.mark.parametrize("kind", ["gbm1d", "basket8", "basket64", "heston"])
def test_launch_configuration_invariance(gb, kind):
    """Each path depends only on its stream index: a window of paths run on
    its own (a smaller persistent grid, so every path lands on another
    thread, block and paths-per-thread count) equals the same window of a
    larger run bit for bit, and so does a run split at an odd offset."""
    if kind == "heston":
        model, steps = dict(kind="heston", **workloads.HESTON_PARAMS), 32
    elif kind == "gbm1d":
        w = workloads.gbm_1d(paths=1, steps=48)
        model, steps = gbm_model(w), 48
    else:
        d = 8 if kind == "basket8" else 64
        s0, sg, corr = workloads.basket_market(d, 3, seed=9)
        model, steps = dict(kind="gbm", s0=s0, sigma=sg, corr=corr, r=0.05), 24
    N, off, n = 1 << 17, 40_961, 3001
    big = gb.simulate(model, dict(steps=steps, T=1.0, paths=N), save_every=steps // 4).cpu().numpy()
    win = gb.simulate(model, dict(steps=steps, T=1.0, paths=n, path_offset=off), save_every=steps // 4).cpu().numpy()
    assert np.array_equal(win, big[..., off:off + n])
    a = gb.simulate(model, dict(steps=steps, T=1.0, paths=777), save_every=steps // 4).cpu().numpy()
    b = gb.simulate(model, dict(steps=steps, T=1.0, paths=N - 777, path_offset=777), save_every=steps // 4).cpu().numpy()
    assert np.array_equal(np.concatenate([a, b], axis=-1), big)
