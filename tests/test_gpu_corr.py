"""GPU parity of the correlation sensitivities (mc_corr_greeks; Sec. I.A.3,
Sec. VI.A.2): the reverse-mode kernel path (FP32 paths, FP64 Cholesky
adjoint) against the oracle's forward-mode tangents on identical streams, per
entry of dP/dLrho and dP/dcorr; the batch-means standard errors against the
oracle's per-path standard errors; and, at the d = 64 workload's full size,
the identity that ties dP/dLrho to the basket delta and vega of mc_greeks on
the same paths.

Tolerance per entry: 2e-5 of the mean absolute per-path contribution (FP32
normals and sums against FP64), plus the contribution of the paths whose
basket lies within the FP32 band 2e-5 K of the strike (their payoff slope may
legitimately differ)."""
import numpy as np
import pytest

import workloads
from gpu_util import BAND, REL, cfg_of, gbm_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _market(d, k=3, seed=13):
    s0, sg, corr = workloads.basket_market(d, k, seed=seed)
    w = np.full(d, 1.0 / d)
    return dict(s0=s0, sigma=sg, corr=corr, weights=w, r=0.05, T=1.0, seed=42, steps=1, paths=1)


def _check_entries(got, per_path, U, K, label):
    """got [d, d, 2] (mean, se); per_path [d, d, N] from the oracle."""
    band = np.abs(U - K) <= BAND * K
    N = per_path.shape[-1]
    mean = per_path.mean(axis=-1)
    scale = np.abs(per_path).mean(axis=-1)
    flips = np.abs(per_path[..., band]).sum(axis=-1) / N
    err = np.abs(got[..., 0] - mean)
    tol = 2e-5 * scale + flips + 1e-12
    bad = np.argwhere(err > tol)
    assert bad.size == 0, (label, bad[:5], err[tuple(bad[0])], tol[tuple(bad[0])], int(band.sum()))
    return mean


def _check_se(got, per_path, label):
    """Batch-means SE against the oracle's per-path SE: median ratio near 1,
    every ratio within the range of a chi distribution with >= 20 degrees of
    freedom."""
    N = per_path.shape[-1]
    d = per_path.shape[0]
    mask = per_path.std(axis=-1) > 0
    mask &= ~np.eye(d, dtype=bool) if label == "drho" else np.tril(np.ones((d, d), dtype=bool))
    se_ref = per_path.std(axis=-1, ddof=1)[mask] / np.sqrt(N)
    ratio = got[..., 1][mask] / se_ref
    assert 0.8 <= np.median(ratio) <= 1.2, (label, np.median(ratio))
    assert ratio.min() >= 0.3 and ratio.max() <= 2.5, (label, ratio.min(), ratio.max())


@pytest.mark.parametrize("d,paths,steps", [(4, 3000, 12), (7, 2900, 9), (64, 2600, 16)])
@pytest.mark.parametrize("kind", ["call", "put"])
def test_corr_greeks_match_oracle(gb, orc, d, paths, steps, kind):
    """d = 4 (whole Philox blocks per step), d = 7 (blocks straddle steps),
    d = 64 (the basket workload's width); >= 20 tiles of 128 paths with a
    ragged last tile."""
    w = _market(d)
    K = float(w["weights"] @ w["s0"]) * (1.0 if kind == "call" else 1.03)
    pay = dict(kind=kind, strike=K)
    (p, pse), dl, dr = gb.corr_greeks(gbm_model(w), cfg_of(w, paths=paths, steps=steps), pay)
    ref = orc.gbm_corr_greeks(w["s0"], w["sigma"], w["corr"], w["r"], w["T"], steps, paths, pay,
                              weights=w["weights"])
    m, se = orc.mean_se(ref["f"])
    assert abs(p - m) <= REL * abs(m), (p, m)
    assert abs(pse - se) <= 1e-3 * se
    _check_entries(dl, ref["dl"], ref["U"], K, "dl")
    _check_entries(dr, ref["drho"], ref["U"], K, "drho")
    assert np.all(dl[..., 0][np.triu_indices(d, 1)] == 0.0)
    assert np.all(dr[..., 0][np.arange(d), np.arange(d)] == 0.0)
    assert np.allclose(dr[..., 0], dr[..., 0].T, rtol=0, atol=1e-12 * np.abs(dr[..., 0]).max())
    _check_se(dl, ref["dl"], "dl")
    _check_se(dr, ref["drho"], "drho")


def test_corr_greeks_edge_cases(gb, orc):
    """Two assets; identity correlation (corr omitted); one tile (<= 128
    paths: one batch, so NaN standard errors for the sensitivities); a path
    offset."""
    w = _market(2)
    K = float(w["weights"] @ w["s0"])
    pay = dict(kind="call", strike=K)
    for corr, paths, off in [(w["corr"], 1000, 0), (None, 700, 12345), (w["corr"], 100, 7)]:
        ww = dict(w, corr=corr)
        (p, _), dl, dr = gb.corr_greeks(gbm_model(ww), cfg_of(ww, paths=paths, steps=6, path_offset=off), pay)
        ref = orc.gbm_corr_greeks(w["s0"], w["sigma"], corr if corr is not None else np.eye(2), w["r"], w["T"], 6,
                                  paths, pay, weights=w["weights"], path_offset=off)
        assert abs(p - ref["f"].mean()) <= REL * abs(ref["f"].mean())
        _check_entries(dl, ref["dl"], ref["U"], K, "dl")
        _check_entries(dr, ref["drho"], ref["U"], K, "drho")
        if paths <= 128:
            assert np.all(np.isnan(dl[..., 1])) and np.all(np.isnan(dr[..., 1]))


def test_corr_greeks_d64_full_shape(gb):
    """The d = 64 workload (2^18 paths, 252 steps, ATM basket call) in full:
    the price equals mc_price's on the same stream, and per path
    sum_b Lrho[a][b] dP/dLrho[a][b] = sigma_a vega_a + sigma_a^2 T S0_a delta_a
    (the diffusion part of vega), so the same holds for the means returned by
    mc_corr_greeks and mc_greeks (both FP32, different kernels)."""
    w = workloads.basket_d64()
    pay = w["payoffs"][0]
    (p, pse), dl, dr = gb.corr_greeks(gbm_model(w), cfg_of(w), pay)
    ref = gb.price(gbm_model(w), cfg_of(w), [pay])
    assert abs(p - ref[0][0]) <= 2 * REL * abs(ref[0][0]), (p, ref)
    _, g = gb.greeks(gbm_model(w), cfg_of(w), [pay])
    d = 64
    delta, vega = g[0, :d, 0], g[0, d:2 * d, 0]
    L = np.linalg.cholesky(w["corr"])
    lhs = (L * dl[..., 0]).sum(axis=1)
    rhs = w["sigma"] * vega + w["sigma"] ** 2 * w["T"] * w["s0"] * delta
    scale = np.abs(rhs).max()
    assert np.max(np.abs(lhs - rhs)) <= 1e-4 * scale, np.max(np.abs(lhs - rhs)) / scale
    # the call gains from correlation (a larger basket variance) on average
    off = dr[..., 0][~np.eye(d, dtype=bool)]
    assert off.mean() > 0
    assert np.all(np.isfinite(dr[..., 1]))


def test_basket_pricer_autograd(gb, orc):
    """BasketPricer: autograd through a parametrised correlation
    corr(theta) = (1 - theta) corr0 + theta 11^T and the spot and volatility
    vectors; the gradients against the oracle's forward-mode sensitivities of
    the same paths (delta, vega, rho; d/dtheta = sum over pairs of
    dP/dcorr[a][b] (1 - corr0[a][b]))."""
    import torch
    d, paths, steps = 6, 4000, 10
    w = _market(d)
    K = float(w["weights"] @ w["s0"])
    pay = dict(kind="call", strike=K)
    theta = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    c0 = torch.tensor(w["corr"])
    corr = (1 - theta) * c0 + theta * torch.ones(d, d, dtype=torch.float64)
    s0 = torch.tensor(w["s0"], requires_grad=True)
    sg = torch.tensor(w["sigma"], requires_grad=True)
    r = torch.tensor(w["r"], dtype=torch.float64, requires_grad=True)
    cfg = cfg_of(w, paths=paths, steps=steps)
    price = gb.BasketPricer.apply(s0, sg, r, corr, cfg, pay, w["weights"])
    price.backward()
    corr_np = corr.detach().numpy()
    ref = orc.gbm_corr_greeks(w["s0"], w["sigma"], corr_np, w["r"], w["T"], steps, paths, pay, weights=w["weights"])
    gpath = orc.gbm_greeks(w["s0"], w["sigma"], w["r"], w["T"], steps, paths, [pay], corr=corr_np,
                           weights=w["weights"])[0]
    band = np.abs(ref["U"] - K) <= BAND * K

    def close(got, per_path, label):
        want = per_path.mean(axis=-1)
        tol = 2e-5 * np.abs(per_path).mean(axis=-1) + np.abs(per_path[..., band]).sum(axis=-1) / paths + 1e-12
        assert np.all(np.abs(got - want) <= tol), (label, got, want, tol)

    assert abs(price.item() - ref["f"].mean()) <= REL * ref["f"].mean()
    close(s0.grad.numpy(), gpath[:d], "s0")
    close(sg.grad.numpy(), gpath[d:2 * d], "sigma")
    close(r.grad.numpy(), gpath[2 * d], "r")
    il = np.tril_indices(d, -1)
    dth_path = (ref["drho"] * (1.0 - w["corr"])[..., None])[il].sum(axis=0)
    close(theta.grad.numpy(), dth_path, "theta")


def _wide_reference(orc, w, steps, paths, pay, pairs):
    """The oracle's forward-mode tangents reduced row by row (no [d, d, paths]
    array): per entry of dP/dLrho the mean, mean |per-path value|, the
    contribution of paths in the strike band and the per-path standard
    error; the same for dP/dcorr on the listed pairs (per path, the inner
    product of the path's dP/dLrho with cholesky_tangent(Lrho, E_ab))."""
    d, K = len(w["s0"]), float(pay["strike"])
    xT, tL = orc.gbm_corr_tangents(w["s0"], w["sigma"], w["corr"], w["r"], w["T"], steps, paths)
    S = np.exp(xT)
    U = w["weights"] @ S
    call = pay["kind"] == "call"
    slope = (U > K).astype(np.float64) if call else -(U < K).astype(np.float64)
    f = np.exp(-w["r"] * w["T"]) * (np.maximum(U - K, 0.0) if call else np.maximum(K - U, 0.0))
    g = np.exp(-w["r"] * w["T"]) * slope[None, :] * w["weights"][:, None] * S
    band = np.abs(U - K) <= BAND * K
    stats = {k: np.zeros((d, d)) for k in ("mean", "scale", "flips", "se")}
    L = np.linalg.cholesky(w["corr"])
    J = {ab: orc.cholesky_tangent(L, _unit_pair(d, *ab)) for ab in pairs}
    pair_paths = {ab: np.zeros(paths) for ab in pairs}
    for a in range(d):
        per = g[a][None, :] * tL[a * (a + 1) // 2: a * (a + 1) // 2 + a + 1]
        stats["mean"][a, :a + 1] = per.mean(axis=1)
        stats["scale"][a, :a + 1] = np.abs(per).mean(axis=1)
        stats["flips"][a, :a + 1] = np.abs(per[:, band]).sum(axis=1) / paths
        stats["se"][a, :a + 1] = per.std(axis=1, ddof=1) / np.sqrt(paths)
        for ab in pairs:
            pair_paths[ab] += J[ab][a, :a + 1] @ per
    return f, U, stats, pair_paths, band


def _unit_pair(d, a, b):
    E = np.zeros((d, d))
    E[a, b] = E[b, a] = 1.0
    return E


@pytest.mark.parametrize("d,paths,steps,kind", [(96, 4096, 6, "call"), (130, 700, 5, "put"), (512, 256, 3, "call")])
def test_corr_greeks_wide_baskets(gb, orc, d, paths, steps, kind):
    """d > 64 (the wide path: summed normals in device memory, FP32 products,
    the Cholesky adjoint per batch in global memory): d = 96 (whole Philox
    blocks, 32 batches, standard errors checked), d = 130 (blocks straddle
    steps, ragged 64-wide tiles), d = 512 (the large-basket workload's
    width).  Every entry of dP/dLrho and the symmetric dP/dcorr on sampled
    pairs against the oracle with the tolerance of the d <= 64 tests."""
    w = _market(d, k=4)
    K = float(w["weights"] @ w["s0"]) * (1.0 if kind == "call" else 1.02)
    pay = dict(kind=kind, strike=K)
    rng = np.random.default_rng(d)
    pairs = [(1, 0), (d - 1, 0), (d - 1, d - 2)] + [tuple(sorted(rng.choice(d, 2, replace=False))[::-1])
                                                     for _ in range(5)]
    (p, pse), dl, dr = gb.corr_greeks(gbm_model(w), cfg_of(w, paths=paths, steps=steps), pay)
    f, U, st, pair_paths, band = _wide_reference(orc, w, steps, paths, pay, pairs)
    m, se = orc.mean_se(f)
    assert abs(p - m) <= REL * abs(m) + 1e-12, (p, m)
    assert abs(pse - se) <= 1e-3 * se
    err = np.abs(dl[..., 0] - st["mean"])
    tol = 2e-5 * st["scale"] + st["flips"] + 1e-12
    bad = np.argwhere(err > tol)
    assert bad.size == 0, (d, bad[:5], err[tuple(bad[0])], tol[tuple(bad[0])], int(band.sum()))
    assert np.all(dl[..., 0][np.triu_indices(d, 1)] == 0.0)
    for (a, b), per in pair_paths.items():
        want = per.mean()
        tol = 2e-5 * np.abs(per).mean() + np.abs(per[band]).sum() / paths + 1e-12
        assert abs(dr[a, b, 0] - want) <= tol, (d, a, b, dr[a, b, 0], want, tol)
        assert dr[a, b, 0] == dr[b, a, 0]
    assert np.all(dr[..., 0][np.arange(d), np.arange(d)] == 0.0)
    if paths >= 32 * 128:
        mask = np.tril(np.ones((d, d), dtype=bool)) & (st["se"] > 0)
        ratio = dl[..., 1][mask] / st["se"][mask]
        assert 0.8 <= np.median(ratio) <= 1.2, np.median(ratio)
        assert ratio.min() >= 0.3 and ratio.max() <= 2.5, (ratio.min(), ratio.max())


@pytest.mark.parametrize("d,paths,steps", [(4, 8000, 12), (7, 2900, 9), (64, 2600, 10)])
@pytest.mark.parametrize("kind", ["asian_call", "asian_put"])
def test_corr_greeks_asian_match_oracle(gb, orc, d, paths, steps, kind):
    """Asian basket (payoff on the average of U over the steps; two passes
    per tile, a d x d outer product per path-step): every entry of dP/dLrho
    and dP/dcorr against the oracle's forward-mode tangents with the same
    tolerance (the band taken on the average), d = 4 / 7 / 64, calls and
    puts, ragged last tiles; standard errors as for the European form (>= 20
    batches; 62 at d = 4, where only six pairs enter the median)."""
    w = _market(d)
    K = float(w["weights"] @ w["s0"]) * (1.0 if kind == "asian_call" else 1.02)
    pay = dict(kind=kind, strike=K)
    (p, pse), dl, dr = gb.corr_greeks(gbm_model(w), cfg_of(w, paths=paths, steps=steps), pay)
    ref = orc.gbm_corr_greeks(w["s0"], w["sigma"], w["corr"], w["r"], w["T"], steps, paths, pay,
                              weights=w["weights"])
    m, se = orc.mean_se(ref["f"])
    assert abs(p - m) <= REL * abs(m), (p, m)
    assert abs(pse - se) <= 1e-3 * se
    _check_entries(dl, ref["dl"], ref["U"], K, "dl")
    _check_entries(dr, ref["drho"], ref["U"], K, "drho")
    assert np.all(dl[..., 0][np.triu_indices(d, 1)] == 0.0)
    assert np.allclose(dr[..., 0], dr[..., 0].T, rtol=0, atol=1e-12 * np.abs(dr[..., 0]).max())
    _check_se(dl, ref["dl"], "dl")
    _check_se(dr, ref["drho"], "drho")
