"""GPU parity of the large-basket kernels (64 < d <= 512): the FP32 path
against the oracle on identical streams, the tensor-core path against the
oracle's normals rounded as the kernel rounds them, basket Greeks (delta,
vega, rho vectors) against the oracle's forward-mode tangents, and the
d = 512 workload in its full launch shape."""
import numpy as np
import pytest

import workloads
from gpu_util import REL, assert_price_close, cfg_of, gbm_model, oracle_gbm
from test_gpu_tc import emulate, flip_bound, payoffs_from_U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _case(d, k, paths, steps, seed=13):
    s0, sg, corr = workloads.basket_market(d, k, seed=seed)
    w = np.full(d, 1.0 / d)
    b0 = float(w @ s0)
    pays = [dict(kind="call", strike=b0), dict(kind="put", strike=1.05 * b0)]
    return dict(s0=s0, sigma=sg, corr=corr, weights=w, r=0.05, T=1.0, steps=steps, paths=paths, seed=42), pays


@pytest.mark.parametrize("d", [65, 128, 250])
def test_fp32_wide_matches_oracle(gb, orc, d):
    w, pays = _case(d, 4, 300, 10)
    got = gb.price(gbm_model(w), cfg_of(w), pays)
    ref = oracle_gbm(orc, w, w["paths"], pays)
    for i in range(2):
        m, se = orc.mean_se(ref[i])
        assert abs(got[i][0] - m) <= REL * abs(m), (d, i, got[i], m)
        assert abs(got[i][1] - se) <= 1e-3 * se


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp8"])
@pytest.mark.parametrize("d", [100, 192, 512])
def test_tc_big_matches_quantised_emulation(gb, orc, prec, d):
    w, pays = _case(d, 8, 300, 6)
    got = gb.price(gbm_model(w), cfg_of(w, precision=prec), pays)
    U, aux = emulate(orc, w, prec, w["paths"], w["steps"], fp8_fixed=True, detail=True)
    want = payoffs_from_U(U, pays, w["r"], w["T"])
    fb = flip_bound(aux, U, pays[:2], w["r"], w["T"])
    for i in range(2):
        m = want[i].mean()
        assert abs(got[i][0] - m) <= 2 * REL * abs(m) + fb[i], (prec, d, i, got[i][0], m)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_basket_greeks_match_oracle(gb, orc, prec):
    w, pays = _case(20, 3, 4000, 8)
    w2 = dict(w)
    pr, g = gb.greeks(gbm_model(w), cfg_of(w, precision=prec), pays[:1])
    ref = orc.gbm_greeks(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], w["paths"], pays[:1], corr=w["corr"],
                         weights=w["weights"])[0]
    d = 20
    scale = np.max(np.abs(ref.mean(axis=1)[:d]))
    for k in range(2 * d + 1):
        m, se = orc.mean_se(ref[k])
        tol = 2e-5 * max(abs(m), scale) if prec == "fp32" else 3 * se + 3e-3 * max(abs(m), scale)
        assert abs(g[0, k, 0] - m) <= tol, (prec, k, g[0, k, 0], m, se)


def test_d512_workload_full_shape(gb):
    """d = 512, 2^20 paths, 252 steps in the launch shape of the report: BF16
    and FP8 within 3 SE of each other, the delta vector of the BF16 run sums
    to a consistent value (sum_n delta_n S0_n = e^{-rT} E[1{B > K} B])."""
    w = workloads.basket_d512()
    pays = w["payoffs"]
    _, g = gb.greeks(gbm_model(w), cfg_of(w, precision="bf16"), pays)
    bf = gb.price(gbm_model(w), cfg_of(w, precision="bf16"), pays)
    f8 = gb.price(gbm_model(w), cfg_of(w, precision="fp8"), pays)
    assert abs(bf[0][0] - f8[0][0]) <= 3 * bf[0][1] + 0.01 * abs(bf[0][0])
    d = 512
    deltas = g[0, :d, 0]
    assert np.all(np.isfinite(deltas)) and np.all(deltas > 0)
    # homogeneity of degree 1 in S0: sum_n S0_n dP/dS0_n = P + K e^{-rT} P(B > K)
    lhs = float(deltas @ w["s0"])
    assert lhs > bf[0][0]


# ---------------------------------------------------------------------------
# The d = 512 workload (16-factor market, ATM basket call) at its full
# horizon of 252 steps.  One FP64 oracle run on the first 2^14 paths serves
# both the 2^14-path accuracy check of every precision and, through its first
# P_EXACT paths (16 tensor-core tiles of 128 paths and a ragged tail), the
# exact checks.
# ---------------------------------------------------------------------------
N_SUBSET = 1 << 14
P_EXACT = 2048 + 77


@pytest.fixture(scope="module")
def c5(orc):
    w = workloads.basket_d512(paths=N_SUBSET)
    b0 = w["payoffs"][0]["strike"]
    pays = [w["payoffs"][0], dict(kind="put", strike=1.05 * b0)]
    ref = oracle_gbm(orc, w, N_SUBSET, pays)  # [2, 2^14] discounted per-path payoffs
    return w, pays, ref


def flip_bound_terminal(aux, U, pays, r, T):
    """flip_bound for European payoffs on U(T) under log-Euler with a fixed
    operand scale: a code change of z_k at any step moves U(T) by at most
    |D| |sum_n w_n S_n(T) sqrt(dt) sigma_n Lq[n, k]| (the same factor for
    every step), so the per-path bound is that factor against the code
    widths summed over the steps; O(paths d^2) instead of O(steps^2)."""
    G = np.abs(np.einsum("pn,n,nk->pk", aux["S"][-1], aux["coef"], aux["Lq"]))
    FT = np.einsum("pk,pk->p", aux["D"].sum(axis=1), G)
    disc, N, uT = np.exp(-r * T), U.shape[1], U[-1]
    out = []
    for p in pays:
        K = p["strike"]
        active = (uT - K > -FT) if p["kind"] == "call" else (K - uT > -FT)
        out.append(disc * float(np.sum(FT * active)) / N)
    return out


def test_d512_full_horizon_fp32_exact(gb, c5):
    """FP32 (register-tiled SIMT contraction) against the FP64 oracle on the
    identical stream: 1e-5 relative per price, standard errors 1e-3."""
    w, pays, ref = c5
    got = gb.price(gbm_model(w), cfg_of(w, paths=P_EXACT, precision="fp32"), pays)
    assert_price_close(got, ref[:, :P_EXACT], pays, label="d512 fp32 252 steps")


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_d512_full_horizon_tensor_cores_exact(gb, orc, c5, prec):
    """The tensor-core kernel (TMEM accumulation over all 252 steps, the
    factor ring wrapping every step) against the oracle's normals rounded as
    the kernel rounds them, within 2e-5 relative plus the rounding-flip bound."""
    w, pays, _ = c5
    got = gb.price(gbm_model(w), cfg_of(w, paths=P_EXACT, precision=prec), pays)
    want, fb = np.zeros(len(pays)), np.zeros(len(pays))
    for off in range(0, P_EXACT, 128):
        n = min(128, P_EXACT - off)
        U, aux = emulate(orc, w, prec, n, w["steps"], path_offset=off, fp8_fixed=True, detail=True)
        want += payoffs_from_U(U, pays, w["r"], w["T"]).sum(axis=1)
        fb += np.array(flip_bound_terminal(aux, U, pays, w["r"], w["T"])) * n
    want, fb = want / P_EXACT, fb / P_EXACT
    for i, p in enumerate(pays):
        print(f"d512 {prec} {p['kind']}: GPU {got[i][0]:.7f} emulation {want[i]:.7f} "
              f"(|diff| {abs(got[i][0] - want[i]):.2e}, flip bound {fb[i]:.2e})")
        assert abs(got[i][0] - want[i]) <= 2 * REL * abs(want[i]) + fb[i], (prec, p, got[i][0], want[i], fb[i])


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_d512_subset_error_vs_fp64(gb, orc, c5, prec):
    """The error of each precision against the unrounded FP64 oracle on the
    first 2^14 paths of the workload (the same paths): printed per price, and
    within 3 standard errors (FP32: within 1e-5 relative)."""
    w, pays, ref = c5
    got = gb.price(gbm_model(w), cfg_of(w, paths=N_SUBSET, precision=prec), pays)
    for i, p in enumerate(pays):
        m, se = orc.mean_se(ref[i])
        err = got[i][0] - m
        print(f"d512 {prec} {p['kind']} 2^14 paths x 252 steps: GPU {got[i][0]:.7f} FP64 {m:.7f} "
              f"error {err:+.3e} ({abs(err) / abs(m):.2e} relative, {abs(err) / se:.3f} SE)")
        assert abs(err) <= 3 * se
        if prec == "fp32":
            assert abs(err) <= REL * abs(m)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_d512_full_horizon_greek_vectors(gb, orc, c5, prec):
    """The 512 deltas, 512 vegas and rho of the basket call from mc_greeks
    against the oracle's forward-mode pathwise tangents on the same P_EXACT
    paths, entry by entry.  The scale of an entry is the largest of its
    mean, the largest mean delta and its mean absolute per-path term (many
    vegas are means of large terms of both signs that nearly cancel, and the
    FP32 error of a mean follows its terms, not the mean); FP32 within 2e-5
    of that scale, BF16 within 3 SE + 3e-3 of it."""
    w, pays, _ = c5
    pr, g = gb.greeks(gbm_model(w), cfg_of(w, paths=P_EXACT, precision=prec), pays[:1])
    ref = orc.gbm_greeks(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], P_EXACT, pays[:1], corr=w["corr"],
                         weights=w["weights"])[0]
    d = len(w["s0"])
    scale = np.max(np.abs(ref.mean(axis=1)[:d]))
    worst = 0.0
    for k in range(2 * d + 1):
        m, se = orc.mean_se(ref[k])
        sc = max(abs(m), scale, float(np.mean(np.abs(ref[k]))))
        tol = 2e-5 * sc if prec == "fp32" else 3 * se + 3e-3 * sc
        worst = max(worst, abs(g[0, k, 0] - m) / tol)
        assert abs(g[0, k, 0] - m) <= tol, (prec, k, g[0, k, 0], m, se)
    print(f"d512 {prec} Greeks: largest |GPU - oracle| / tolerance over the {2 * d + 1} entries {worst:.3f}")
