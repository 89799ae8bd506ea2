"""GPU parity of the tensor-core contraction (BF16 / FP16 / E4M3 operands,
FP32 accumulation and state).

Two checks per case:
  1. exact pipeline check: the expected price is rebuilt from the oracle's
     FP64 normals with the operands rounded exactly as the kernel rounds them
     (tests/quant.py) and the rest of the step in FP64; the kernel must match
     it to 1e-5 relative (+ the barrier band), so any layout, swizzle or
     descriptor error fails;
  2. reduced-precision error: the relative error against the unrounded FP64
     oracle on the same stream is reported and must stay within 3 standard
     errors (Sec. V.A: low-precision multiplies add no significant bias).
"""
import numpy as np
import pytest

import workloads
from gpu_util import BAND, REL, cfg_of, gbm_model, oracle_gbm
from quant import quantize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def normal_error_bound(zf):
    """Bound on |GPU normal - FP64 normal| for a stream prefix zf [paths, n]
    (n even; Box-Muller pairs (2m, 2m + 1) share the radius r): the SFU's
    sin / cos (absolute error ~2^-20.5 near [-pi, pi]) and the one-FMA angle
    scale with r; the absolute error of lg2.approx (~2^-22) moves -2 ln u by
    1.4 * 2^-22, hence r by 1.7e-7 / r, capped at sqrt(1.4 * 2^-22) ~ 6e-4
    where r -> 0 (u -> 1); plus a margin."""
    r = np.hypot(zf[:, 0::2], zf[:, 1::2]).repeat(2, axis=1)
    return np.minimum(1.5e-6 * r + 1.7e-7 / np.maximum(r, 1e-30) + 3e-7, 6e-4)


def emulate(orc, w, prec, paths, steps, scheme="log_euler", path_offset=0, fp8_fixed=False, fold=None,
            detail=False, flip=False):
    """Per-path monitored U of the quantised-operand scheme:
    dW_n = sqrt(dt) sigma_n sum_k Lq[n,k] zq[k] / (s_n s_z); E4M3 normals are
    scaled per path and step by 448 / max|z| (fp8_fixed: by 448 / 6).  Row
    scales s_n: E4M3 448 / max_k |L[n,k]|; BF16 on the d <= 64 path (fold)
    the column scale c sqrt(dt) sigma_n, c = log2(e) (log-Euler) or 1
    (Euler); otherwise 1.

    detail=True also returns what flip_bound needs: the kernel rounds its own
    FP32 normals, which differ from the oracle's by up to
    normal_error_bound, so an operand whose window [z - e, z + e] straddles a
    rounding boundary may take either neighbouring code; D [paths, steps, d]
    is the width of the codes the window can reach (in units of z).
    flip=True rounds every such operand to the code at the other end of its
    window instead (a planted worst case for checking flip_bound)."""
    d = len(w["s0"])
    if fold is None:
        fold = prec == "bf16" and d <= 64
    L = orc.cholesky(w["corr"]) if w.get("corr") is not None else np.eye(d)
    dt = w["T"] / steps
    s_n = np.ones(d)
    if prec == "fp8":
        s_n = np.where(np.abs(L).max(axis=1) > 0, 448.0 / np.abs(L).max(axis=1), 1.0)
    elif fold:
        c = np.log2(np.e) if scheme == "log_euler" else 1.0
        col = c * np.sqrt(dt) * np.asarray(w["sigma"], dtype=np.float64)
        s_n = np.where(col > 0, col, 1.0)
    Lq = quantize((L * s_n[:, None]).astype(np.float32), prec) / s_n[:, None]
    nz = steps * d + (steps * d) % 2
    Zf = np.stack([orc.normals(w["seed"], path_offset + n, 0, nz) for n in range(paths)]).reshape(paths, nz)
    E = normal_error_bound(Zf)[:, :steps * d].reshape(paths, steps, d)
    Z = Zf[:, :steps * d].reshape(paths, steps, d)
    Z32 = Z.astype(np.float32)
    rel_s = np.zeros((paths, steps, 1))
    if prec == "fp8" and fp8_fixed:
        s = np.float32(448.0 / 6.0)
        Zq = quantize((Z32 * s).astype(np.float32), "fp8") / np.float64(s)
        ex = s * E + np.abs(Z32 * s) * 1.2e-7
        lo = quantize(Z32 * s - ex, "fp8") / np.float64(s)
        hi = quantize(Z32 * s + ex, "fp8") / np.float64(s)
    elif prec == "fp8":
        amax = np.abs(Z32).max(axis=2, keepdims=True)
        s = (np.float32(448.0) / amax).astype(np.float32)
        # the kernel multiplies by amax/448 computed in binary32
        Zq = quantize((Z32 * s).astype(np.float32), "fp8") * (amax / np.float32(448.0)).astype(np.float32)
        # the kernel's amax comes from its own normals: relative error of s
        rel_s = np.take_along_axis(E, np.abs(Z32).argmax(axis=2)[..., None], axis=2) / amax + 2.4e-7
        x = Z32.astype(np.float64) * s
        ex = s * E + np.abs(x) * rel_s
        lo = quantize(x - ex, "fp8") * (amax / 448.0)
        hi = quantize(x + ex, "fp8") * (amax / 448.0)
    else:
        Zq = quantize(Z32, prec)
        lo, hi = quantize(Z - E, prec), quantize(Z + E, prec)
    D = hi - lo
    if flip:  # every ambiguous operand takes the code at the other end of its window
        Zq = np.where(D > 0, np.where(np.abs(Zq - lo) <= np.abs(Zq - hi), hi, lo), Zq)
    sig, s0, wt = w["sigma"], w["s0"], w["weights"]
    x = np.log(s0)[None, :].repeat(paths, 0) if scheme == "log_euler" else s0[None, :].repeat(paths, 0).copy()
    U = np.empty((steps + 1, paths))
    U[0] = wt @ s0
    S_hist = np.empty((steps + 1, paths, d))
    S_hist[0] = s0[None, :]
    dW_hist = np.empty((steps, paths, d))
    for i in range(steps):
        dW = np.sqrt(dt) * sig[None, :] * (Zq[:, i, :] @ Lq.T)
        dW_hist[i] = dW
        if scheme == "log_euler":
            x = x + (w["r"] - 0.5 * sig ** 2) * dt + dW
            S = np.exp(x)
        else:
            x = x * (1.0 + w["r"] * dt + dW)
            S = x
        S_hist[i + 1] = S
        U[i + 1] = S @ wt
    if not detail:
        return U
    # dS_n(t) / dW_n(i), t > i: S_n(t) (log-Euler), S_n(t) / (1 + r dt + dW_n(i)) (Euler)
    R = np.ones((steps, paths, d)) if scheme == "log_euler" else 1.0 / (1.0 + w["r"] * dt + dW_hist)
    coef = np.asarray(wt) * np.sqrt(dt) * np.asarray(sig)
    return U, dict(S=S_hist, dW=dW_hist, R=R, Lq=Lq, D=D, rel_s=rel_s, coef=coef, w=np.asarray(wt))


def flip_bound(aux, U, pays, r, T):
    """First-order bound on how far each price can move when the kernel
    rounds any subset of the ambiguous operands (emulate's D) to the other
    code: a change of z_k at step i moves U(t), t > i, by at most
    |D| |sum_n w_n S_n(t) sqrt(dt) sigma_n Lq[n,k]|, and every payoff moves
    by at most its slope (<= 1) times that, on paths where it can be active.
    E4M3 with a per-row scale adds the rescaling of the whole row by the
    kernel's own amax (rel_s).  Barrier payoffs add the call value of paths
    whose monitored maximum can cross H."""
    S, D, R, Lq, coef = aux["S"], aux["D"], aux["R"], aux["Lq"], aux["coef"]
    steps, paths = D.shape[1], D.shape[0]
    FT, FS = np.zeros(paths), np.zeros(paths)
    rel = aux["rel_s"][..., 0]                                            # [p, i]
    for i in range(steps):
        # |dU(t) / dz_k(i)| for t = i + 1 .. M: [t, p, k]
        G = np.abs(np.einsum("tpn,pn,n,nk->tpk", S[i + 1:], R[i], coef, Lq))
        FT += np.einsum("pk,pk->p", D[:, i, :], G[-1])
        FS += np.einsum("pk,pk->p", D[:, i, :], G.max(axis=0))
        if np.any(rel[:, i] > 0):  # the row's rescaling by the kernel's own amax
            dWr = np.abs(aux["dW"][i]) * R[i] * aux["w"]
            FT += rel[:, i] * np.einsum("pn,pn->p", S[-1], dWr)
            FS += rel[:, i] * np.einsum("pn,pn->p", S[i + 1:].max(axis=0), dWr)
    disc, N = np.exp(-r * T), U.shape[1]
    uT, avg, mx = U[-1], U[1:].mean(axis=0), U[1:].max(axis=0)
    out = []
    for p in pays:
        K, k = p["strike"], p["kind"]
        if k == "call":
            b = np.sum(FT * (uT - K > -FT))
        elif k == "put":
            b = np.sum(FT * (K - uT > -FT))
        elif k == "asian_call":
            b = np.sum(FS * (avg - K > -FS))
        elif k in ("uo_call", "ui_call"):
            near = np.abs(mx - p["barrier"]) <= FS
            b = np.sum(FT * (uT - K > -FT)) + np.sum(np.maximum(uT - K + FT, 0)[near])
        else:
            raise ValueError(k)
        out.append(disc * float(b) / N)
    return out


def payoffs_from_U(U, pays, r, T):
    disc = np.exp(-r * T)
    uT, avg, mx, mn = U[-1], U[1:].mean(axis=0), U[1:].max(axis=0), U[1:].min(axis=0)
    out = []
    for p in pays:
        K, H, k = p["strike"], p.get("barrier", np.inf), p["kind"]
        call, put = np.maximum(uT - K, 0), np.maximum(K - uT, 0)
        v = {"call": call, "put": put, "asian_call": np.maximum(avg - K, 0),
             "uo_call": np.where(mx >= H, 0, call), "ui_call": np.where(mx >= H, call, 0)}[k]
        out.append(disc * v)
    return np.array(out)


def band(U, pays, per_path):
    m = []
    for i, p in enumerate(pays):
        if p["kind"].startswith("u") and "barrier" in p:
            near = np.abs(U[1:].max(axis=0) - p["barrier"]) <= BAND * p["barrier"]
            m.append(float(np.sum(np.maximum(U[-1][near] - p["strike"], 0))) / U.shape[1] * 1.01 + 1e-12)
        else:
            m.append(0.0)
    return m


def _case(d, k, paths, steps, seed=5):
    s0, sg, corr = workloads.basket_market(d, k, seed=seed)
    w = np.full(d, 1.0 / d)
    b0 = float(w @ s0)
    pays = [dict(kind="call", strike=b0), dict(kind="put", strike=b0), dict(kind="asian_call", strike=b0),
            dict(kind="uo_call", strike=b0, barrier=1.1 * b0), dict(kind="ui_call", strike=b0, barrier=1.1 * b0)]
    return dict(s0=s0, sigma=sg, corr=corr, weights=w, r=0.05, T=1.0, steps=steps, paths=paths, seed=42), pays


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp8"])
@pytest.mark.parametrize("d,scheme", [(64, "log_euler"), (40, "log_euler"), (64, "euler"), (7, "log_euler")])
def test_tc_matches_quantised_emulation(gb, orc, prec, d, scheme):
    w, pays = _case(d, 3, 1000, 12)
    got = gb.price(gbm_model(w), cfg_of(w, precision=prec, scheme=scheme), pays)
    U, aux = emulate(orc, w, prec, w["paths"], w["steps"], scheme, detail=True)
    want = payoffs_from_U(U, pays, w["r"], w["T"])
    bm = band(U, pays, want)
    fb = flip_bound(aux, U, pays, w["r"], w["T"])
    for i, p in enumerate(pays):
        m = want[i].mean()
        tol = REL * max(abs(m), 1e-6) + bm[i] + fb[i]
        assert abs(got[i][0] - m) <= tol, (prec, d, scheme, p, got[i][0], m, tol)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp8"])
def test_tc_reduced_precision_error_vs_fp64(gb, orc, prec):
    """The d = 64 workload on 4096 paths: error of the reduced-precision
    contraction against the FP64 oracle (same stream) within 3 SE."""
    w = workloads.basket_d64(paths=4096)
    got = gb.price(gbm_model(w), cfg_of(w, precision=prec), w["payoffs"])
    ref = oracle_gbm(orc, w, w["paths"], w["payoffs"])
    for i, p in enumerate(w["payoffs"]):
        m, se = orc.mean_se(ref[i])
        rel = abs(got[i][0] - m) / abs(m)
        print(f"{prec} {p['kind']}: {got[i][0]:.6f} vs FP64 {m:.6f}  rel err {rel:.2e}  (SE {se:.4f})")
        assert abs(got[i][0] - m) <= 3 * se


def test_tc_full_size_bf16_vs_fp32(gb):
    """Full d = 64 workload (2^18 paths x 252 steps) in the benchmark's launch
    shape: BF16 and FP32 contractions agree within 3 SE of each other, and
    the BF16 run equals the combination of its 4 path shards."""
    w = workloads.basket_d64()
    bf = gb.price(gbm_model(w), cfg_of(w, precision="bf16"), w["payoffs"])
    fp = gb.price(gbm_model(w), cfg_of(w), w["payoffs"])
    for i in range(len(w["payoffs"])):
        assert abs(bf[i][0] - fp[i][0]) <= 3 * fp[i][1]
    N = w["paths"]
    parts = [gb.price(gbm_model(w), cfg_of(w, paths=N // 4, path_offset=k * N // 4, precision="bf16"), w["payoffs"])
             for k in range(4)]
    for i in range(len(w["payoffs"])):
        assert abs(np.mean([p[i][0] for p in parts]) - bf[i][0]) <= 1e-6 * abs(bf[i][0])


def test_tc_sampled_windows_full_range(gb, orc):
    """Windows sampled across the full 2^18-path range match the quantised
    emulation exactly (the counter-based stream makes any window reproducible)."""
    w = workloads.basket_d64()
    pays = w["payoffs"]
    steps = 20
    for off in (0, 131_101, (1 << 18) - 200):
        got = gb.price(gbm_model(w), cfg_of(w, paths=200, path_offset=off, steps=steps, precision="bf16"), pays)
        U, aux = emulate(orc, w, "bf16", 200, steps, path_offset=off, detail=True)
        want = payoffs_from_U(U, pays, w["r"], w["T"])
        bm = band(U, pays, want)
        fb = flip_bound(aux, U, pays, w["r"], w["T"])
        for i in range(len(pays)):
            m = want[i].mean()
            assert abs(got[i][0] - m) <= REL * abs(m) + bm[i] + fb[i], (off, pays[i], got[i][0], m)
