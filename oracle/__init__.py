"""FP64 CPU oracle for the financial Monte Carlo method of Belletti et al.,
"Tensor Processing Units for Financial Monte Carlo" (2019).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports, links or falls back to it, and this package imports nothing
from the library: the two share no code.  Inputs come from the seeded
generators in ``workloads.py``, which hold none of the method's arithmetic.

Contents
  oracle.c   plain C, IEEE double, one path at a time (compiled by ``build()``
             with gcc -O2 -ffp-contract=off, no fast-math; OpenMP only over
             independent paths, each writing its own output slot, so results do
             not depend on the thread count):
             Philox4x32-10 (Sec. IV.A), Box-Muller (Sec. VI.D), Cholesky
             (Sec. II.A.3), correlated GBM Euler / log-Euler steps (Sec. II.A.1,
             II.A.2), Heston full-truncation Euler, European / Asian / barrier
             payoffs (Sec. I.A.2), continuous barrier monitoring through the
             Brownian-bridge extremes (Sec. VI.A.1), the factor-model
             correlation (rho = B B^T + diag(e^2)), randomised Sobol
             quasi-Monte Carlo (Sec. IV, VI.D), forward-mode pathwise Greeks
             (Sec. I.A.3) including the tangents of the terminal log-prices
             in the Cholesky-factor entries, the estimator of Eq. 3 with its
             standard error.
  (here)     the forward derivative of the Cholesky factor and the chain rule
             from factor tangents to correlation sensitivities (numpy).
  mlp.py     FP64 numpy forward / backward of the pricing surrogate.
  risk.py    VaR / CVaR of Sec. VI.B and nested revaluation.

Pins (tests/test_oracle_*.py, all ``-m "not gpu"``): Philox against PyTorch's
independent header-only Philox engine; uniform-map exactness; normal moments;
Black-Scholes closed form incl. the paper's vanilla-call value (Sec. VI.A.1);
martingale and put-call parity; discrete geometric-Asian closed form and the
AM >= GM invariant; one-step barrier closed form and in + out = vanilla;
Cholesky against numpy; d = 1 basket = scalar GBM; geometric-basket closed
form; Heston xi = 0 reduction to Black-Scholes; Greeks against Black-Scholes
closed forms and common-random-number finite differences; the Brownian-bridge
barrier against the paper's "In and Out Put" value 23.1371783926 and the
continuous down-and-in call closed form, at one step and at many; the Sobol
recurrence against its definition, one-dimensional stratification, the
(0, m, 2)-net property of the first two dimensions, and the randomised-QMC
price against Black-Scholes and its error rate against plain Monte Carlo;
the Cholesky tangent against LAPACK differences, per-path correlation
tangents against bumped simulations, the geometric-basket correlation
sensitivity against its closed form and the arithmetic basket's against
common-random-number differences; the nested up-and-out value against the
discretely monitored barrier of the GBM pricer; the random digital shift
against the uniform law (Box-Muller normals of the shifted origin); Heston
barriers against the monitored maxima of its saved paths; Cholesky refusals
against LAPACK's; VaR as the sample's upper quantile found by scanning the
losses.  The closed forms themselves are pinned by quadrature, parity,
differences and their limits (tests/test_closed_forms.py).  A mutation check
(tests/test_oracle_mutants.py) plants one plausible mistake at a time in a
copy of this package and requires a pin to fail for each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Payoff vocabulary shared by name with the library's binding; the integer
# codes below are this file's own.
PAYOFF_CODES = {
    "call": 0, "put": 1, "asian_call": 2, "asian_put": 3,
    "uo_call": 4, "ui_call": 5, "uo_put": 6, "ui_put": 7,
    "do_call": 8, "di_call": 9, "do_put": 10, "di_put": 11,
}
HESTON_GREEKS = ("delta", "vega_v0", "rho", "d_kappa", "d_theta", "d_xi", "d_rho")
HESTON_PARAM_ORDER = ("s0", "v0", "r", "kappa", "theta", "xi", "rho")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, no CUDA).
    With GBMC_ORACLE_SANITIZE=1 the AddressSanitizer + UndefinedBehaviorSanitizer
    build liboracle_asan.so instead (the sanitizer tests load it with the
    sanitizer runtimes preloaded)."""
    san = os.environ.get("GBMC_ORACLE_SANITIZE") == "1"
    path = _LIB_PATH.replace("liboracle.so", "liboracle_asan.so") if san else _LIB_PATH
    with _lock:
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            return path
        tmp = path + f".tmp{os.getpid()}"
        opt = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
               "-fno-omit-frame-pointer"] if san else ["-O2"]
        cmd = ["gcc", *opt, "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
        return path


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    d_p, i_p, u32_p = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint32)
    i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    lib.orc_philox4x32_10.argtypes = [u32_p, u32_p, u32_p]
    lib.orc_uniform.argtypes = [ctypes.c_uint32]
    lib.orc_uniform.restype = dbl
    lib.orc_normals.argtypes = [u64, u64, u64, i64, d_p]
    lib.orc_cholesky.argtypes = [i32, d_p, d_p]
    lib.orc_cholesky.restype = i32
    gbm_common = [i32, d_p, d_p, d_p, d_p, dbl, dbl, i32, i32, u64, i64, i64]
    lib.orc_gbm_payoffs.argtypes = gbm_common + [i32, i_p, d_p, d_p, d_p]
    lib.orc_gbm_payoffs.restype = i32
    lib.orc_gbm_paths.argtypes = gbm_common + [i32, d_p]
    lib.orc_gbm_paths.restype = i32
    lib.orc_gbm_greeks.argtypes = gbm_common + [i32, i_p, d_p, d_p]
    lib.orc_gbm_greeks.restype = i32
    lib.orc_gbm_corr_tangents.argtypes = [i32, d_p, d_p, d_p, dbl, dbl, i32, u64, i64, i64, d_p, d_p]
    lib.orc_gbm_corr_tangents.restype = i32
    lib.orc_gbm_corr_asian_tangents.argtypes = [i32, d_p, d_p, d_p, d_p, dbl, dbl, i32, u64, i64, i64, d_p, d_p]
    lib.orc_gbm_corr_asian_tangents.restype = i32
    lib.orc_gbm1d_bridge_payoffs.argtypes = [dbl] * 5 + [i32, u64, i64, i64, i32, i_p, d_p, d_p, d_p]
    lib.orc_gbm1d_bridge_payoffs.restype = i32
    lib.orc_gbm_factor_payoffs.argtypes = [i32, i32, d_p, d_p, d_p, d_p, dbl, dbl, i32, i32, u64, i64, i64, i32, i_p,
                                           d_p, d_p, d_p, d_p]
    lib.orc_gbm_factor_payoffs.restype = i32
    lib.orc_sobol_directions.argtypes = [i32, u32_p]
    lib.orc_sobol_directions.restype = i32
    lib.orc_sobol_points.argtypes = [i32, i64, i64, u32_p]
    lib.orc_sobol_points.restype = i32
    lib.orc_qmc_gbm_payoffs.argtypes = [i32, d_p, d_p, d_p, d_p, dbl, dbl, i32, i32, u64, i64, i64, i64, i32, i_p,
                                        d_p, d_p, d_p]
    lib.orc_qmc_gbm_payoffs.restype = i32
    hes_common = [dbl] * 8 + [i32, u64, i64, i64]
    lib.orc_heston_payoffs.argtypes = hes_common + [i32, i_p, d_p, d_p, d_p]
    lib.orc_heston_payoffs.restype = i32
    lib.orc_heston_paths.argtypes = hes_common + [i32, d_p]
    lib.orc_heston_paths.restype = i32
    lib.orc_heston_greeks.argtypes = hes_common + [i32, i_p, d_p, d_p]
    lib.orc_heston_greeks.restype = i32
    lib.orc_mean_se.argtypes = [d_p, i64, d_p, d_p]
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


# --------------------------------------------------------------------------
# Random stream (Sec. IV.A keyed counter-based generation; Sec. VI.D Box-Muller)
# --------------------------------------------------------------------------
def philox(counter, key):
    """One Philox4x32-10 block: counter = 4 words, key = 2 words -> 4 words."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32_p = ctypes.POINTER(ctypes.c_uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(u32_p), k.ctypes.data_as(u32_p), out.ctypes.data_as(u32_p))
    return out


def uniform(x: int) -> float:
    return _load().orc_uniform(int(x) & 0xFFFFFFFF)


def normals(seed: int, stream: int, j0: int, count: int) -> np.ndarray:
    """Normals j0 .. j0+count-1 of stream `stream` (path index) under `seed`."""
    z = np.empty(count, dtype=np.float64)
    _load().orc_normals(seed, stream, j0, count, _dptr(z))
    return z


def cholesky(A) -> np.ndarray:
    A = _f64(A)
    d = A.shape[0]
    L = np.empty_like(A)
    rc = _load().orc_cholesky(d, _dptr(A), _dptr(L))
    if rc != 0:
        raise OracleError("matrix is not positive definite")
    return L


def mean_se(f) -> tuple[float, float]:
    """Eq. 3 estimator and its standard error, compensated sums in index order."""
    f = _f64(f).ravel()
    m, s = ctypes.c_double(), ctypes.c_double()
    _load().orc_mean_se(_dptr(f), f.size, ctypes.byref(m), ctypes.byref(s))
    return m.value, s.value


# --------------------------------------------------------------------------
# Payoff list helpers
# --------------------------------------------------------------------------
def _payoff_arrays(payoffs):
    kinds = np.array([PAYOFF_CODES[p["kind"]] for p in payoffs], dtype=np.int32)
    K = np.array([float(p.get("strike", 0.0)) for p in payoffs], dtype=np.float64)
    H = np.array([float(p.get("barrier", np.inf)) for p in payoffs], dtype=np.float64)
    return kinds, K, H


def _gbm_args(s0, sigma, corr, weights):
    s0 = _f64(np.atleast_1d(s0))
    sigma = _f64(np.atleast_1d(sigma))
    d = s0.size
    corr = None if corr is None else _f64(corr).reshape(d, d)
    w = np.full(d, 1.0 / d) if weights is None else _f64(weights)
    return d, s0, sigma, corr, w


# --------------------------------------------------------------------------
# Correlated GBM (Sec. II.A.1 scalar and II.A.2 multivariate Euler-Maruyama)
# --------------------------------------------------------------------------
def gbm_payoffs(s0, sigma, r, T, steps, paths, payoffs, corr=None, weights=None,
                scheme="log_euler", seed=42, path_offset=0) -> np.ndarray:
    """Discounted per-path payoffs, shape [len(payoffs), paths]."""
    d, s0, sigma, corr, w = _gbm_args(s0, sigma, corr, weights)
    kinds, K, H = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), paths), dtype=np.float64)
    ip = kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rc = _load().orc_gbm_payoffs(d, _dptr(s0), _dptr(sigma), _dptr(corr), _dptr(w), r, T, steps,
                                 0 if scheme == "log_euler" else 1, seed, path_offset, paths,
                                 len(payoffs), ip, _dptr(K), _dptr(H), _dptr(out))
    _check(rc, "orc_gbm_payoffs")
    return out


def gbm1d_bridge_payoffs(s0, sigma, r, T, steps, paths, payoffs, weight=1.0, seed=42, path_offset=0) -> np.ndarray:
    """Discounted per-path payoffs of a single-asset GBM whose barriers are
    monitored continuously through the Brownian-bridge extremes (Sec. VI.A.1),
    shape [len(payoffs), paths]."""
    kinds, K, H = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), paths), dtype=np.float64)
    rc = _load().orc_gbm1d_bridge_payoffs(float(s0), float(sigma), float(weight), float(r), float(T), int(steps),
                                          seed, path_offset, paths, len(payoffs),
                                          kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(K), _dptr(H),
                                          _dptr(out))
    _check(rc, "orc_gbm1d_bridge_payoffs")
    return out


def gbm_factor_payoffs(s0, sigma, loadings, r, T, steps, paths, payoffs, weights=None, scheme="log_euler", seed=42,
                       path_offset=0, terminal=False):
    """Discounted per-path payoffs [len(payoffs), paths] of the factor-model
    GBM basket (loadings B: [d, k]); with terminal=True also the terminal
    prices [d, paths]."""
    s0 = _f64(np.atleast_1d(s0))
    sigma = _f64(np.atleast_1d(sigma))
    d = s0.size
    B = _f64(np.asarray(loadings, dtype=np.float64).reshape(d, -1))
    k = B.shape[1]
    w = np.full(d, 1.0 / d) if weights is None else _f64(weights)
    kinds, K, H = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), paths), dtype=np.float64)
    ST = np.empty((d, paths), dtype=np.float64) if terminal else None
    rc = _load().orc_gbm_factor_payoffs(d, k, _dptr(s0), _dptr(sigma), _dptr(B) if k else None, _dptr(w), r, T, steps,
                                        0 if scheme == "log_euler" else 1, seed, path_offset, paths, len(payoffs),
                                        kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(K), _dptr(H),
                                        _dptr(out), _dptr(ST))
    _check(rc, "orc_gbm_factor_payoffs")
    return (out, ST) if terminal else out


def gbm_factor_greeks(s0, sigma, loadings, r, T, steps, paths, payoff, weights=None, seed=42, path_offset=0):
    """Per-path discounted pathwise Greeks [2d + 1, paths] of a European
    basket call or put under the factor model, log-Euler (Sec. I.A.3: the
    derivative of the discounted payoff along the path, the normals held
    fixed).  With ln S_a(T) = ln S0_a + (r - sigma_a^2/2) T + sigma_a X_a,
    X_a a sum of the path's normals that depends on neither parameter, and
    f' the payoff's slope in U = sum_a w_a S_a(T):
      d/dS0_a    = e^{-rT} f' w_a S_a / S0_a                    (a < d)
      d/dsigma_a = e^{-rT} f' w_a S_a (ln(S_a / S0_a) - (r + sigma_a^2/2) T) / sigma_a
      d/dr       = e^{-rT} (f' U T - T f)                       (k = 2d)"""
    s0 = _f64(np.atleast_1d(s0))
    sigma = _f64(np.atleast_1d(sigma))
    d = s0.size
    w = np.full(d, 1.0 / d) if weights is None else _f64(weights)
    kind, K = payoff["kind"], float(payoff["strike"])
    if kind not in ("call", "put"):
        raise ValueError("European call or put only")
    f, ST = gbm_factor_payoffs(s0, sigma, loadings, r, T, steps, paths, [payoff], weights=w, seed=seed,
                               path_offset=path_offset, terminal=True)
    disc = np.exp(-r * T)
    U = w @ ST
    slope = (U > K).astype(np.float64) if kind == "call" else -(U < K).astype(np.float64)
    wS = w[:, None] * ST
    out = np.empty((2 * d + 1, paths), dtype=np.float64)
    out[:d] = disc * slope[None, :] * wS / s0[:, None]
    out[d:2 * d] = disc * slope[None, :] * wS * (np.log(ST / s0[:, None]) - ((r + 0.5 * sigma ** 2) * T)[:, None]) \
        / sigma[:, None]
    out[2 * d] = disc * slope * U * T - T * f[0]
    return out


def sobol_directions(ndim: int) -> np.ndarray:
    """Direction numbers V[j][k] (uint32) of the oracle's Sobol sequence."""
    V = np.zeros((ndim, 32), dtype=np.uint32)
    _check(_load().orc_sobol_directions(ndim, V.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), "orc_sobol_directions")
    return V


def sobol_points(ndim: int, n: int, n0: int = 0) -> np.ndarray:
    """Unshifted 32-bit Sobol words of points n0 .. n0 + n - 1: [n, ndim]."""
    P = np.zeros((n, ndim), dtype=np.uint32)
    _check(_load().orc_sobol_points(ndim, n0, n, P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), "orc_sobol_points")
    return P


def qmc_gbm_payoffs(s0, sigma, r, T, steps, points, payoffs, rep=0, corr=None, weights=None, scheme="log_euler",
                    seed=42, point_offset=0) -> np.ndarray:
    """Discounted payoffs of the randomised-Sobol GBM paths of replication
    `rep`, shape [len(payoffs), points]."""
    d, s0, sigma, corr, w = _gbm_args(s0, sigma, corr, weights)
    kinds, K, H = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), points), dtype=np.float64)
    rc = _load().orc_qmc_gbm_payoffs(d, _dptr(s0), _dptr(sigma), _dptr(corr), _dptr(w), r, T, steps,
                                     0 if scheme == "log_euler" else 1, seed, rep, point_offset, points,
                                     len(payoffs), kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(K),
                                     _dptr(H), _dptr(out))
    _check(rc, "orc_qmc_gbm_payoffs")
    return out


def gbm_paths(s0, sigma, r, T, steps, paths, corr=None, weights=None, scheme="log_euler",
              seed=42, path_offset=0, save_every=1) -> np.ndarray:
    """Asset prices at steps 0, k, 2k, ..., M: shape [M/k + 1, d, paths]."""
    d, s0, sigma, corr, w = _gbm_args(s0, sigma, corr, weights)
    nsave = steps // save_every + 1
    out = np.empty((nsave, d, paths), dtype=np.float64)
    rc = _load().orc_gbm_paths(d, _dptr(s0), _dptr(sigma), _dptr(corr), _dptr(w), r, T, steps,
                               0 if scheme == "log_euler" else 1, seed, path_offset, paths,
                               save_every, _dptr(out))
    _check(rc, "orc_gbm_paths")
    return out


def gbm_greeks(s0, sigma, r, T, steps, paths, payoffs, corr=None, weights=None,
               scheme="log_euler", seed=42, path_offset=0) -> np.ndarray:
    """Per-path discounted pathwise Greeks, shape [len(payoffs), 2d+1, paths]:
    d/dS0_a (a < d), d/dsigma_a (d <= k < 2d), d/dr (k = 2d)."""
    d, s0, sigma, corr, w = _gbm_args(s0, sigma, corr, weights)
    kinds, K, _ = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), 2 * d + 1, paths), dtype=np.float64)
    ip = kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rc = _load().orc_gbm_greeks(d, _dptr(s0), _dptr(sigma), _dptr(corr), _dptr(w), r, T, steps,
                                0 if scheme == "log_euler" else 1, seed, path_offset, paths,
                                len(payoffs), ip, _dptr(K), _dptr(out))
    _check(rc, "orc_gbm_greeks")
    return out


def gbm_corr_tangents(s0, sigma, corr, r, T, steps, paths, seed=42, path_offset=0):
    """log-Euler terminal log-prices x_a(T), shape [d, paths], and their
    forward tangents d x_a(T) / d Lrho[a][b] (b <= a, Lrho = chol(corr), drift
    held fixed), packed row by row, shape [d (d + 1) / 2, paths]."""
    d, s0, sigma, corr, _ = _gbm_args(s0, sigma, corr, None)
    xT = np.empty((d, paths), dtype=np.float64)
    tL = np.empty((d * (d + 1) // 2, paths), dtype=np.float64)
    rc = _load().orc_gbm_corr_tangents(d, _dptr(s0), _dptr(sigma), _dptr(corr), r, T, steps, seed, path_offset,
                                       paths, _dptr(xT), _dptr(tL))
    _check(rc, "orc_gbm_corr_tangents")
    return xT, tL


def gbm_corr_asian_tangents(s0, sigma, corr, weights, r, T, steps, paths, seed=42, path_offset=0):
    """The arithmetic average A = (1/M) sum_i U(t_i) of the basket U = w . S
    over the steps, shape [paths], and its forward tangents dA / d Lrho[a][b]
    (b <= a, drift held fixed), packed row by row, [d (d + 1) / 2, paths]."""
    d, s0, sigma, corr, w = _gbm_args(s0, sigma, corr, weights)
    A = np.empty(paths, dtype=np.float64)
    tA = np.empty((d * (d + 1) // 2, paths), dtype=np.float64)
    rc = _load().orc_gbm_corr_asian_tangents(d, _dptr(s0), _dptr(sigma), _dptr(corr), _dptr(w), r, T, steps, seed,
                                             path_offset, paths, _dptr(A), _dptr(tA))
    _check(rc, "orc_gbm_corr_asian_tangents")
    return A, tA


def cholesky_tangent(L, E) -> np.ndarray:
    """Forward derivative of the Cholesky factor: if A = L L^T moves by a
    symmetric E, L moves by L Phi(L^-1 E L^-T), Phi = the lower triangle with
    the diagonal halved (differentiating A = L L^T and keeping L lower
    triangular)."""
    L = np.asarray(L, dtype=np.float64)
    Li = np.linalg.inv(L)
    X = Li @ np.asarray(E, dtype=np.float64) @ Li.T
    return L @ (np.tril(X, -1) + 0.5 * np.diag(np.diag(X)))


def gbm_corr_greeks(s0, sigma, corr, r, T, steps, paths, payoff, weights=None, seed=42, path_offset=0):
    """Per-path discounted pathwise correlation sensitivities of a European
    basket call or put on U = sum_a w_a S_a(T), or of an Asian one on the
    average A of U over the steps (log-Euler), forward mode:
      f     [paths]        discounted payoff
      U     [paths]        the basket value at T (Asian: the average A)
      dl    [d, d, paths]  d/d Lrho[a][b] (b <= a; zero above the diagonal)
      drho  [d, d, paths]  d/d corr[a][b] for a != b, corr[a][b] and
                           corr[b][a] moved together; zero on the diagonal
    The payoff's slope in x_a is w_a S_a 1{U > K} (call), -w_a S_a 1{U < K}
    (put); d/d corr[a][b] = sum over (c, e) of d/d Lrho[c][e] times the
    (c, e) entry of cholesky_tangent(Lrho, E_ab), E_ab the symmetric unit
    direction of the pair."""
    d, s0, sigma, corr, w = _gbm_args(s0, sigma, corr, weights)
    corr = np.eye(d) if corr is None else corr
    kind, K = payoff["kind"], float(payoff["strike"])
    if kind in ("asian_call", "asian_put"):
        # the payoff on the average A of the basket over the steps
        A, tA = gbm_corr_asian_tangents(s0, sigma, corr, w, r, T, steps, paths, seed, path_offset)
        disc = np.exp(-r * T)
        if kind == "asian_call":
            f, slope = np.maximum(A - K, 0.0), (A > K).astype(np.float64)
        else:
            f, slope = np.maximum(K - A, 0.0), -(A < K).astype(np.float64)
        dl = np.zeros((d, d, paths))
        for a in range(d):
            for b in range(a + 1):
                dl[a, b] = disc * slope * tA[a * (a + 1) // 2 + b]
        return dict(f=disc * f, U=A, dl=dl, drho=corr_chain(corr, dl))
    if kind not in ("call", "put"):
        raise ValueError("European or Asian call or put only")
    xT, tL = gbm_corr_tangents(s0, sigma, corr, r, T, steps, paths, seed, path_offset)
    S = np.exp(xT)
    U = w @ S
    disc = np.exp(-r * T)
    if kind == "call":
        f, slope = np.maximum(U - K, 0.0), (U > K).astype(np.float64)
    else:
        f, slope = np.maximum(K - U, 0.0), -(U < K).astype(np.float64)
    g = disc * slope[None, :] * w[:, None] * S          # d (discounted payoff) / d x_a
    dl = np.zeros((d, d, paths))
    for a in range(d):
        for b in range(a + 1):
            dl[a, b] = g[a] * tL[a * (a + 1) // 2 + b]
    return dict(f=disc * f, U=U, dl=dl, drho=corr_chain(corr, dl))


def corr_chain(corr, dl) -> np.ndarray:
    """Chain rule from d/d Lrho (shape [d, d, ...], lower triangle) to
    d/d corr[a][b], a != b, with corr[a][b] and corr[b][a] moved together:
    the inner product of dl with cholesky_tangent(chol(corr), E_ab) for every
    pair.  Returns the symmetric array, zero on the diagonal."""
    d = dl.shape[0]
    rest = dl.shape[2:]
    flat = dl.reshape(d * d, -1)
    Lr = cholesky(corr)
    pairs = [(a, b) for a in range(d) for b in range(a)]
    drho = np.zeros((d, d, flat.shape[1]))
    if pairs:
        J = np.empty((len(pairs), d * d))
        for k, (a, b) in enumerate(pairs):
            E = np.zeros((d, d))
            E[a, b] = E[b, a] = 1.0
            J[k] = cholesky_tangent(Lr, E).ravel()
        vals = J @ flat
        for k, (a, b) in enumerate(pairs):
            drho[a, b] = drho[b, a] = vals[k]
    return drho.reshape((d, d) + rest)


# --------------------------------------------------------------------------
# Heston, full-truncation Euler
# --------------------------------------------------------------------------
def _hes(h):
    return (float(h["s0"]), float(h["v0"]), float(h["r"]), float(h["kappa"]), float(h["theta"]),
            float(h["xi"]), float(h["rho"]))


def heston_payoffs(h, T, steps, paths, payoffs, seed=42, path_offset=0) -> np.ndarray:
    kinds, K, H = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), paths), dtype=np.float64)
    ip = kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rc = _load().orc_heston_payoffs(*_hes(h), T, steps, seed, path_offset, paths, len(payoffs), ip,
                                    _dptr(K), _dptr(H), _dptr(out))
    _check(rc, "orc_heston_payoffs")
    return out


def heston_paths(h, T, steps, paths, seed=42, path_offset=0, save_every=1) -> np.ndarray:
    """[M/k + 1, 2, paths]: component 0 price, 1 variance."""
    out = np.empty((steps // save_every + 1, 2, paths), dtype=np.float64)
    rc = _load().orc_heston_paths(*_hes(h), T, steps, seed, path_offset, paths, save_every, _dptr(out))
    _check(rc, "orc_heston_paths")
    return out


def heston_greeks(h, T, steps, paths, payoffs, seed=42, path_offset=0) -> np.ndarray:
    """[len(payoffs), 7, paths] in the order of HESTON_GREEKS."""
    kinds, K, _ = _payoff_arrays(payoffs)
    out = np.empty((len(payoffs), 7, paths), dtype=np.float64)
    ip = kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rc = _load().orc_heston_greeks(*_hes(h), T, steps, seed, path_offset, paths, len(payoffs), ip,
                                   _dptr(K), _dptr(out))
    _check(rc, "orc_heston_greeks")
    return out


def price(per_path: np.ndarray):
    """Mean and standard error of each row of a [n_payoff, paths] array."""
    return [mean_se(row) for row in np.atleast_2d(per_path)]
