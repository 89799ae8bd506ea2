"""Mutation check of the oracle's pins.  Each case plants one plausible
mistake in a copy of the oracle (a dropped term, a wrong sign, a wrong index
or a transposed operand) and runs the pins named beside it against that copy:
at least one of them must fail by an assertion (not by a build or import
error).  A control copy without a mistake must pass the same pins, so a
failure is the planted mistake's doing.

The copy sits in a temporary directory; tests/conftest.py puts it ahead of
the repository's oracle on the import path when GBMC_ORACLE_DIR names it, and
the copy builds its own liboracle.so beside its oracle.c.  Nothing here runs
on, or touches, the CUDA library."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
import tempfile

import pytest

pytestmark = pytest.mark.slow

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T = "tests/"

# (name, file under oracle/, text, replacement, pin tests that must catch it)
MUTANTS = [
    # Philox4x32-10 round function and key schedule (Sec. IV.A)
    ("philox_high_word", "oracle.c", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;",
     [T + "test_oracle_rng.py::test_philox_bit_exact_vs_torch_engine"]),
    ("philox_weyl_swap", "oracle.c", "k0 += W0; k1 += W1;", "k0 += W1; k1 += W0;",
     [T + "test_oracle_rng.py::test_philox_bit_exact_vs_torch_engine"]),
    # uniform map and Box-Muller (Sec. VI.D)
    ("uniform_offset", "oracle.c", "((double)(x >> 9) + 0.5)", "((double)(x >> 9) + 1.0)",
     [T + "test_oracle_rng.py"]),
    ("box_muller_radius", "oracle.c", "double rad = sqrt(-2.0 * log(u1));", "double rad = sqrt(-log(u1));",
     [T + "test_oracle_rng.py"]),
    ("box_muller_angle", "oracle.c", "rad * sin(2.0 * M_PI * u2)", "rad * sin(M_PI * u2)",
     [T + "test_oracle_rng.py"]),
    # Cholesky factor of the correlation (Sec. II.A.3)
    ("cholesky_transposed_operand", "oracle.c", "s -= L[(size_t)i * d + k] * L[(size_t)j * d + k];",
     "s -= L[(size_t)i * d + k] * L[(size_t)k * d + j];", [T + "test_oracle_gbm.py::test_cholesky_against_lapack"]),
    # GBM step (Sec. II.A.1, II.A.2)
    ("log_euler_drift_sign", "oracle.c", "x[a] += (m->r - 0.5 * m->sig[a] * m->sig[a]) * dt + dW;",
     "x[a] += (m->r + 0.5 * m->sig[a] * m->sig[a]) * dt + dW;", [T + "test_oracle_gbm.py"]),
    ("increment_scale", "oracle.c", "double dW = sdt * m->sig[a] * y[a];", "double dW = dt * m->sig[a] * y[a];",
     [T + "test_oracle_gbm.py"]),
    ("factor_transposed", "oracle.c", "for (int k = 0; k <= a; ++k) s += m->Lrho[(size_t)a * d + k] * z[k];",
     "for (int k = 0; k <= a; ++k) s += m->Lrho[(size_t)k * d + a] * z[k];", [T + "test_oracle_gbm.py"]),
    ("euler_drift_dropped", "oracle.c", "double g = 1.0 + m->r * dt + dW;", "double g = 1.0 + dW;",
     [T + "test_oracle_gbm.py"]),
    # payoffs and monitoring (Sec. I.A.2)
    ("asian_average_count", "oracle.c", "stats->u_T = u; stats->avg = sum / M;",
     "stats->u_T = u; stats->avg = sum / (M + 1);", [T + "test_oracle_gbm.py"]),
    ("barrier_at_maturity_only", "oracle.c", "int up_hit = p->umax >= H,", "int up_hit = p->u_T >= H,",
     [T + "test_oracle_gbm.py"]),
    ("down_barrier_direction", "oracle.c", "down_hit = p->umin <= H;", "down_hit = p->umin >= H;",
     [T + "test_oracle_gbm.py", T + "test_oracle_bridge.py"]),
    ("up_in_put_pays_call", "oracle.c", "case ORC_UI_PUT: return up_hit ? put : 0.0;",
     "case ORC_UI_PUT: return up_hit ? call : 0.0;", [T + "test_oracle_gbm.py"]),
    ("discount_without_maturity", "oracle.c",
     "    const double disc = exp(-r * T);\n#pragma omp parallel\n    {\n"
     "        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);",
     "    const double disc = exp(-r);\n#pragma omp parallel\n    {\n"
     "        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);", [T + "test_oracle_gbm.py"]),
    # Brownian-bridge extremes (Sec. VI.A.1)
    ("bridge_variance_half", "oracle.c", "- 2.0 * dt * sig * sig * log(Ui)", "- dt * sig * sig * log(Ui)",
     [T + "test_oracle_bridge.py"]),
    ("bridge_minimum_sign", "oracle.c", "0.5 * (x + y - sqrt(", "0.5 * (x + y + sqrt(",
     [T + "test_oracle_bridge.py"]),
    # factor-model correlation
    ("factor_idiosyncratic_variance", "oracle.c", "e[a] = sqrt(q < 1.0 ? 1.0 - q : 0.0);",
     "e[a] = q < 1.0 ? 1.0 - q : 0.0;", [T + "test_oracle_factor.py"]),
    ("factor_noise_reuses_factors", "oracle.c",
     "eps[a] = stream_normal(&st, base + (uint64_t)k + (uint64_t)a);",
     "eps[a] = stream_normal(&st, base + (uint64_t)a);", [T + "test_oracle_factor.py"]),
    # Sobol directions and points (Sec. IV, VI.D)
    ("sobol_recurrence_shift", "oracle.c", "uint32_t v = m[k - s] ^ (m[k - s] << s);",
     "uint32_t v = m[k - s] ^ (m[k - s] << (s - 1));", [T + "test_oracle_qmc.py"]),
    ("sobol_direction_scale", "oracle.c", "= m[k] << (32 - k);", "= m[k] << (31 - k);",
     [T + "test_oracle_qmc.py"]),
    ("qmc_shift_shared_by_a_pair", "oracle.c", "^ shift[2 * jn + 1]);", "^ shift[2 * jn]);",
     [T + "test_oracle_qmc.py"]),
    # forward-mode pathwise Greeks (Sec. I.A.3)
    ("vega_tangent_sign", "oracle.c", "tg->tsig[a] += -m->sig[a] * dt + sdt * y[a];",
     "tg->tsig[a] += m->sig[a] * dt + sdt * y[a];", [T + "test_oracle_greeks.py"]),
    ("rho_discount_term_dropped", "oracle.c",
     "g[((size_t)p * ng + 2 * d) * npaths + n] = disc * (slope * dr - T * f);",
     "g[((size_t)p * ng + 2 * d) * npaths + n] = disc * slope * dr;", [T + "test_oracle_greeks.py"]),
    ("asian_tangent_unaveraged", "oracle.c", "tg->aS0[a] += m->w[a] * f * tg->tS0[a] / M;",
     "tg->aS0[a] += m->w[a] * f * tg->tS0[a];", [T + "test_oracle_greeks.py"]),
    ("euler_vega_tangent_growth", "oracle.c", "tg->tsig[a] = tg->tsig[a] * g + x[a] * sdt * y[a];",
     "tg->tsig[a] = tg->tsig[a] + x[a] * sdt * y[a];", [T + "test_oracle_greeks.py"]),
    # correlation tangents (Sec. I.A.3, VI.A.2)
    ("corr_tangent_wrong_normal", "oracle.c",
     "t[(size_t)a * (a + 1) / 2 + b] += sdt * sig[a] * z[b];\n                }\n            }\n"
     "            for (int a = 0; a < d; ++a) xT[",
     "t[(size_t)a * (a + 1) / 2 + b] += sdt * sig[a] * z[a];\n                }\n            }\n"
     "            for (int a = 0; a < d; ++a) xT[", [T + "test_oracle_corr.py"]),
    ("corr_asian_tangent_unweighted", "oracle.c", "acc[(size_t)a * (a + 1) / 2 + b] += v * t[",
     "acc[(size_t)a * (a + 1) / 2 + b] += t[", [T + "test_oracle_corr.py"]),
    # Heston full-truncation Euler and its tangents
    ("heston_correlation_root", "oracle.c", "const double rc = sqrt(1.0 - h->rho * h->rho);",
     "const double rc = 1.0 - h->rho * h->rho;", [T + "test_oracle_heston.py"]),
    ("heston_mean_reversion_sign", "oracle.c", "h->kappa * (h->theta - vp) * dt", "h->kappa * (vp - h->theta) * dt",
     [T + "test_oracle_heston.py"]),
    ("heston_rho_tangent_sign", "oracle.c", "(z1 - h->rho / rc * z2)", "(z1 + h->rho / rc * z2)",
     [T + "test_oracle_greeks.py"]),
    ("heston_root_tangent_factor", "oracle.c", "dt * dvp / (2.0 * sq)", "dt * dvp / sq",
     [T + "test_oracle_greeks.py"]),
    # estimator (Eq. 3)
    ("standard_error_divisor", "oracle.c", "/ (double)(n - 1)) : 0.0;", "/ (double)n) : 0.0;",
     [T + "test_oracle_gbm.py::test_mean_se_definition"]),
    # risk scenarios, nested values, labels (Sec. VI.B)
    ("scenario_horizon_root", "oracle.c", "sqrt(h) * sig[u] * w", "h * sig[u] * w",
     [T + "test_oracle_risk.py::test_scenario_moments"]),
    ("nested_discount_one_step", "oracle.c", "return exp(-r * steps * dt) * sum / inner;",
     "return exp(-r * dt) * sum / inner;", [T + "test_oracle_risk.py::test_nested_value_is_black_scholes"]),
    ("nested_barrier_at_maturity_only", "oracle.c", "if (kind == ORC_UO_CALL && exp(mx) >= H) f = 0.0;",
     "if (kind == ORC_UO_CALL && ST >= H) f = 0.0;", [T + "test_oracle_risk.py::test_nested_up_and_out_monitors_every_step"]),
    ("label_vega_sign", "oracle.c", "(sqrt(dt) * zs - sig * tau)", "(sqrt(dt) * zs + sig * tau)",
     [T + "test_oracle_risk.py::test_label_greeks_pins"]),
    ("loss_sign", "risk.py", "l = np.sort(-np.asarray(pnl, dtype=np.float64))[::-1]",
     "l = np.sort(np.asarray(pnl, dtype=np.float64))[::-1]",
     [T + "test_oracle_risk.py::test_var_cvar_normal_closed_form"]),
    ("var_rank_off_by_one", "risk.py", "    var = l[k - 1]", "    var = l[min(k, l.size - 1)]",
     [T + "test_oracle_risk.py::test_var_is_the_upper_quantile_of_the_sample"]),
    ("var_rank_rounded_down", "risk.py", "k = max(1, math.ceil((1.0 - alpha) * l.size - 1e-9))",
     "k = max(1, math.floor((1.0 - alpha) * l.size))",
     [T + "test_oracle_risk.py::test_var_is_the_upper_quantile_of_the_sample"]),
    ("cvar_tail_includes_var", "risk.py", "tail = l[:k][l[:k] > var]", "tail = l[:k]",
     [T + "test_oracle_risk.py::test_var_is_the_upper_quantile_of_the_sample"]),
    # Cholesky tangent and the chain rule to correlation sensitivities (numpy)
    ("cholesky_tangent_full_diagonal", "__init__.py", "np.tril(X, -1) + 0.5 * np.diag(np.diag(X))",
     "np.tril(X, -1) + np.diag(np.diag(X))", [T + "test_oracle_corr.py"]),
    ("cholesky_tangent_transposed", "__init__.py", "X = Li @ np.asarray(E, dtype=np.float64) @ Li.T",
     "X = Li.T @ np.asarray(E, dtype=np.float64) @ Li", [T + "test_oracle_corr.py"]),
    ("corr_chain_one_sided", "__init__.py", "drho[a, b] = drho[b, a] = vals[k]", "drho[a, b] = vals[k]",
     [T + "test_oracle_corr.py"]),
    ("corr_put_slope_sign", "__init__.py", "f, slope = np.maximum(K - U, 0.0), -(U < K).astype(np.float64)",
     "f, slope = np.maximum(K - U, 0.0), (U < K).astype(np.float64)", [T + "test_oracle_corr.py"]),
    ("factor_vega_drift_sign", "__init__.py", "((r + 0.5 * sigma ** 2) * T)", "((r - 0.5 * sigma ** 2) * T)",
     [T + "test_oracle_factor.py"]),
    ("factor_rho_discount_term_dropped", "__init__.py", "out[2 * d] = disc * slope * U * T - T * f[0]",
     "out[2 * d] = disc * slope * U * T", [T + "test_oracle_factor.py"]),
    # stream layout: both words of the key, the stream index and the counter
    ("stream_counter_high_word", "oracle.c",
     "uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)s->stream, (uint32_t)(s->stream >> 32)};",
     "uint32_t ctr[4] = {(uint32_t)q, 0u, (uint32_t)s->stream, (uint32_t)(s->stream >> 32)};",
     [T + "test_oracle_rng.py::test_box_muller_pairs"]),
    ("stream_index_high_word", "oracle.c",
     "uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)s->stream, (uint32_t)(s->stream >> 32)};",
     "uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)s->stream, 0u};",
     [T + "test_oracle_rng.py::test_box_muller_pairs"]),
    ("key_high_word", "oracle.c", "uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};",
     "uint32_t key[2] = {(uint32_t)s->seed, 0u};", [T + "test_oracle_rng.py::test_box_muller_pairs"]),
    ("path_offset_ignored", "oracle.c",
     "gbm_path(&m, path0 + n, NULL, 0, 0, 0, NULL, &ps, NULL, work);\n            for (int p = 0; p < npay; ++p)\n"
     "                out",
     "gbm_path(&m, n, NULL, 0, 0, 0, NULL, &ps, NULL, work);\n            for (int p = 0; p < npay; ++p)\n"
     "                out", [T + "test_oracle_gbm.py"]),
    ("saved_path_slot", "oracle.c",
     "save[((size_t)slot * d + a) * ld + col] = (m->scheme == 0) ? exp(x[a]) : x[a];",
     "save[((size_t)(slot - 1) * d + a) * ld + col] = (m->scheme == 0) ? exp(x[a]) : x[a];",
     [T + "test_oracle_gbm.py"]),
    ("estimator_compensation_sign", "oracle.c", "(a - t) + b : (b - t) + a;", "(a - t) - b : (b - t) + a;",
     [T + "test_oracle_gbm.py::test_mean_se_definition"]),
    # more of the bridge, factor model, Sobol and risk paths
    ("bridge_uniform_lane", "oracle.c", "return orc_uniform(x[j & 3]);", "return orc_uniform(x[0]);",
     [T + "test_oracle_bridge.py"]),
    ("bridge_maximum_on_grid_only", "oracle.c", "if (hi > mmax) mmax = hi;", "if (y > mmax) mmax = y;",
     [T + "test_oracle_bridge.py"]),
    ("bridge_average_unweighted", "oracle.c", "sum += w * exp(x);", "sum += exp(x);", [T + "test_oracle_bridge.py"]),
    ("factor_euler_drift_dropped", "oracle.c", "else x[a] *= 1.0 + r * dt + dW;\n                    u += w[a]",
     "else x[a] *= 1.0 + dW;\n                    u += w[a]", [T + "test_oracle_factor.py"]),
    ("factor_loadings_transposed", "oracle.c", "for (int j = 0; j < k; ++j) f += B[(size_t)a * k + j] * z[j];",
     "for (int j = 0; j < k; ++j) f += B[(size_t)j * d + a] * z[j];", [T + "test_oracle_factor.py"]),
    ("sobol_first_dimension_bits", "oracle.c", "for (int k = 0; k < 32; ++k) V[k] = (uint32_t)1 << (31 - k);",
     "for (int k = 0; k < 32; ++k) V[k] = (uint32_t)1 << (31 - (k ^ 1));", [T + "test_oracle_qmc.py"]),
    ("qmc_factor_wrong_normal", "oracle.c",
     "for (int k = 0; k <= a; ++k) acc += m.Lrho[(size_t)a * d + k] * z[k];",
     "for (int k = 0; k <= a; ++k) acc += m.Lrho[(size_t)a * d + k] * z[a];", [T + "test_oracle_qmc.py"]),
    ("scenario_drift_sign", "oracle.c", "exp((mu - 0.5 * sig[u] * sig[u]) * h", "exp((mu + 0.5 * sig[u] * sig[u]) * h",
     [T + "test_oracle_risk.py::test_scenario_moments"]),
    ("scenario_factor_transposed", "oracle.c", "for (int k = 0; k <= u; ++k) w += L[(size_t)u * d + k] * z[k];",
     "for (int k = 0; k <= u; ++k) w += L[(size_t)k * d + u] * z[k];",
     [T + "test_oracle_risk.py::test_scenario_moments"]),
    ("base_values_skip_the_horizon", "oracle.c", "rem[o] + hsteps, inner, seed, 5,", "rem[o], inner, seed, 5,",
     [T + "test_oracle_risk.py::test_base_values_run_the_full_maturity"]),
    ("label_delta_ratio_dropped", "oracle.c", "disc * in * ST / S,", "disc * in * ST,",
     [T + "test_oracle_risk.py::test_label_greeks_pins"]),
    ("label_greeks_undiscounted", "oracle.c",
     "const double v[3] = {disc * (ST > 1.0 ? ST - 1.0 : 0.0), disc * in * ST / S,",
     "const double v[3] = {disc * (ST > 1.0 ? ST - 1.0 : 0.0), in * ST / S,",
     [T + "test_oracle_risk.py::test_label_greeks_pins"]),
    # more Greeks: GBM, Heston, correlation
    ("r_tangent_scaled", "oracle.c", "tg->tr[a] += dt;", "tg->tr[a] += dt * m->sig[a];", [T + "test_oracle_greeks.py"]),
    ("euler_delta_tangent_init", "oracle.c", "tg->tS0[a] = (m->scheme == 0) ? 1.0 / m->s0[a] : 1.0;",
     "tg->tS0[a] = 1.0 / m->s0[a];", [T + "test_oracle_greeks.py"]),
    ("asian_rho_from_terminal", "oracle.c", "dr += asian ? tg.ar[a] : m.w[a] * tg.tr[a];", "dr += m.w[a] * tg.tr[a];",
     [T + "test_oracle_greeks.py"]),
    ("heston_v0_tangent_seed", "oracle.c", "tv[1] = 1.0;", "tv[1] = 0.0;", [T + "test_oracle_greeks.py"]),
    ("heston_rho_greek_maturity", "oracle.c", "if (k == 2) v -= T * disc * f;", "if (k == 2) v -= disc * f;",
     [T + "test_oracle_greeks.py"]),
    ("heston_truncation_tangent", "oracle.c", "double dvp = v > 0.0 ? tv[k] : 0.0;", "double dvp = tv[k];",
     [T + "test_oracle_greeks.py"]),
    ("heston_theta_tangent_sign", "oracle.c", "h->kappa * (dth - dvp)", "h->kappa * (dth + dvp)",
     [T + "test_oracle_greeks.py"]),
    ("heston_kappa_tangent_sign", "oracle.c", "(dkap * (h->theta - vp)", "(dkap * (h->theta + vp)",
     [T + "test_oracle_greeks.py"]),
    ("heston_xi_tangent_dropped", "oracle.c", "+ (dxi * sq + h->xi * dsq) * z1;", "+ (h->xi * dsq) * z1;",
     [T + "test_oracle_greeks.py"]),
    ("heston_asian_tangent_unaveraged", "oracle.c", "ta[k] += S * tx[k] / M;", "ta[k] += S * tx[k];",
     [T + "test_oracle_greeks.py"]),
    ("heston_variance_noise_wrong_normal", "oracle.c", "+ h->xi * sq * z1;", "+ h->xi * sq * z2;",
     [T + "test_oracle_heston.py"]),
    ("heston_saved_variance_truncated", "oracle.c", "save[((size_t)slot * 2 + 1) * ld + col] = v;",
     "save[((size_t)slot * 2 + 1) * ld + col] = vp;", [T + "test_oracle_heston.py"]),
    ("corr_asian_average_count", "oracle.c", "A[n] = sumU / steps;", "A[n] = sumU / (steps + 1);",
     [T + "test_oracle_corr.py"]),
    ("corr_weight_dropped", "__init__.py", "g = disc * slope[None, :] * w[:, None] * S",
     "g = disc * slope[None, :] * S", [T + "test_oracle_corr.py"]),
    ("corr_asian_undiscounted", "__init__.py", "dl[a, b] = disc * slope * tA[a * (a + 1) // 2 + b]",
     "dl[a, b] = slope * tA[a * (a + 1) // 2 + b]", [T + "test_oracle_corr.py"]),
    ("corr_asian_put_slope_sign", "__init__.py",
     "f, slope = np.maximum(K - A, 0.0), -(A < K).astype(np.float64)",
     "f, slope = np.maximum(K - A, 0.0), (A < K).astype(np.float64)", [T + "test_oracle_corr.py"]),
    ("cholesky_tangent_upper_triangle", "__init__.py", "return L @ (np.tril(X, -1) + 0.5 * np.diag(np.diag(X)))",
     "return L @ (np.triu(X, 1) + 0.5 * np.diag(np.diag(X)))", [T + "test_oracle_corr.py"]),
    ("factor_put_slope_sign", "__init__.py",
     'slope = (U > K).astype(np.float64) if kind == "call" else -(U < K).astype(np.float64)\n    wS',
     'slope = (U > K).astype(np.float64) if kind == "call" else (U < K).astype(np.float64)\n    wS',
     [T + "test_oracle_factor.py"]),
    ("factor_delta_ratio_dropped", "__init__.py", "out[:d] = disc * slope[None, :] * wS / s0[:, None]",
     "out[:d] = disc * slope[None, :] * wS", [T + "test_oracle_factor.py"]),
    # statistics, discounting and schemes of the other pricers
    ("factor_average_count", "oracle.c",
     "ps.u_T = u; ps.avg = sum / steps; ps.umax = umax; ps.umin = umin;\n"
     "            for (int p = 0; p < npay; ++p) out[(size_t)p * npaths + n]",
     "ps.u_T = u; ps.avg = sum / (steps + 1); ps.umax = umax; ps.umin = umin;\n"
     "            for (int p = 0; p < npay; ++p) out[(size_t)p * npaths + n]", [T + "test_oracle_factor.py"]),
    ("qmc_average_count", "oracle.c",
     "ps.u_T = u; ps.avg = sum / steps; ps.umax = umax; ps.umin = umin;\n"
     "        for (int p = 0; p < npay; ++p) out[(size_t)p * npts + i]",
     "ps.u_T = u; ps.avg = sum / (steps + 1); ps.umax = umax; ps.umin = umin;\n"
     "        for (int p = 0; p < npay; ++p) out[(size_t)p * npts + i]", [T + "test_oracle_qmc.py"]),
    ("qmc_discount_without_maturity", "oracle.c",
     "    const double dt = T / steps, sdt = sqrt(dt), disc = exp(-r * T);\n#pragma omp parallel for schedule(static)\n"
     "    for (int64_t i = 0; i < npts; ++i) {",
     "    const double dt = T / steps, sdt = sqrt(dt), disc = exp(-r);\n#pragma omp parallel for schedule(static)\n"
     "    for (int64_t i = 0; i < npts; ++i) {", [T + "test_oracle_qmc.py"]),
    ("qmc_euler_drift_dropped", "oracle.c",
     "                else x[a] *= 1.0 + r * dt + dW;\n                u += w[a] * ((scheme == 0) ? exp(x[a]) : x[a]);\n"
     "            }\n            sum += u;",
     "                else x[a] *= 1.0 + dW;\n                u += w[a] * ((scheme == 0) ? exp(x[a]) : x[a]);\n"
     "            }\n            sum += u;", [T + "test_oracle_qmc.py"]),
    ("heston_average_count", "oracle.c", "if (stats) { stats->u_T = S; stats->avg = sum / M;",
     "if (stats) { stats->u_T = S; stats->avg = sum / (M + 1);", [T + "test_oracle_heston.py", T + "test_oracle_greeks.py"]),
    ("heston_drift_rate_dropped", "oracle.c", "double xn = x + (h->r - 0.5 * vp) * dt + sq * c;",
     "double xn = x + (-0.5 * vp) * dt + sq * c;", [T + "test_oracle_heston.py"]),
    ("heston_maximum_is_terminal", "oracle.c", "if (S > umax) umax = S;", "umax = S;", [T + "test_oracle_heston.py"]),
    ("bridge_maximum_unweighted", "oracle.c", "ps.umax = w * exp(mmax);", "ps.umax = exp(mmax);",
     [T + "test_oracle_bridge.py"]),
    ("bridge_minimum_unweighted", "oracle.c", "ps.umin = w * exp(mmin);", "ps.umin = exp(mmin);",
     [T + "test_oracle_bridge.py"]),
    ("saved_start_first_asset", "oracle.c", "for (int a = 0; a < d; ++a) save[(size_t)a * ld + col] = m->s0[a];",
     "for (int a = 0; a < d; ++a) save[(size_t)a * ld + col] = m->s0[0];", [T + "test_oracle_gbm.py"]),
    ("estimator_single_sample_error", "oracle.c", "*se = n > 1 ? sqrt(", "*se = n > 0 ? sqrt(",
     [T + "test_oracle_gbm.py"]),
    ("rho_greek_payoff_kind", "oracle.c",
     "double f = payoff_value(kind[p], strike[p], 0.0, &ps);\n                int asian",
     "double f = payoff_value(ORC_CALL, strike[p], 0.0, &ps);\n                int asian", [T + "test_oracle_greeks.py"]),
    ("corr_tangent_time_scale", "oracle.c",
     "for (int b = 0; b <= a; ++b) t[(size_t)a * (a + 1) / 2 + b] += sdt * sig[a] * z[b];\n                }\n"
     "            }\n            for",
     "for (int b = 0; b <= a; ++b) t[(size_t)a * (a + 1) / 2 + b] += dt * sig[a] * z[b];\n                }\n"
     "            }\n            for", [T + "test_oracle_corr.py"]),
    # nested revaluation, scenarios and labels: streams and payoffs
    ("nested_knock_at_start_dropped", "oracle.c", "if (kind == ORC_UO_CALL && S >= H) return 0.0;",
     "if (kind == ORC_UO_CALL && S > 2 * H) return 0.0;", [T + "test_oracle_risk.py::test_nested_value_is_black_scholes"]),
    ("nested_put_pays_call", "oracle.c", "if (kind == ORC_PUT) f = K > ST ? K - ST : 0.0;",
     "if (kind == ORC_PUT) f = ST > K ? ST - K : 0.0;", [T + "test_oracle_risk.py::test_nested_value_is_black_scholes"]),
    ("nested_paths_share_a_stream", "oracle.c", "stream_init(&st, seed, domain_tag(domain, base | (uint64_t)p));",
     "stream_init(&st, seed, domain_tag(domain, base));", [T + "test_oracle_risk.py::test_nested_value_is_black_scholes"]),
    ("scenarios_share_a_stream", "oracle.c", "stream_init(&st, seed, domain_tag(2, (uint64_t)s));",
     "stream_init(&st, seed, domain_tag(2, 0));", [T + "test_oracle_risk.py::test_scenario_moments"]),
    ("label_points_share_streams", "oracle.c", "4, (uint64_t)p << 16);", "4, 0);", [T + "test_oracle_risk.py"]),
    ("label_vega_sums_squares", "oracle.c", "                zs += z;", "                zs += z * z;",
     [T + "test_oracle_risk.py::test_label_greeks_pins"]),
    # payoff kinds, slopes and barrier conventions
    ("down_out_call_watches_the_maximum", "oracle.c", "case ORC_DO_CALL: return down_hit ? 0.0 : call;",
     "case ORC_DO_CALL: return up_hit ? 0.0 : call;", [T + "test_oracle_gbm.py", T + "test_oracle_bridge.py"]),
    ("up_out_put_watches_the_minimum", "oracle.c", "case ORC_UO_PUT: return up_hit ? 0.0 : put;",
     "case ORC_UO_PUT: return down_hit ? 0.0 : put;", [T + "test_oracle_gbm.py", T + "test_oracle_bridge.py"]),
    ("down_in_put_pays_call", "oracle.c", "case ORC_DI_PUT: return down_hit ? put : 0.0;",
     "case ORC_DI_PUT: return down_hit ? call : 0.0;", [T + "test_oracle_gbm.py", T + "test_oracle_bridge.py"]),
    ("asian_put_on_terminal", "oracle.c", "case ORC_ASIAN_PUT: return K > p->avg ? K - p->avg : 0.0;",
     "case ORC_ASIAN_PUT: return K > p->u_T ? K - p->u_T : 0.0;",
     [T + "test_oracle_gbm.py", T + "test_oracle_greeks.py", T + "test_oracle_corr.py"]),
    ("up_barrier_needs_a_margin", "oracle.c", "int up_hit = p->umax >= H,", "int up_hit = p->umax > H * (1 + 1e-3),",
     [T + "test_oracle_gbm.py"]),
    ("asian_slope_on_terminal", "oracle.c", "case ORC_ASIAN_CALL: return p->avg > K ? 1.0 : 0.0;",
     "case ORC_ASIAN_CALL: return p->u_T > K ? 1.0 : 0.0;", [T + "test_oracle_greeks.py"]),
    ("put_slope_sign", "oracle.c", "case ORC_PUT: return K > p->u_T ? -1.0 : 0.0;",
     "case ORC_PUT: return K > p->u_T ? 1.0 : 0.0;", [T + "test_oracle_greeks.py"]),
    # set-up, tangents, Sobol and Heston details
    ("cholesky_accepts_indefinite", "oracle.c", "if (!(s > 0.0)) return -1;", "if (!(s > -1.0)) return -1;",
     [T + "test_oracle_gbm.py::test_cholesky_rejects_what_lapack_rejects"]),
    ("identity_factor_scaled", "oracle.c", "for (int a = 0; a < d; ++a) m->Lrho[(size_t)a * d + a] = 1.0;",
     "for (int a = 0; a < d; ++a) m->Lrho[(size_t)a * d + a] = 1.0 + (a > 0);", [T + "test_oracle_gbm.py"]),
    ("euler_delta_tangent_not_grown", "oracle.c", "tg->tS0[a] = tg->tS0[a] * g;", "tg->tS0[a] = tg->tS0[a];",
     [T + "test_oracle_greeks.py"]),
    ("euler_rho_tangent_not_grown", "oracle.c", "tg->tr[a] = tg->tr[a] * g + x[a] * dt;",
     "tg->tr[a] = tg->tr[a] + x[a] * dt;", [T + "test_oracle_greeks.py"]),
    ("factor_terminal_prices_as_logs", "oracle.c",
     "for (int a = 0; a < d; ++a) ST[(size_t)a * npaths + n] = (scheme == 0) ? exp(x[a]) : x[a];",
     "for (int a = 0; a < d; ++a) ST[(size_t)a * npaths + n] = exp(x[a]);", [T + "test_oracle_factor.py"]),
    ("primitivity_test_incomplete", "oracle.c", "        if (gf2_xpow_mod(order / q, p, s) == 1) return 0;\n", "",
     [T + "test_oracle_qmc.py"]),
    ("qmc_shift_one_lane", "oracle.c",
     "for (int l = 0; l < 4 && 4 * q + l < ndim; ++l) shift[4 * q + l] = x[l];",
     "for (int l = 0; l < 4 && 4 * q + l < ndim; ++l) shift[4 * q + l] = x[0];", [T + "test_oracle_qmc.py"]),
    ("qmc_second_uniform_dimension", "oracle.c",
     "const double u2 = orc_uniform(sobol_word(V + (size_t)(2 * jn + 1) * 32, (uint64_t)(n0 + i))",
     "const double u2 = orc_uniform(sobol_word(V + (size_t)(2 * jn) * 32, (uint64_t)(n0 + i))",
     [T + "test_oracle_qmc.py"]),
    ("qmc_point_offset_ignored", "oracle.c",
     "sobol_word(V + (size_t)(2 * jn) * 32, (uint64_t)(n0 + i)) ^ shift[2 * jn]);",
     "sobol_word(V + (size_t)(2 * jn) * 32, (uint64_t)(i)) ^ shift[2 * jn]);",
     [T + "test_oracle_qmc.py::test_point_offset_selects_points"]),
    ("heston_correlated_noise_swapped", "oracle.c", "double c = h->rho * z1 + rc * z2;",
     "double c = h->rho * z2 + rc * z1;", [T + "test_oracle_heston.py"]),
    ("heston_drift_untruncated_variance", "oracle.c",
     "double vn = v + h->kappa * (h->theta - vp) * dt + h->xi * sq * z1;",
     "double vn = v + h->kappa * (h->theta - v) * dt + h->xi * sq * z1;",
     [T + "test_oracle_heston.py", T + "test_oracle_greeks.py"]),
    ("nested_barrier_margin", "oracle.c", "if (kind == ORC_UO_CALL && exp(mx) >= H) f = 0.0;",
     "if (kind == ORC_UO_CALL && exp(mx) > H * 1.01) f = 0.0;",
     [T + "test_oracle_risk.py::test_nested_up_and_out_monitors_every_step"]),
    ("corr_chain_includes_diagonal", "__init__.py", "pairs = [(a, b) for a in range(d) for b in range(a)]",
     "pairs = [(a, b) for a in range(d) for b in range(a + 1)]", [T + "test_oracle_corr.py"]),
    ("corr_asian_payoff_undiscounted", "__init__.py", "return dict(f=disc * f, U=A, dl=dl, drho=corr_chain(corr, dl))",
     "return dict(f=f, U=A, dl=dl, drho=corr_chain(corr, dl))", [T + "test_oracle_corr.py"]),
    ("factor_greeks_discount_maturity", "__init__.py", "    disc = np.exp(-r * T)\n    U = w @ ST",
     "    disc = np.exp(-r)\n    U = w @ ST", [T + "test_oracle_factor.py"]),
    # surrogate network, loss and optimiser
    ("mlp_activation_derivative_dropped", "mlp.py", "dz = dh if l == len(params) - 1 else dh * silu_grad(z)",
     "dz = dh", [T + "test_oracle_mlp.py"]),
    ("mlp_bias_gradient_mean", "mlp.py", "grads[l] = (h.T @ dz, dz.sum(axis=0))",
     "grads[l] = (h.T @ dz, dz.mean(axis=0))", [T + "test_oracle_mlp.py"]),
    ("silu_derivative_sign", "mlp.py", "return s * (1.0 + z * (1.0 - s))", "return s * (1.0 - z * (1.0 - s))",
     [T + "test_oracle_mlp.py"]),
    ("silu_second_derivative_term", "mlp.py", "(2.0 + z * (1.0 - 2.0 * s))", "(2.0 + z * (1.0 - s))",
     [T + "test_oracle_mlp.py"]),
    ("derivative_loss_second_order_dropped", "mlp.py",
     "zbar = hbar * silu_grad(z) + sum(dhbar[k] * silu_grad2(z) * dzs[l - 1][k] for k in range(K))",
     "zbar = hbar * silu_grad(z)", [T + "test_oracle_mlp.py"]),
    ("derivative_loss_tangent_weight_gradient_dropped", "mlp.py",
     "gW = hs[l].T @ zbar + sum(dhs[l][k].T @ dzbar[k] for k in range(K))", "gW = hs[l].T @ zbar",
     [T + "test_oracle_mlp.py"]),
    ("derivative_loss_seed_halved", "mlp.py",
     "dzbar = np.stack([(2.0 * lams[k] / n) * rd[k][:, None] for k in range(K)]) if K else np.zeros((0, n, 1))",
     "dzbar = np.stack([(lams[k] / n) * rd[k][:, None] for k in range(K)]) if K else np.zeros((0, n, 1))",
     [T + "test_oracle_mlp.py"]),
    ("input_tangent_activation_dropped", "mlp.py", "hh, dh = silu(z), silu_grad(z) * dz", "hh, dh = silu(z), dz",
     [T + "test_oracle_mlp.py"]),
    ("output_layer_activated", "mlp.py", "        h = silu(z) if l < len(params) - 1 else z\n", "        h = silu(z)\n",
     [T + "test_oracle_mlp.py"]),
    ("input_tangent_takes_bias", "mlp.py", "            dz = dh @ W\n            if l < len(params) - 1:",
     "            dz = dh @ W + b\n            if l < len(params) - 1:", [T + "test_oracle_mlp.py"]),
    ("derivative_labels_unmasked", "mlp.py", "r, rd = y - t, m * (dy - gz)", "r, rd = y - t, (dy - gz)",
     [T + "test_oracle_mlp.py"]),
    ("bias_gradient_takes_tangents", "mlp.py", "        grads[l] = (gW, zbar.sum(axis=0))\n        if l == 0:",
     "        grads[l] = (gW, zbar.sum(axis=0) + dzbar.sum(axis=(0, 1)))\n        if l == 0:",
     [T + "test_oracle_mlp.py"]),
    ("adam_bias_correction_dropped", "mlp.py", "mh = m2 / (1 - beta1 ** step)", "mh = m2",
     [T + "test_oracle_mlp.py"]),
    ("adam_denominator_without_root", "mlp.py", "new.append((p_ - lr * mh / (np.sqrt(vh) + eps), m2, v2))",
     "new.append((p_ - lr * mh / (vh + eps), m2, v2))", [T + "test_oracle_mlp.py"]),
    ("unpack_bias_offset", "mlp.py", "        bb = np.asarray(flat[o:o + b], dtype=np.float64)\n        o += b",
     "        bb = np.asarray(flat[o:o + b], dtype=np.float64)\n        o += 0", [T + "test_oracle_mlp.py"]),
    ("adam_second_moment_correction_dropped", "mlp.py", "vh = v2 / (1 - beta2 ** step)", "vh = v2",
     [T + "test_oracle_mlp.py"]),
]


def _copy(dst, mutant=None):
    src = os.path.join(ROOT, "oracle")
    out = os.path.join(dst, "oracle")
    os.makedirs(out)
    for name in ("__init__.py", "oracle.c", "mlp.py", "risk.py"):
        shutil.copyfile(os.path.join(src, name), os.path.join(out, name))
    if mutant is not None:
        _, fname, old, new, _ = mutant
        path = os.path.join(out, fname)
        text = open(path).read()
        assert text.count(old) == 1, f"{mutant[0]}: the text to change must occur once in {fname}"
        open(path, "w").write(text.replace(old, new))
    return out


def _run_pins(alt_dir, targets):
    env = dict(os.environ, GBMC_ORACLE_DIR=alt_dir, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *targets, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    summary = out.strip().splitlines()[-1] if out.strip() else ""
    return r.returncode, summary, out


def _case(mutant):
    with tempfile.TemporaryDirectory(prefix="orc_mutant_") as tmp:
        pkg = _copy(tmp, mutant)
        rc, summary, out = _run_pins(tmp, mutant[4])
        built = mutant[1] != "oracle.c" or os.path.exists(os.path.join(pkg, "liboracle.so"))
        return mutant[0], rc, summary, built, out


def test_every_planted_mistake_fails_a_pin():
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    # control: the unchanged copy passes every pin the mutants use (run
    # beside the planted copies)
    targets = sorted({t.split("::")[0] for m in MUTANTS for t in m[4]})

    def control():
        with tempfile.TemporaryDirectory(prefix="orc_control_") as tmp:
            _copy(tmp)
            return _run_pins(tmp, targets)

    with cf.ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        ctl = ex.submit(control)
        results = list(ex.map(_case, MUTANTS))
        rc, summary, out = ctl.result()
    assert rc == 0, "control copy fails its pins:\n" + out[-3000:]
    survivors = []
    for name, rc, summary, built, out in results:
        assert built, f"{name}: the planted copy did not build\n{out[-2000:]}"
        caught = rc == 1 and re.search(r"\b\d+ failed\b", summary) and "error" not in summary
        print(f"{name:40s} {'caught' if caught else 'SURVIVED'}: {summary}")
        if not caught:
            survivors.append((name, summary))
    assert not survivors, survivors
