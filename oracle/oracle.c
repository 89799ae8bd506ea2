/*
 * FP64 CPU oracle for the Monte Carlo method of "Tensor Processing Units for
 * Financial Monte Carlo" (Belletti et al., 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the library never links, calls or falls back to it, and it includes no header
 * of the library.  Every floating-point quantity is IEEE double; no blocking,
 * fusion or reordering beyond what each cited passage states.
 *
 * Parity status: every function below is pinned by the tests listed in the
 * oracle package docstring, except orc_heston_* whose pins are the xi = 0
 * Black-Scholes reduction and finite differences (no closed form at xi > 0).
 *
 * Random stream (the paper fixes the generator family, Sec. IV.A, not the
 * layout; the layout below is this library's convention):
 *   key     = (seed mod 2^32, seed div 2^32)
 *   normal j of stream s is produced from Philox4x32-10 block q = j div 4 at
 *   counter (q mod 2^32, q div 2^32, s mod 2^32, s div 2^32), lane j mod 4;
 *   lanes (0,1) and (2,3) form Box-Muller pairs.
 *   Uniform map U(x) = (floor(x / 2^9) + 1/2) * 2^-23, which is exact in both
 *   binary32 and binary64 and lies in [2^-24, 1 - 2^-24].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: the keyed, multi-stream generator named for GPUs in       */
/* Sec. IV.A (Salmon et al., SC'11, whose published round function this is). */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from one 32-bit word, exact in binary32 and binary64. */
double orc_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); /* 2^-23 */
}

/* Normal number j of stream `stream` under key `seed` (Box-Muller on the pair of
 * uniforms that shares j's block; the transform the paper uses in Sec. VI.D). */
typedef struct {
    uint64_t seed, stream;
    uint64_t cached_q;
    int have;
    double z[4];
} orc_stream;

static void stream_init(orc_stream *s, uint64_t seed, uint64_t stream)
{
    s->seed = seed; s->stream = stream; s->have = 0; s->cached_q = 0;
}

static double stream_normal(orc_stream *s, uint64_t j)
{
    uint64_t q = j >> 2;
    if (!s->have || s->cached_q != q) {
        uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)s->stream, (uint32_t)(s->stream >> 32)};
        uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = orc_uniform(x[2 * pair]);
            double u2 = orc_uniform(x[2 * pair + 1]);
            double rad = sqrt(-2.0 * log(u1));
            s->z[2 * pair] = rad * cos(2.0 * M_PI * u2);
            s->z[2 * pair + 1] = rad * sin(2.0 * M_PI * u2);
        }
        s->cached_q = q; s->have = 1;
    }
    return s->z[j & 3];
}

void orc_normals(uint64_t seed, uint64_t stream, uint64_t j0, int64_t count, double *z)
{
    orc_stream s;
    stream_init(&s, seed, stream);
    for (int64_t k = 0; k < count; ++k) z[k] = stream_normal(&s, j0 + (uint64_t)k);
}

/* ------------------------------------------------------------------------ */
/* Cholesky factor L with L L^T = A (Sec. II.A.3 uses it for the Grammian;   */
/* here it factors the asset correlation so that L z has covariance A).      */
/* Plain Cholesky-Banachiewicz; returns 0, or -1 if A is not positive        */
/* definite.  A and L are row-major d x d; the upper triangle of L is zero.  */
/* ------------------------------------------------------------------------ */
int orc_cholesky(int d, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)d * (size_t)d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[(size_t)i * d + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * d + k] * L[(size_t)j * d + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[(size_t)i * d + i] = sqrt(s);
            } else {
                L[(size_t)i * d + j] = s / L[(size_t)j * d + j];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Payoffs on the monitored underlying U(t_i), i = 1..M (Sec. I.A.2: path-   */
/* dependent outcomes f(X_{0:T}); barrier and Asian options).                */
/* ------------------------------------------------------------------------ */
enum {
    ORC_CALL = 0, ORC_PUT = 1, ORC_ASIAN_CALL = 2, ORC_ASIAN_PUT = 3,
    ORC_UO_CALL = 4, ORC_UI_CALL = 5, ORC_UO_PUT = 6, ORC_UI_PUT = 7,
    ORC_DO_CALL = 8, ORC_DI_CALL = 9, ORC_DO_PUT = 10, ORC_DI_PUT = 11
};

typedef struct {
    double u_T;   /* U(t_M) */
    double avg;   /* (1/M) sum_{i=1..M} U(t_i) */
    double umax;  /* max_{i=1..M} U(t_i) */
    double umin;  /* min_{i=1..M} U(t_i) */
} orc_pathstats;

static double payoff_value(int kind, double K, double H, const orc_pathstats *p)
{
    double call = p->u_T > K ? p->u_T - K : 0.0;
    double put = K > p->u_T ? K - p->u_T : 0.0;
    int up_hit = p->umax >= H, down_hit = p->umin <= H;
    switch (kind) {
    case ORC_CALL: return call;
    case ORC_PUT: return put;
    case ORC_ASIAN_CALL: return p->avg > K ? p->avg - K : 0.0;
    case ORC_ASIAN_PUT: return K > p->avg ? K - p->avg : 0.0;
    case ORC_UO_CALL: return up_hit ? 0.0 : call;
    case ORC_UI_CALL: return up_hit ? call : 0.0;
    case ORC_UO_PUT: return up_hit ? 0.0 : put;
    case ORC_UI_PUT: return up_hit ? put : 0.0;
    case ORC_DO_CALL: return down_hit ? 0.0 : call;
    case ORC_DI_CALL: return down_hit ? call : 0.0;
    case ORC_DO_PUT: return down_hit ? 0.0 : put;
    case ORC_DI_PUT: return down_hit ? put : 0.0;
    default: return NAN;
    }
}

/* Derivative of the undiscounted payoff with respect to the quantity it is
 * written on (u_T for European kinds, avg for Asian kinds); the indicator
 * convention d/dx (x-K)^+ = 1{x > K}.  Barrier kinds have no pathwise
 * derivative (the knock indicator is discontinuous): returns NAN. */
static double payoff_slope(int kind, double K, const orc_pathstats *p)
{
    switch (kind) {
    case ORC_CALL: return p->u_T > K ? 1.0 : 0.0;
    case ORC_PUT: return K > p->u_T ? -1.0 : 0.0;
    case ORC_ASIAN_CALL: return p->avg > K ? 1.0 : 0.0;
    case ORC_ASIAN_PUT: return K > p->avg ? -1.0 : 0.0;
    default: return NAN;
    }
}

static int payoff_is_asian(int kind) { return kind == ORC_ASIAN_CALL || kind == ORC_ASIAN_PUT; }

/* ------------------------------------------------------------------------ */
/* Correlated geometric Brownian motion, d >= 1 assets (Eq. 1 with           */
/* mu(X) = r X and sigma(X) = diag(X) diag(sig) Lrho; the multivariate       */
/* Euler-Maruyama step of Sec. II.A.2, which for d = 1 is the scalar step of  */
/* Sec. II.A.1).  scheme 0: log-Euler on log S; scheme 1: Euler on S.         */
/*   dW_a = sqrt(Delta) * sig_a * sum_{k<=a} Lrho[a][k] z_k,  z = normals     */
/*          i*d .. i*d+d-1 of stream path0+n.                                */
/*   log-Euler: x_a += (r - sig_a^2/2) Delta + dW_a                          */
/*   Euler:     S_a += S_a (r Delta + dW_a)                                   */
/* U(t) = sum_a w_a S_a(t).                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int d;
    const double *s0, *sig, *w;
    double *Lrho; /* d x d */
    double r, T;
    int steps, scheme;
    uint64_t seed;
} orc_gbm;

static int gbm_setup(orc_gbm *m, int d, const double *s0, const double *sig, const double *corr,
                     const double *w, double r, double T, int steps, int scheme, uint64_t seed)
{
    m->d = d; m->s0 = s0; m->sig = sig; m->w = w; m->r = r; m->T = T;
    m->steps = steps; m->scheme = scheme; m->seed = seed;
    m->Lrho = (double *)malloc(sizeof(double) * (size_t)d * (size_t)d);
    if (!m->Lrho) return -3;
    if (corr) {
        if (orc_cholesky(d, corr, m->Lrho) != 0) { free(m->Lrho); return -2; }
    } else {
        memset(m->Lrho, 0, sizeof(double) * (size_t)d * (size_t)d);
        for (int a = 0; a < d; ++a) m->Lrho[(size_t)a * d + a] = 1.0;
    }
    return 0;
}

/* Simulate one path.  Optional outputs:
 *   save: [n_saved][d][ld] prices at steps 0, save_every, 2 save_every, ..., M
 *   S_T:  [d] terminal prices;  stats: monitored statistics of U.
 *   tangents (Greeks, forward mode): per asset a, dS_a/dS0_a, dS_a/dsig_a,
 *   dS_a/dr at the end (tS0, tsig, tr) and their (1/M) sum over i = 1..M of
 *   w_a * tangent (aS0, asig, ar) for the Asian average. */
typedef struct {
    double *tS0, *tsig, *tr;   /* [d] terminal tangents of S_a */
    double *aS0, *asig, *ar;   /* [d] tangents of the Asian average */
} orc_tangents;

static void gbm_path(const orc_gbm *m, int64_t n, double *save, int64_t col, int save_every, int64_t ld,
                     double *S_T, orc_pathstats *stats, orc_tangents *tg,
                     double *work /* 3*d */)
{
    const int d = m->d, M = m->steps;
    const double dt = m->T / M, sdt = sqrt(dt);
    double *x = work, *z = work + d, *y = work + 2 * d; /* state, normals, Lrho z */
    orc_stream st;
    stream_init(&st, m->seed, (uint64_t)n);
    for (int a = 0; a < d; ++a) x[a] = (m->scheme == 0) ? log(m->s0[a]) : m->s0[a];
    if (tg) {
        for (int a = 0; a < d; ++a) {
            /* log-Euler tangents are of x = log S; Euler tangents are of S. */
            tg->tS0[a] = (m->scheme == 0) ? 1.0 / m->s0[a] : 1.0;
            tg->tsig[a] = 0.0; tg->tr[a] = 0.0;
            tg->aS0[a] = 0.0; tg->asig[a] = 0.0; tg->ar[a] = 0.0;
        }
    }
    if (save) {
        for (int a = 0; a < d; ++a) save[(size_t)a * ld + col] = m->s0[a];
    }
    double sum = 0.0, umax = -INFINITY, umin = INFINITY, u = 0.0;
    for (int i = 0; i < M; ++i) {
        for (int a = 0; a < d; ++a) z[a] = stream_normal(&st, (uint64_t)i * d + a);
        for (int a = 0; a < d; ++a) {
            double s = 0.0;
            for (int k = 0; k <= a; ++k) s += m->Lrho[(size_t)a * d + k] * z[k];
            y[a] = s;
        }
        for (int a = 0; a < d; ++a) {
            double dW = sdt * m->sig[a] * y[a];
            if (m->scheme == 0) {
                x[a] += (m->r - 0.5 * m->sig[a] * m->sig[a]) * dt + dW;
                if (tg) {
                    tg->tsig[a] += -m->sig[a] * dt + sdt * y[a];
                    tg->tr[a] += dt;
                }
            } else {
                double g = 1.0 + m->r * dt + dW;
                if (tg) {
                    tg->tS0[a] = tg->tS0[a] * g;
                    tg->tsig[a] = tg->tsig[a] * g + x[a] * sdt * y[a];
                    tg->tr[a] = tg->tr[a] * g + x[a] * dt;
                }
                x[a] = x[a] * g;
            }
        }
        u = 0.0;
        for (int a = 0; a < d; ++a) {
            double Sa = (m->scheme == 0) ? exp(x[a]) : x[a];
            u += m->w[a] * Sa;
            if (tg) {
                /* dS_a/dp = S_a dx_a/dp for log-Euler, the tangent itself for Euler */
                double f = (m->scheme == 0) ? Sa : 1.0;
                tg->aS0[a] += m->w[a] * f * tg->tS0[a] / M;
                tg->asig[a] += m->w[a] * f * tg->tsig[a] / M;
                tg->ar[a] += m->w[a] * f * tg->tr[a] / M;
            }
        }
        sum += u;
        if (u > umax) umax = u;
        if (u < umin) umin = u;
        if (save && save_every > 0 && (i + 1) % save_every == 0) {
            int slot = (i + 1) / save_every;
            for (int a = 0; a < d; ++a)
                save[((size_t)slot * d + a) * ld + col] = (m->scheme == 0) ? exp(x[a]) : x[a];
        }
    }
    for (int a = 0; a < d; ++a) {
        double Sa = (m->scheme == 0) ? exp(x[a]) : x[a];
        if (S_T) S_T[a] = Sa;
        if (tg && m->scheme == 0) {
            tg->tS0[a] *= Sa; tg->tsig[a] *= Sa; tg->tr[a] *= Sa;
        }
    }
    if (stats) {
        stats->u_T = u; stats->avg = sum / M; stats->umax = umax; stats->umin = umin;
    }
}

/* Discounted payoffs of every path: out[p * npaths + n], path index path0 + n.
 * Returns 0, -1 on bad arguments, -2 if corr is not positive definite. */
int orc_gbm_payoffs(int d, const double *s0, const double *sig, const double *corr, const double *w,
                    double r, double T, int steps, int scheme, uint64_t seed,
                    int64_t path0, int64_t npaths,
                    int npay, const int *kind, const double *strike, const double *barrier,
                    double *out)
{
    if (d < 1 || steps < 1 || npaths < 0 || !(T > 0.0) || (scheme != 0 && scheme != 1)) return -1;
    orc_gbm m;
    int rc = gbm_setup(&m, d, s0, sig, corr, w, r, T, steps, scheme, seed);
    if (rc) return rc;
    const double disc = exp(-r * T);
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);
#pragma omp for schedule(static)
        for (int64_t n = 0; n < npaths; ++n) {
            orc_pathstats ps;
            gbm_path(&m, path0 + n, NULL, 0, 0, 0, NULL, &ps, NULL, work);
            for (int p = 0; p < npay; ++p)
                out[(size_t)p * npaths + n] = disc * payoff_value(kind[p], strike[p], barrier[p], &ps);
        }
        free(work);
    }
    free(m.Lrho);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-asset GBM with continuously monitored barriers through the         */
/* Brownian bridge (Sec. VI.A.1, the "In and Out Put" experiment).  log-Euler */
/* on x = log S (exact in law at the grid); between consecutive grid values   */
/* x = x_i and y = x_{i+1} the maximum of the bridge of log S is drawn as     */
/*   m_i = (x + y + sqrt((x - y)^2 - 2 dt sig^2 ln U_i)) / 2                 */
/* and the minimum as (x + y - sqrt((x - y)^2 - 2 dt sig^2 ln V_i)) / 2; the  */
/* path's maximum (minimum) over [0, T] is the largest m_i (smallest).        */
/* U_i, V_i: uniforms 2i and 2i + 1 of stream 2^56 + n (the bridge domain of  */
/* path n), from the same Philox blocks and uniform map as the normals.       */
/* The monitored underlying is U = w S.                                       */
/* ------------------------------------------------------------------------ */
static double bridge_uniform(uint64_t seed, uint64_t stream, uint64_t j)
{
    uint64_t q = j >> 2;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    return orc_uniform(x[j & 3]);
}

int orc_gbm1d_bridge_payoffs(double s0, double sig, double w, double r, double T, int steps, uint64_t seed,
                             int64_t path0, int64_t npaths, int npay, const int *kind, const double *strike,
                             const double *barrier, double *out)
{
    if (steps < 1 || npaths < 0 || !(T > 0.0) || !(s0 > 0.0) || !(sig >= 0.0)) return -1;
    const double dt = T / steps, sdt = sqrt(dt), disc = exp(-r * T);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < npaths; ++n) {
        const uint64_t path = (uint64_t)(path0 + n);
        const uint64_t bstream = ((uint64_t)1 << 56) | path;
        orc_stream st;
        stream_init(&st, seed, path);
        double x = log(s0), sum = 0.0, mmax = -INFINITY, mmin = INFINITY;
        for (int i = 0; i < steps; ++i) {
            const double z = stream_normal(&st, (uint64_t)i);
            const double y = x + (r - 0.5 * sig * sig) * dt + sig * sdt * z;
            const double Ui = bridge_uniform(seed, bstream, 2 * (uint64_t)i);
            const double Vi = bridge_uniform(seed, bstream, 2 * (uint64_t)i + 1);
            const double hi = 0.5 * (x + y + sqrt((x - y) * (x - y) - 2.0 * dt * sig * sig * log(Ui)));
            const double lo = 0.5 * (x + y - sqrt((x - y) * (x - y) - 2.0 * dt * sig * sig * log(Vi)));
            if (hi > mmax) mmax = hi;
            if (lo < mmin) mmin = lo;
            x = y;
            sum += w * exp(x);
        }
        orc_pathstats ps;
        ps.u_T = w * exp(x);
        ps.avg = sum / steps;
        ps.umax = w * exp(mmax);
        ps.umin = w * exp(mmin);
        for (int p = 0; p < npay; ++p)
            out[(size_t)p * npaths + n] = disc * payoff_value(kind[p], strike[p], barrier[p], &ps);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Factor-model correlated GBM: the correlation is rho = B B^T + diag(e^2)    */
/* with loadings B (d x k) and idiosyncratic weights e_a = sqrt(1 - sum_j    */
/* B_aj^2), and the increment of step i is                                   */
/*   dW_a = sqrt(dt) sig_a (sum_j B_aj z_j + e_a eps_a),                      */
/* z_j = normal i (k + d) + j, eps_a = normal i (k + d) + k + a of the path's */
/* stream (O(d k) per step instead of the Cholesky O(d^2); exact in law).     */
/* Otherwise the step, statistics and payoffs of gbm_path.  Discounted        */
/* payoffs out[p * npaths + n]; terminal prices ST[a * npaths + n] if ST.     */
/* ------------------------------------------------------------------------ */
int orc_gbm_factor_payoffs(int d, int k, const double *s0, const double *sig, const double *B, const double *w,
                           double r, double T, int steps, int scheme, uint64_t seed, int64_t path0, int64_t npaths,
                           int npay, const int *kind, const double *strike, const double *barrier, double *out,
                           double *ST)
{
    if (d < 1 || k < 0 || steps < 1 || npaths < 0 || !(T > 0.0) || (scheme != 0 && scheme != 1)) return -1;
    double *e = (double *)malloc(sizeof(double) * (size_t)d);
    if (!e) return -3;
    for (int a = 0; a < d; ++a) {
        double q = 0.0;
        for (int j = 0; j < k; ++j) q += B[(size_t)a * k + j] * B[(size_t)a * k + j];
        if (q > 1.0 + 1e-12) { free(e); return -2; }
        e[a] = sqrt(q < 1.0 ? 1.0 - q : 0.0);
    }
    const double dt = T / steps, sdt = sqrt(dt), disc = exp(-r * T);
    int bad = 0;
#pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * (size_t)(2 * d + k + 1));
        if (!x) bad = 1;
#pragma omp for schedule(static)
        for (int64_t n = 0; n < npaths; ++n) {
            if (!x) continue;
            double *eps = x + d, *z = x + 2 * d;
            orc_stream st;
            stream_init(&st, seed, (uint64_t)(path0 + n));
            for (int a = 0; a < d; ++a) x[a] = (scheme == 0) ? log(s0[a]) : s0[a];
            double sum = 0.0, umax = -INFINITY, umin = INFINITY, u = 0.0;
            for (int i = 0; i < steps; ++i) {
                const uint64_t base = (uint64_t)i * (uint64_t)(k + d);
                for (int j = 0; j < k; ++j) z[j] = stream_normal(&st, base + (uint64_t)j);
                for (int a = 0; a < d; ++a) eps[a] = stream_normal(&st, base + (uint64_t)k + (uint64_t)a);
                u = 0.0;
                for (int a = 0; a < d; ++a) {
                    double f = e[a] * eps[a];
                    for (int j = 0; j < k; ++j) f += B[(size_t)a * k + j] * z[j];
                    const double dW = sdt * sig[a] * f;
                    if (scheme == 0) x[a] += (r - 0.5 * sig[a] * sig[a]) * dt + dW;
                    else x[a] *= 1.0 + r * dt + dW;
                    u += w[a] * ((scheme == 0) ? exp(x[a]) : x[a]);
                }
                sum += u;
                if (u > umax) umax = u;
                if (u < umin) umin = u;
            }
            orc_pathstats ps;
            ps.u_T = u; ps.avg = sum / steps; ps.umax = umax; ps.umin = umin;
            for (int p = 0; p < npay; ++p) out[(size_t)p * npaths + n] = disc * payoff_value(kind[p], strike[p], barrier[p], &ps);
            if (ST)
                for (int a = 0; a < d; ++a) ST[(size_t)a * npaths + n] = (scheme == 0) ? exp(x[a]) : x[a];
        }
        free(x);
    }
    free(e);
    return bad ? -3 : 0;
}

/* ------------------------------------------------------------------------ */
/* Sobol sequence and randomised quasi-Monte Carlo (Sec. IV, QRNGs; the      */
/* basket experiment of Sec. VI.D).  Dimension 1 is the van der Corput       */
/* sequence (m_k = 1).  Dimension j >= 2 uses the (j-1)-th primitive         */
/* polynomial over GF(2), enumerated by degree s and then by its integer     */
/* value x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1, with initial m_1..m_s = 1   */
/* and the recurrence (Bratley-Fox)                                          */
/*   m_k = 2 a_1 m_{k-1} ^ 4 a_2 m_{k-2} ^ ... ^ 2^{s-1} a_{s-1} m_{k-s+1}   */
/*         ^ 2^s m_{k-s} ^ m_{k-s};                                           */
/* direction numbers V_k = m_k 2^{32-k}; point n (natural order) is the XOR  */
/* of V_{k+1} over the set bits k of n.  Replication r shifts every point of */
/* dimension j by the XOR of Philox word j of stream 6 * 2^56 + r (a random   */
/* digital shift).  Uniforms use the map of orc_uniform; normal a is the      */
/* cosine branch of Box-Muller on dimensions (2a, 2a + 1).                    */
/* ------------------------------------------------------------------------ */
#define ORC_SOBOL_MAX_DIM 64

static int gf2_degree(uint32_t p)
{
    int d = -1;
    while (p) { ++d; p >>= 1; }
    return d;
}

/* a * b mod p over GF(2); a, b of degree < s, p of degree s */
static uint32_t gf2_mulmod(uint32_t a, uint32_t b, uint32_t p, int s)
{
    uint64_t prod = 0;
    for (int i = 0; i < s; ++i)
        if ((b >> i) & 1) prod ^= (uint64_t)a << i;
    for (int i = 2 * s - 2; i >= s; --i)
        if ((prod >> i) & 1) prod ^= (uint64_t)p << (i - s);
    return (uint32_t)prod;
}

/* x^e mod p over GF(2) */
static uint32_t gf2_xpow_mod(uint64_t e, uint32_t p, int s)
{
    uint32_t r = 1, b = (s == 1) ? (2u ^ p) : 2u; /* x reduced mod p */
    for (; e; e >>= 1) {
        if (e & 1) r = gf2_mulmod(r, b, p, s);
        b = gf2_mulmod(b, b, p, s);
    }
    return r;
}

/* p primitive: x has multiplicative order exactly 2^s - 1 modulo p, i.e.
 * x^(2^s - 1) = 1 and x^((2^s - 1) / q) != 1 for every prime q dividing it. */
static int gf2_primitive(uint32_t p)
{
    const int s = gf2_degree(p);
    if (s < 1 || !(p & 1)) return 0;
    const uint64_t order = ((uint64_t)1 << s) - 1;
    if (gf2_xpow_mod(order, p, s) != 1) return 0;
    uint64_t n = order;
    for (uint64_t q = 2; q <= n; ++q) {
        if (n % q) continue;
        if (gf2_xpow_mod(order / q, p, s) == 1) return 0;
        while (n % q == 0) n /= q;
    }
    return 1;
}

/* Direction numbers V[j][k] (k = 0..31) of dimensions j = 0..ndim-1. */
int orc_sobol_directions(int ndim, uint32_t *V)
{
    if (ndim < 1 || ndim > ORC_SOBOL_MAX_DIM) return -1;
    for (int k = 0; k < 32; ++k) V[k] = (uint32_t)1 << (31 - k);
    uint32_t p = 2;
    for (int j = 1; j < ndim; ++j) {
        do { ++p; } while (!gf2_primitive(p));
        int s = gf2_degree(p);
        uint32_t m[33];
        for (int k = 1; k <= s && k <= 32; ++k) m[k] = 1;
        for (int k = s + 1; k <= 32; ++k) {
            uint32_t v = m[k - s] ^ (m[k - s] << s);
            for (int i = 1; i < s; ++i)
                if ((p >> (s - i)) & 1) v ^= m[k - i] << i; /* a_i = coefficient of x^{s-i} */
            m[k] = v;
        }
        for (int k = 1; k <= 32; ++k) V[(size_t)j * 32 + (k - 1)] = m[k] << (32 - k);
    }
    return 0;
}

static uint32_t sobol_word(const uint32_t *Vj, uint64_t n)
{
    uint32_t x = 0;
    for (int k = 0; n; ++k, n >>= 1) if (n & 1) x ^= Vj[k];
    return x;
}

int orc_sobol_points(int ndim, int64_t n0, int64_t npts, uint32_t *out /* [npts][ndim] */)
{
    uint32_t V[ORC_SOBOL_MAX_DIM * 32];
    if (orc_sobol_directions(ndim, V)) return -1;
    for (int64_t i = 0; i < npts; ++i)
        for (int j = 0; j < ndim; ++j) out[(size_t)i * ndim + j] = sobol_word(V + (size_t)j * 32, (uint64_t)(n0 + i));
    return 0;
}

/* Correlated GBM baskets on randomised Sobol points: replication `rep`,
 * points [n0, n0 + npts); 2 d steps <= 64 dimensions; the normal of step i,
 * asset a is normal i d + a of the point; otherwise the step, statistics and
 * payoffs of gbm_path (log-Euler or Euler).  Discounted payoffs
 * out[p * npts + i]. */
int orc_qmc_gbm_payoffs(int d, const double *s0, const double *sig, const double *corr, const double *w,
                        double r, double T, int steps, int scheme, uint64_t seed, int64_t rep, int64_t n0,
                        int64_t npts, int npay, const int *kind, const double *strike, const double *barrier,
                        double *out)
{
    const int ndim = 2 * d * steps;
    if (d < 1 || steps < 1 || ndim > ORC_SOBOL_MAX_DIM || npts < 0 || (scheme != 0 && scheme != 1)) return -1;
    orc_gbm m;
    int rc = gbm_setup(&m, d, s0, sig, corr, w, r, T, steps, scheme, seed);
    if (rc) return rc;
    uint32_t V[ORC_SOBOL_MAX_DIM * 32], shift[ORC_SOBOL_MAX_DIM];
    orc_sobol_directions(ndim, V);
    {
        const uint64_t stream = ((uint64_t)6 << 56) | (uint64_t)rep;
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int q = 0; q * 4 < ndim; ++q) {
            uint32_t ctr[4] = {(uint32_t)q, 0u, (uint32_t)stream, (uint32_t)(stream >> 32)}, x[4];
            orc_philox4x32_10(ctr, key, x);
            for (int l = 0; l < 4 && 4 * q + l < ndim; ++l) shift[4 * q + l] = x[l];
        }
    }
    const double dt = T / steps, sdt = sqrt(dt), disc = exp(-r * T);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npts; ++i) {
        double x[64], y[64], z[64];
        double sum = 0.0, umax = -INFINITY, umin = INFINITY, u = 0.0;
        for (int a = 0; a < d; ++a) x[a] = (scheme == 0) ? log(s0[a]) : s0[a];
        for (int st = 0; st < steps; ++st) {
            for (int a = 0; a < d; ++a) {
                const int jn = st * d + a;
                const double u1 = orc_uniform(sobol_word(V + (size_t)(2 * jn) * 32, (uint64_t)(n0 + i)) ^ shift[2 * jn]);
                const double u2 = orc_uniform(sobol_word(V + (size_t)(2 * jn + 1) * 32, (uint64_t)(n0 + i)) ^ shift[2 * jn + 1]);
                z[a] = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            }
            for (int a = 0; a < d; ++a) {
                double acc = 0.0;
                for (int k = 0; k <= a; ++k) acc += m.Lrho[(size_t)a * d + k] * z[k];
                y[a] = acc;
            }
            u = 0.0;
            for (int a = 0; a < d; ++a) {
                const double dW = sdt * sig[a] * y[a];
                if (scheme == 0) x[a] += (r - 0.5 * sig[a] * sig[a]) * dt + dW;
                else x[a] *= 1.0 + r * dt + dW;
                u += w[a] * ((scheme == 0) ? exp(x[a]) : x[a]);
            }
            sum += u;
            if (u > umax) umax = u;
            if (u < umin) umin = u;
        }
        orc_pathstats ps;
        ps.u_T = u; ps.avg = sum / steps; ps.umax = umax; ps.umin = umin;
        for (int p = 0; p < npay; ++p) out[(size_t)p * npts + i] = disc * payoff_value(kind[p], strike[p], barrier[p], &ps);
    }
    free(m.Lrho);
    return 0;
}

/* Materialised paths: save[(slot*d + a)*npaths + n] = S_a at step slot*save_every
 * (slot 0 is t_0), for n in [0, npaths), path index path0 + n. */
int orc_gbm_paths(int d, const double *s0, const double *sig, const double *corr, const double *w,
                  double r, double T, int steps, int scheme, uint64_t seed,
                  int64_t path0, int64_t npaths, int save_every, double *save)
{
    if (d < 1 || steps < 1 || npaths < 0 || !(T > 0.0) || save_every < 1 || steps % save_every) return -1;
    orc_gbm m;
    int rc = gbm_setup(&m, d, s0, sig, corr, w, r, T, steps, scheme, seed);
    if (rc) return rc;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);
#pragma omp for schedule(static)
        for (int64_t n = 0; n < npaths; ++n) {
            gbm_path(&m, path0 + n, save, n, save_every, npaths, NULL, NULL, NULL, work);
        }
        free(work);
    }
    free(m.Lrho);
    return 0;
}

/* Pathwise (infinitesimal perturbation) Greeks in forward mode (Sec. I.A.3,
 * Sec. VI.A.2 "Basket European option Delta"), per path, discounted:
 *   g[((p*(2d+1)) + k) * npaths + n],  k = 0..d-1: d/dS0_k,  k = d..2d-1:
 *   d/dsig_{k-d},  k = 2d: d/dr (includes the -T * discounted payoff term).
 * European and Asian kinds only; returns -4 for a barrier kind. */
int orc_gbm_greeks(int d, const double *s0, const double *sig, const double *corr, const double *w,
                   double r, double T, int steps, int scheme, uint64_t seed,
                   int64_t path0, int64_t npaths,
                   int npay, const int *kind, const double *strike,
                   double *g)
{
    if (d < 1 || steps < 1 || npaths < 0 || !(T > 0.0) || (scheme != 0 && scheme != 1)) return -1;
    for (int p = 0; p < npay; ++p)
        if (kind[p] > ORC_ASIAN_PUT || kind[p] < 0) return -4;
    orc_gbm m;
    int rc = gbm_setup(&m, d, s0, sig, corr, w, r, T, steps, scheme, seed);
    if (rc) return rc;
    const double disc = exp(-r * T);
    const int ng = 2 * d + 1;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 9 * (size_t)d);
        orc_tangents tg = {work + 3 * d, work + 4 * d, work + 5 * d, work + 6 * d, work + 7 * d, work + 8 * d};
#pragma omp for schedule(static)
        for (int64_t n = 0; n < npaths; ++n) {
            orc_pathstats ps;
            gbm_path(&m, path0 + n, NULL, 0, 0, 0, NULL, &ps, &tg, work);
            for (int p = 0; p < npay; ++p) {
                double slope = payoff_slope(kind[p], strike[p], &ps);
                double f = payoff_value(kind[p], strike[p], 0.0, &ps);
                int asian = payoff_is_asian(kind[p]);
                double dr = 0.0;
                for (int a = 0; a < d; ++a) {
                    double dS0 = asian ? tg.aS0[a] : m.w[a] * tg.tS0[a];
                    double dsg = asian ? tg.asig[a] : m.w[a] * tg.tsig[a];
                    dr += asian ? tg.ar[a] : m.w[a] * tg.tr[a];
                    g[((size_t)p * ng + a) * npaths + n] = disc * slope * dS0;
                    g[((size_t)p * ng + d + a) * npaths + n] = disc * slope * dsg;
                }
                g[((size_t)p * ng + 2 * d) * npaths + n] = disc * (slope * dr - T * f);
            }
        }
        free(work);
    }
    free(m.Lrho);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Correlation sensitivities, forward mode (Sec. I.A.3: sensitivities to     */
/* model parameters; Sec. VI.A.2 differentiates the basket simulation).      */
/* log-Euler only.  With dW_a = sqrt(Delta) sig_a sum_{b<=a} Lrho[a][b] z_b,  */
/* the tangent of x_a = log S_a with respect to the factor entry Lrho[a][b]   */
/* (b <= a; the drift (r - sig_a^2/2) held fixed) grows at every step by      */
/*   d x_a / d Lrho[a][b]  +=  sqrt(Delta) sig_a z_b,                         */
/* and x_c (c != a) does not depend on Lrho[a][b].  Per path n:               */
/*   xT[a * npaths + n]               = x_a(T)                                */
/*   tL[(a(a+1)/2 + b) * npaths + n]  = d x_a(T) / d Lrho[a][b],  b <= a.     */
/* The map from these to d/d corr goes through the derivative of the          */
/* Cholesky factor (oracle/__init__.py, forward mode).                        */
/* ------------------------------------------------------------------------ */
int orc_gbm_corr_tangents(int d, const double *s0, const double *sig, const double *corr, double r, double T,
                          int steps, uint64_t seed, int64_t path0, int64_t npaths, double *xT, double *tL)
{
    if (d < 1 || steps < 1 || npaths < 0 || !(T > 0.0)) return -1;
    orc_gbm m;
    int rc = gbm_setup(&m, d, s0, sig, corr, NULL, r, T, steps, 0, seed);
    if (rc) return rc;
    const double dt = T / steps, sdt = sqrt(dt);
    const size_t nt = (size_t)d * (d + 1) / 2;
#pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * (2 * (size_t)d + nt));
        double *z = x + d, *t = z + d;
#pragma omp for schedule(static)
        for (int64_t n = 0; n < npaths; ++n) {
            orc_stream st;
            stream_init(&st, seed, (uint64_t)(path0 + n));
            for (int a = 0; a < d; ++a) x[a] = log(s0[a]);
            for (size_t k = 0; k < nt; ++k) t[k] = 0.0;
            for (int i = 0; i < steps; ++i) {
                for (int a = 0; a < d; ++a) z[a] = stream_normal(&st, (uint64_t)i * d + a);
                for (int a = 0; a < d; ++a) {
                    double y = 0.0;
                    for (int b = 0; b <= a; ++b) y += m.Lrho[(size_t)a * d + b] * z[b];
                    x[a] += (r - 0.5 * sig[a] * sig[a]) * dt + sdt * sig[a] * y;
                    for (int b = 0; b <= a; ++b) t[(size_t)a * (a + 1) / 2 + b] += sdt * sig[a] * z[b];
                }
            }
            for (int a = 0; a < d; ++a) xT[(size_t)a * npaths + n] = x[a];
            for (size_t k = 0; k < nt; ++k) tL[k * npaths + n] = t[k];
        }
        free(x);
    }
    free(m.Lrho);
    return 0;
}

/* Arithmetic-average basket (Asian) version: the average                    */
/*   A = (1/M) sum_{i=1..M} U(t_i),  U = sum_a w_a S_a,                        */
/* and its tangents dA / d Lrho[a][b] = (1/M) sum_i w_a S_a(t_i) t_ab(t_i),   */
/* t_ab(t_i) the running tangent of x_a above after step i.  Per path n:     */
/*   A[n], tA[(a(a+1)/2 + b) * npaths + n].                                   */
int orc_gbm_corr_asian_tangents(int d, const double *s0, const double *sig, const double *corr, const double *w,
                                double r, double T, int steps, uint64_t seed, int64_t path0, int64_t npaths,
                                double *A, double *tA)
{
    if (d < 1 || steps < 1 || npaths < 0 || !(T > 0.0)) return -1;
    orc_gbm m;
    int rc = gbm_setup(&m, d, s0, sig, corr, NULL, r, T, steps, 0, seed);
    if (rc) return rc;
    const double dt = T / steps, sdt = sqrt(dt);
    const size_t nt = (size_t)d * (d + 1) / 2;
#pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * (2 * (size_t)d + 2 * nt));
        double *z = x + d, *t = z + d, *acc = t + nt;
#pragma omp for schedule(static)
        for (int64_t n = 0; n < npaths; ++n) {
            orc_stream st;
            stream_init(&st, seed, (uint64_t)(path0 + n));
            for (int a = 0; a < d; ++a) x[a] = log(s0[a]);
            for (size_t k = 0; k < nt; ++k) t[k] = acc[k] = 0.0;
            double sumU = 0.0;
            for (int i = 0; i < steps; ++i) {
                for (int a = 0; a < d; ++a) z[a] = stream_normal(&st, (uint64_t)i * d + a);
                for (int a = 0; a < d; ++a) {
                    double y = 0.0;
                    for (int b = 0; b <= a; ++b) y += m.Lrho[(size_t)a * d + b] * z[b];
                    x[a] += (r - 0.5 * sig[a] * sig[a]) * dt + sdt * sig[a] * y;
                    for (int b = 0; b <= a; ++b) t[(size_t)a * (a + 1) / 2 + b] += sdt * sig[a] * z[b];
                }
                for (int a = 0; a < d; ++a) {
                    const double v = w[a] * exp(x[a]);
                    sumU += v;
                    for (int b = 0; b <= a; ++b) acc[(size_t)a * (a + 1) / 2 + b] += v * t[(size_t)a * (a + 1) / 2 + b];
                }
            }
            A[n] = sumU / steps;
            for (size_t k = 0; k < nt; ++k) tA[k * npaths + n] = acc[k] / steps;
        }
        free(x);
    }
    free(m.Lrho);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Heston stochastic volatility (Sec. II.A.1 names stochastic-volatility     */
/* extensions of the scalar Euler scheme), full-truncation Euler on          */
/* (x = log S, v), two normals per step: z1 = normal 2i, z2 = normal 2i+1.   */
/*   v+ = max(v, 0)                                                          */
/*   x <- x + (r - v+/2) Delta + sqrt(v+ Delta) (rho z1 + sqrt(1-rho^2) z2)  */
/*   v <- v + kappa (theta - v+) Delta + xi sqrt(v+ Delta) z1                */
/* both right-hand sides use the state before the step.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s0, v0, r, kappa, theta, xi, rho, T;
    int steps;
    uint64_t seed;
} orc_heston;

/* tangent index order: 0 S0, 1 v0, 2 r, 3 kappa, 4 theta, 5 xi, 6 rho */
#define ORC_HN 7

static void heston_path(const orc_heston *h, int64_t n, double *save, int64_t col, int save_every, int64_t ld,
                        orc_pathstats *stats, double *dST /* [7] or NULL */, double *dAvg /* [7] */)
{
    const int M = h->steps;
    const double dt = h->T / M;
    const double rc = sqrt(1.0 - h->rho * h->rho);
    orc_stream st;
    stream_init(&st, h->seed, (uint64_t)n);
    double x = log(h->s0), v = h->v0;
    double tx[ORC_HN] = {0}, tv[ORC_HN] = {0}, ta[ORC_HN] = {0};
    tx[0] = 1.0 / h->s0;
    tv[1] = 1.0;
    if (save) { save[col] = h->s0; save[ld + col] = h->v0; }
    double sum = 0.0, umax = -INFINITY, umin = INFINITY, S = h->s0;
    for (int i = 0; i < M; ++i) {
        double z1 = stream_normal(&st, 2 * (uint64_t)i);
        double z2 = stream_normal(&st, 2 * (uint64_t)i + 1);
        double vp = v > 0.0 ? v : 0.0;
        double sq = sqrt(vp * dt);
        double c = h->rho * z1 + rc * z2;
        double xn = x + (h->r - 0.5 * vp) * dt + sq * c;
        double vn = v + h->kappa * (h->theta - vp) * dt + h->xi * sq * z1;
        if (dST) {
            for (int k = 0; k < ORC_HN; ++k) {
                double dvp = v > 0.0 ? tv[k] : 0.0;
                /* d sqrt(v+ dt) = dt dv+ / (2 sqrt(v+ dt)) for v+ > 0, 0 otherwise */
                double dsq = vp > 0.0 ? dt * dvp / (2.0 * sq) : 0.0;
                double dc = (k == 6) ? (z1 - h->rho / rc * z2) : 0.0;
                double dr = (k == 2) ? 1.0 : 0.0;
                double dkap = (k == 3) ? 1.0 : 0.0, dth = (k == 4) ? 1.0 : 0.0, dxi = (k == 5) ? 1.0 : 0.0;
                double ntx = tx[k] + (dr - 0.5 * dvp) * dt + dsq * c + sq * dc;
                double ntv = tv[k] + (dkap * (h->theta - vp) + h->kappa * (dth - dvp)) * dt
                             + (dxi * sq + h->xi * dsq) * z1;
                tx[k] = ntx; tv[k] = ntv;
            }
        }
        x = xn; v = vn;
        S = exp(x);
        sum += S;
        if (S > umax) umax = S;
        if (S < umin) umin = S;
        if (dST) for (int k = 0; k < ORC_HN; ++k) ta[k] += S * tx[k] / M;
        if (save && save_every > 0 && (i + 1) % save_every == 0) {
            int slot = (i + 1) / save_every;
            save[((size_t)slot * 2) * ld + col] = S;
            save[((size_t)slot * 2 + 1) * ld + col] = v;
        }
    }
    if (stats) { stats->u_T = S; stats->avg = sum / M; stats->umax = umax; stats->umin = umin; }
    if (dST) for (int k = 0; k < ORC_HN; ++k) { dST[k] = S * tx[k]; dAvg[k] = ta[k]; }
}

static int heston_check(double v0, double kappa, double theta, double xi, double rho, double T, int steps)
{
    if (steps < 1 || !(T > 0.0) || !(rho > -1.0 && rho < 1.0) || v0 < 0.0 || kappa < 0.0 || theta < 0.0 || xi < 0.0)
        return -1;
    return 0;
}

int orc_heston_payoffs(double s0, double v0, double r, double kappa, double theta, double xi, double rho,
                       double T, int steps, uint64_t seed, int64_t path0, int64_t npaths,
                       int npay, const int *kind, const double *strike, const double *barrier, double *out)
{
    if (heston_check(v0, kappa, theta, xi, rho, T, steps) || npaths < 0) return -1;
    orc_heston h = {s0, v0, r, kappa, theta, xi, rho, T, steps, seed};
    const double disc = exp(-r * T);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < npaths; ++n) {
        orc_pathstats ps;
        heston_path(&h, path0 + n, NULL, 0, 0, 0, &ps, NULL, NULL);
        for (int p = 0; p < npay; ++p)
            out[(size_t)p * npaths + n] = disc * payoff_value(kind[p], strike[p], barrier[p], &ps);
    }
    return 0;
}

/* save[(slot*2 + c)*npaths + n]: c = 0 price S, c = 1 variance v (before truncation). */
int orc_heston_paths(double s0, double v0, double r, double kappa, double theta, double xi, double rho,
                     double T, int steps, uint64_t seed, int64_t path0, int64_t npaths,
                     int save_every, double *save)
{
    if (heston_check(v0, kappa, theta, xi, rho, T, steps) || npaths < 0 || save_every < 1 || steps % save_every)
        return -1;
    orc_heston h = {s0, v0, r, kappa, theta, xi, rho, T, steps, seed};
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < npaths; ++n)
        heston_path(&h, path0 + n, save, n, save_every, npaths, NULL, NULL, NULL);
    return 0;
}

/* Forward-mode pathwise Greeks of the Heston pricer, discounted, per path:
 * g[(p*7 + k)*npaths + n], k: 0 d/dS0, 1 d/dv0, 2 d/dr (with the -T P term),
 * 3 d/dkappa, 4 d/dtheta, 5 d/dxi, 6 d/drho.  European and Asian kinds only. */
int orc_heston_greeks(double s0, double v0, double r, double kappa, double theta, double xi, double rho,
                      double T, int steps, uint64_t seed, int64_t path0, int64_t npaths,
                      int npay, const int *kind, const double *strike, double *g)
{
    if (heston_check(v0, kappa, theta, xi, rho, T, steps) || npaths < 0) return -1;
    for (int p = 0; p < npay; ++p)
        if (kind[p] > ORC_ASIAN_PUT || kind[p] < 0) return -4;
    orc_heston h = {s0, v0, r, kappa, theta, xi, rho, T, steps, seed};
    const double disc = exp(-r * T);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < npaths; ++n) {
        orc_pathstats ps;
        double dST[ORC_HN], dAvg[ORC_HN];
        heston_path(&h, path0 + n, NULL, 0, 0, 0, &ps, dST, dAvg);
        for (int p = 0; p < npay; ++p) {
            double slope = payoff_slope(kind[p], strike[p], &ps);
            double f = payoff_value(kind[p], strike[p], 0.0, &ps);
            const double *dU = payoff_is_asian(kind[p]) ? dAvg : dST;
            for (int k = 0; k < ORC_HN; ++k) {
                double v = disc * slope * dU[k];
                if (k == 2) v -= T * disc * f;
                g[((size_t)p * ORC_HN + k) * npaths + n] = v;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Estimator (Eq. 3): mean of N samples and its standard error             */
/*   se = sqrt((sum f^2 / N - mean^2) / (N - 1)),                           */
/* with Neumaier-compensated sums taken in index order.                      */
/* ------------------------------------------------------------------------ */
static void neumaier_add(double *sum, double *comp, double b)
{
    double a = *sum, t = a + b;
    *comp += (fabs(a) >= fabs(b)) ? (a - t) + b : (b - t) + a;
    *sum = t;
}

void orc_mean_se(const double *f, int64_t n, double *mean, double *se)
{
    double s = 0.0, cs = 0.0, q = 0.0, cq = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        neumaier_add(&s, &cs, f[i]);
        neumaier_add(&q, &cq, f[i] * f[i]);
    }
    double m = (s + cs) / (double)n;
    double m2 = (q + cq) / (double)n;
    *mean = m;
    *se = n > 1 ? sqrt(fmax(m2 - m * m, 0.0) / (double)(n - 1)) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Portfolio risk (Sec. VI.B) and surrogate labels.  Stream indices carry a  */
/* domain tag in the top byte: 2 scenarios, 3 inner paths, 4 labels, 5 base  */
/* values.                                                                   */
/* ------------------------------------------------------------------------ */
static uint64_t domain_tag(uint64_t domain, uint64_t idx) { return (domain << 56) | idx; }

/* Scenario s: S'_u = S0_u exp((mu - sig_u^2/2) h + sqrt(h) sig_u (Lrho z)_u),
 * z_u = normal u of stream tag(2, s). */
int orc_risk_scenarios(int d, const double *s0, const double *sig, const double *corr, double mu, double h,
                       int64_t nscen, uint64_t seed, double *Sp)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)d * (size_t)d);
    if (!L) return -3;
    if (orc_cholesky(d, corr, L) != 0) { free(L); return -2; }
#pragma omp parallel
    {
        double *z = (double *)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(static)
        for (int64_t s = 0; s < nscen; ++s) {
            orc_stream st;
            stream_init(&st, seed, domain_tag(2, (uint64_t)s));
            for (int u = 0; u < d; ++u) z[u] = stream_normal(&st, (uint64_t)u);
            for (int u = 0; u < d; ++u) {
                double w = 0.0;
                for (int k = 0; k <= u; ++k) w += L[(size_t)u * d + k] * z[k];
                Sp[(size_t)s * d + u] = s0[u] * exp((mu - 0.5 * sig[u] * sig[u]) * h + sqrt(h) * sig[u] * w);
            }
        }
        free(z);
    }
    free(L);
    return 0;
}

/* Monte Carlo value of option o of underlying u at state S (log-Euler steps
 * of dt, `steps` of them to maturity, up-and-out monitored at every step and
 * worthless if S already >= H), with `inner` paths of streams tag(domain,
 * base | path).  kind: 0 call, 1 put, 4 up-and-out call (the payoff codes). */
static double nested_value(double S, double sig, double r, double dt, int kind, double K, double H, int steps,
                           int inner, uint64_t seed, uint64_t domain, uint64_t base)
{
    if (kind == ORC_UO_CALL && S >= H) return 0.0;
    double sum = 0.0;
    for (int p = 0; p < inner; ++p) {
        orc_stream st;
        stream_init(&st, seed, domain_tag(domain, base | (uint64_t)p));
        double x = log(S), mx = -INFINITY;
        for (int i = 0; i < steps; ++i) {
            x += (r - 0.5 * sig * sig) * dt + sig * sqrt(dt) * stream_normal(&st, (uint64_t)i);
            if (x > mx) mx = x;
        }
        double ST = exp(x), f;
        if (kind == ORC_PUT) f = K > ST ? K - ST : 0.0;
        else f = ST > K ? ST - K : 0.0;
        if (kind == ORC_UO_CALL && exp(mx) >= H) f = 0.0;
        sum += f;
    }
    return exp(-r * steps * dt) * sum / inner;
}

/* Revaluation of every option: base values (scen < 0: state s0, steps =
 * rem + hsteps, streams tag(5, (u << 24) | path)) or scenario `scen` (state
 * Sp[scen], steps = rem, streams tag(3, ((scen d + u) << 16) | path)). */
int orc_risk_values(int d, const double *state, const double *sig, double r, double dt, int hsteps, int64_t scen,
                    int nopt, const int *under, const int *kind, const double *K, const double *H, const int *rem,
                    int inner, uint64_t seed, double *V)
{
#pragma omp parallel for schedule(dynamic)
    for (int o = 0; o < nopt; ++o) {
        const int u = under[o];
        if (scen < 0)
            V[o] = nested_value(state[u], sig[u], r, dt, kind[o], K[o], H[o], rem[o] + hsteps, inner, seed, 5,
                                (uint64_t)u << 24);
        else
            V[o] = nested_value(state[u], sig[u], r, dt, kind[o], K[o], H[o], rem[o], inner, seed, 3,
                                ((uint64_t)scen * (uint64_t)d + (uint64_t)u) << 16);
    }
    return 0;
}

/* Surrogate label of point p = (S/K, sig, tau, r, K/H): discounted Monte Carlo
 * call price / K (up-and-out with H = K / (K/H) when K/H > 0), `paths` paths
 * of streams tag(4, (p << 16) | path), round(tau * spy) steps. */
/* Pathwise Greeks of the surrogate's European labels (Sec. I.A.3: the
 * derivative of each simulated payoff with respect to the inputs, averaged
 * over the paths).  Point (S/K, sigma, tau, r, K/H) with K/H = 0; the same
 * paths as orc_surrogate_labels (log-Euler in ln S, round(tau spy) steps,
 * stream tag(4, p << 16 | path)).  Per path, with f = e^{-r tau} (S_T - 1)^+
 * in units of K and ln S_T = ln S + (r - sigma^2/2) tau + sigma sqrt(dt) sum z:
 *   df/dS     = e^{-r tau} 1{S_T > 1} S_T / S
 *   df/dsigma = e^{-r tau} 1{S_T > 1} S_T (sqrt(dt) sum z - sigma tau).
 * out[p][0..5] = mean and standard error (Eq. 3) of f, df/dS, df/dsigma;
 * all NaN for barrier points (K/H > 0: a knock-out has no pathwise Greek). */
int orc_surrogate_label_greeks(int64_t npts, const double *pts, int paths, int spy, uint64_t seed, double *out)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t p = 0; p < npts; ++p) {
        const double *q = pts + 5 * p;
        double *o = out + 6 * p;
        if (q[4] > 0.0) {
            for (int k = 0; k < 6; ++k) o[k] = NAN;
            continue;
        }
        const double S = q[0], sig = q[1], r = q[3];
        int M = (int)lround(q[2] * spy);
        if (M < 1) M = 1;
        const double dt = q[2] / M, tau = M * dt, disc = exp(-r * tau);
        double s[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
        for (int n = 0; n < paths; ++n) {
            orc_stream st;
            stream_init(&st, seed, domain_tag(4, ((uint64_t)p << 16) | (uint64_t)n));
            double x = log(S), zs = 0.0;
            for (int i = 0; i < M; ++i) {
                const double z = stream_normal(&st, (uint64_t)i);
                x += (r - 0.5 * sig * sig) * dt + sig * sqrt(dt) * z;
                zs += z;
            }
            const double ST = exp(x), in = ST > 1.0 ? 1.0 : 0.0;
            const double v[3] = {disc * (ST > 1.0 ? ST - 1.0 : 0.0), disc * in * ST / S,
                                 disc * in * ST * (sqrt(dt) * zs - sig * tau)};
            for (int k = 0; k < 3; ++k) {
                s[k] += v[k];
                s2[k] += v[k] * v[k];
            }
        }
        for (int k = 0; k < 3; ++k) {
            const double m = s[k] / paths, var = s2[k] / paths - m * m;
            o[2 * k] = m;
            o[2 * k + 1] = paths > 1 ? sqrt(var > 0.0 ? var / (paths - 1) : 0.0) : 0.0;
        }
    }
    return 0;
}

int orc_surrogate_labels(int64_t npts, const double *pts, int paths, int spy, uint64_t seed, double *labels)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t p = 0; p < npts; ++p) {
        const double *q = pts + 5 * p;
        int M = (int)lround(q[2] * spy);
        if (M < 1) M = 1;
        const double dt = q[2] / M;
        const double H = q[4] > 0.0 ? 1.0 / q[4] : INFINITY;
        labels[p] = nested_value(q[0], q[1], q[3], dt, q[4] > 0.0 ? ORC_UO_CALL : ORC_CALL, 1.0, H, M, paths, seed,
                                 4, (uint64_t)p << 16);
    }
    return 0;
}
