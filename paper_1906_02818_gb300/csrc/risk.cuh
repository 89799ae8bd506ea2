// Portfolio-risk kernels (k_risk.cu): arguments and launchers.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace gbmc {

constexpr int kRiskMaxUnder = 64;        // underlyings
constexpr int kRiskMaxOptPerUnder = 32;  // options per underlying

// Options are grouped by underlying (under_start[u] .. under_start[u+1]) and
// sorted by maturity within a group.  rem[o]: steps from the scenario date
// to maturity; the base date adds horizon_steps.  Device pointers.
struct RiskArgs {
    int d, nopt;
    const float *s0, *sigma;
    float r, dt;
    int horizon_steps;
    const int *under, *under_start, *kind, *rem;
    const float *strike, *barrier;
    const double *pos, *base;
    double *base_out;
    int inner;
    RoundKeys rk;      // Philox round keys of the seed
    int64_t scen_off;  // global index of the first scenario (stream indices)
};

// dlabels: NULL, or [npts][2] pathwise d label / d(S/K) and d label / d sigma
// of the European points (NaN for barrier points).
cudaError_t launch_labels(int64_t npts, const float *pts, int paths, float steps_per_year, const RoundKeys &rk,
                          float *labels, float *inputs, float *dlabels, cudaStream_t s);
cudaError_t launch_outer(int64_t nscen, int64_t off, int d, const float *Lc, const float *drift, const float *s0,
                         const RoundKeys &rk, float *Sp, cudaStream_t s);
cudaError_t launch_nested(const RiskArgs &a, int64_t nscen, const float *Sp, double *contrib, cudaStream_t s);
cudaError_t launch_sum_under(int64_t nscen, int d, const double *contrib, double *pnl, cudaStream_t s);
cudaError_t launch_features(const RiskArgs &a, int64_t nscen, const float *Sp, float *x, cudaStream_t s);
cudaError_t launch_pnl(const RiskArgs &a, int64_t nscen, const float *Sp, const float *y, double *pnl, cudaStream_t s);
cudaError_t launch_tail(int64_t n, const double *pnl, double *work, int64_t npow2, double alpha, double *res,
                        cudaStream_t s);

}  // namespace gbmc
