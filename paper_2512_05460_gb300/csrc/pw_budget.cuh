// Budget (Algorithm 1 line 1; Eqs. B-value, G-value, R-value, K-value) and
// the per-probe U-statistic (Eq. Q-Ustat) from the probe's S1 and S2, shared by
// the batch pipeline and the server.  FP64 expressions are written operation by operation (no fused
// multiply-add; the library is compiled with --fmad=false as well) in the
// order the oracle evaluates them, so plans and statistics are bit-identical.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

__host__ __device__ __forceinline__ double ceil_tol(double x) { return ceil(x * (1.0 - 1e-12)); }

// R of Eq. R-value before the ceiling.
__host__ __device__ __forceinline__ double r_theory_raw(double eps, int32_t L, double d_min, double ds, double dt) {
  const double inv = 1.0 / ds + 1.0 / dt;
  return 128.0 * (double)(L + 1) * (double)(L + 1) / (d_min * d_min * (1.0 - eps / 2.0) * inv * inv);
}

// Plan of one query from its arguments and the degrees of s and t.  Invalid
// arguments give status PW_ERR_ARG and no work; s == t gives no work and an
// estimate of exactly 0.  PP (pilot plan) gets K0 x R0 in PILOT mode.
__host__ __device__ inline void plan_query(int64_t s, int64_t t, double eps, int32_t L, uint64_t seed, int64_t n,
                                           int32_t deg_s, int32_t deg_t, const BudgetArgs& A, QPlan* out,
                                           QPlan* pilot_out) {
  QPlan P;
  memset(&P, 0, sizeof P);
  P.eps = eps;
  P.L = L;
  P.status = PW_OK;
  QPlan PP = P;
  if (s < 0 || s >= n || t < 0 || t >= n || !(eps > 0.0 && eps < 1.0) || L < 0) {
    P.status = PW_ERR_ARG;
  } else {
    P.s = (int32_t)s;
    P.t = (int32_t)t;
    P.seed = seed;
    if (s != t) {
      const double ds = (double)deg_s, dt = (double)deg_t, dmin = (double)A.d_min;
      double B = 0.0, R = 0.0;
      const double G = (double)A.G;
      switch (A.mode) {
        case PW_BUDGET_THEORY:
          B = ceil_tol(448.0 / (eps * eps));
          R = ceil_tol(r_theory_raw(eps, L, dmin, ds, dt));
          if (R < 2.0) R = 2.0;
          break;
        case PW_BUDGET_SCALED:
          B = ceil_tol(A.c_B * 448.0 / (eps * eps));
          if (B < 1.0) B = 1.0;
          R = ceil_tol(A.c_R * r_theory_raw(eps, L, dmin, ds, dt));
          if (R < 2.0) R = 2.0;
          if (R > (double)A.R_max) R = (double)A.R_max;
          break;
        case PW_BUDGET_FIXED:
          B = (double)A.B_fixed;
          R = (double)A.R_fixed;
          break;
        default:  // PILOT and ADAPTIVE
          B = ceil_tol(A.c_B / (eps * eps));
          if (B < 1.0) B = 1.0;
          R = 0.0;
          break;
      }
      if (B * G >= 4294967296.0 || R >= 4294967296.0) {
        P.status = PW_ERR_ARG;  // budget beyond 2^32 probes or replicas
      } else {
        P.B = (uint32_t)B;
        P.G = A.G;
        if (A.mode == PW_BUDGET_ADAPTIVE) {  // first stage: ceil(B/4) probes per block
          const double Bmax = ceil_tol(A.cap * (double)P.B);
          P.Bmax = Bmax * (double)P.G >= 4294967296.0 ? 0u : (uint32_t)Bmax;
          if (P.Bmax == 0) P.status = PW_ERR_ARG;
          P.B = (P.B + 3u) / 4u;
        }
        P.K = P.B * P.G;
        P.R = (uint32_t)R;
        P.chunks = (P.R + 31u) / 32u;
        if (A.mode == PW_BUDGET_PILOT || A.mode == PW_BUDGET_ADAPTIVE) {
          PP.s = P.s;
          PP.t = P.t;
          PP.seed = P.seed;
          PP.K = (uint32_t)A.K0;
          PP.R = (uint32_t)A.R0;
          PP.chunks = 1;
        }
      }
    }
  }
  if (P.status != PW_OK) {
    P.K = 0;
    P.R = 0;
    P.chunks = 0;
  }
  *out = P;
  if (pilot_out) *pilot_out = PP;
}

// Q slots a query reserves: G Bmax for ADAPTIVE (its B may grow to Bmax), else K.
__host__ __device__ __forceinline__ uint64_t q_slots(const QPlan& P) {
  return P.Bmax ? (uint64_t)P.G * P.Bmax : (uint64_t)P.K;
}

// ADAPTIVE stopping rule: from the first stage's G*B1 values of Q_R (q), the
// smallest B with z standard errors of the median of means, sqrt(pi/2) sd(Q) /
// sqrt(G B), inside eps theta, theta = max(mean Q, theta_0); clamped to
// [B1, Bmax].  Sums in index order, operation by operation as the oracle.
__host__ __device__ inline uint32_t adaptive_B(const double* q, uint32_t B1, uint32_t Bmax, uint32_t G, double eps,
                                               double z, int32_t deg_s, int32_t deg_t) {
  const uint64_t K1 = (uint64_t)G * B1;
  double sum = 0.0;
  for (uint64_t k = 0; k < K1; ++k) sum = sum + q[k];
  const double mean = sum / (double)K1;
  double ss = 0.0;
  for (uint64_t k = 0; k < K1; ++k) ss = ss + (q[k] - mean) * (q[k] - mean);
  const double s2 = K1 > 1 ? ss / (double)(K1 - 1) : 0.0;
  const double inv = 1.0 / (double)deg_s + 1.0 / (double)deg_t;
  const double theta0 = (1.0 / 8.0) * (1.0 - eps / 2.0) * inv * inv;
  const double theta = mean > theta0 ? mean : theta0;
  double x = 1.5707963267948966 * z * z * s2;
  x = x / (theta * theta);
  x = x / ((double)G * eps * eps);
  double B = ceil_tol(x);
  if (B < (double)B1) B = (double)B1;
  if (B > (double)Bmax) B = (double)Bmax;
  return (uint32_t)B;
}

// Q_R = (S1^2 - S2) / (R (R - 1)) (Eq. Q-Ustat).
__host__ __device__ __forceinline__ double u_statistic(double S1, double S2, uint32_t R) {
  const double Rd = (double)R;
#ifdef __CUDA_ARCH__
  return __ddiv_rn(__dsub_rn(__dmul_rn(S1, S1), S2), __dmul_rn(Rd, __dsub_rn(Rd, 1.0)));
#else
  return (S1 * S1 - S2) / (Rd * (Rd - 1.0));
#endif
}

// One pilot probe's contribution: within-probe sample variance and Q.
__host__ __device__ __forceinline__ void pilot_accumulate(double& sum_var, double& sum_q, double S1, double S2,
                                                          uint32_t R0u) {
  const double R0 = (double)R0u;
#ifdef __CUDA_ARCH__
  const double Q = __ddiv_rn(__dsub_rn(__dmul_rn(S1, S1), S2), __dmul_rn(R0, __dsub_rn(R0, 1.0)));
  sum_var = __dadd_rn(sum_var, __ddiv_rn(__dsub_rn(S2, __ddiv_rn(__dmul_rn(S1, S1), R0)), __dsub_rn(R0, 1.0)));
  sum_q = __dadd_rn(sum_q, Q);
#else
  const double Q = (S1 * S1 - S2) / (R0 * (R0 - 1.0));
  sum_var = sum_var + (S2 - S1 * S1 / R0) / (R0 - 1.0);
  sum_q = sum_q + Q;
#endif
}

// R from the pilot: ceil(c_R 4 sigma2 / theta), theta = max(mean Q, theta_0),
// at least 2, rounded up to whole warps of 32, at most R_max.
__host__ __device__ inline void pilot_finish(QPlan& P, double sum_var, double sum_q, uint32_t K0, int32_t deg_s,
                                             int32_t deg_t, const BudgetArgs& A) {
  const double sigma2 = sum_var / (double)K0;
  const double q_bar = sum_q / (double)K0;
  const double ds = (double)deg_s, dt = (double)deg_t;
  const double inv = 1.0 / ds + 1.0 / dt;
  const double theta0 = (1.0 / 8.0) * (1.0 - P.eps / 2.0) * inv * inv;
  const double theta = q_bar > theta0 ? q_bar : theta0;
  double R = ceil_tol(A.c_R * 4.0 * sigma2 / theta);
  if (R < 2.0) R = 2.0;
  R = 32.0 * ceil(R / 32.0);
  if (R > (double)A.R_max) R = (double)A.R_max;
  P.R = (uint32_t)R;
  P.chunks = (P.R + 31u) / 32u;
  P.sigma2 = sigma2;
  P.qbar = q_bar;
  P.theta = theta;
}

}  // namespace pw
