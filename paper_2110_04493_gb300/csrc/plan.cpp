// Host-side scalar choices of Algorithm 4.2: the Taylor error bound of Eq. (4.5)
// and the (M, N) enumeration of Eq. (4.20).  No GPU is involved.
#include <cmath>
#include <algorithm>
#include <climits>
#include <cstdint>

#include "../../include/sexpm.h"

extern "C" double sexpm_rho(int32_t M, double x) {
  // (1/M!) sum_{k>=0} x^{M+1+k} / (k! (M+1+k))  =  (1/M!) int_0^x u^M e^u du,
  // i.e. (-1)^{M+1} gamma(M+1, -x) / M!  (Eq. 4.5).  All terms are positive, so the
  // forward sum is accurate; it stops once a term no longer changes the sum.
  if (M < 0 || !(x >= 0.0)) return NAN;
  if (x == 0.0) return 0.0;
  double lead = 1.0;  // x^{M+1} / M!
  for (int j = 1; j <= M; ++j) lead *= x / j;
  lead *= x;
  double sum = 0.0;
  double c = lead;    // x^{M+1+k} / (M! k!)
  for (int k = 0; k < 100000; ++k) {
    const double term = c / (double)(M + 1 + k);
    sum += term;
    if (term <= 1e-18 * sum || c == 0.0) break;
    c *= x / (double)(k + 1);
  }
  return sum;
}

extern "C" int sexpm_choose_MN(double norm_H, double eps, int32_t n_extra, int32_t max_M, int32_t* M_out,
                               int32_t* N_out) {
  if (!M_out || !N_out || !(eps > 0.0) || !std::isfinite(eps) || !(norm_H >= 0.0) || !std::isfinite(norm_H) ||
      n_extra < 0 || max_M < 1)
    return SEXPM_EINVAL;
  if (norm_H == 0.0) {
    *M_out = 0;
    *N_out = 0;
    return SEXPM_OK;
  }
  int e = 0;
  const double m = std::frexp(norm_H, &e);  // norm_H = m 2^e, m in [0.5, 1)
  const int ceil_log2 = (m == 0.5) ? e - 1 : e;
  const int N0 = ceil_log2 > 0 ? ceil_log2 : 0;
  bool found = false;
  double best_cost = 0.0;
  int best_M = 0, best_N = 0;
  for (int N = N0; N <= N0 + n_extra; ++N) {
    const double x = std::ldexp(norm_H, -N);  // <= 1 for N >= N0
    int Mn = 1;
    while (Mn <= max_M && std::ldexp(sexpm_rho(Mn, x), N) > eps) ++Mn;
    if (Mn > max_M) continue;
    const double cost = std::ldexp((double)Mn, N);
    bool better = !found || cost < best_cost;
    if (found && cost == best_cost) {
      if (Mn + N != best_M + best_N) better = Mn + N < best_M + best_N;
      else better = N < best_N;
    }
    if (better) {
      found = true;
      best_cost = cost;
      best_M = Mn;
      best_N = N;
    }
  }
  if (!found) return SEXPM_ENOPARAM;
  *M_out = best_M;
  *N_out = best_N;
  return SEXPM_OK;
}

namespace sexpm {
// h_{M1,Np} = max over M1+1 <= k <= 2 M1 + 1 of ||(H 2^-Np)^k||^(1/k), from pnorms[k-1] = ||H^k||
// (Sec. 4.2, the refined norm of [11]); -1 when pnorms does not reach k = 2 M1 + 1.
double h_refined(const double* pnorms, int32_t kmax, int32_t M1, int32_t Np) {
  if (2 * M1 + 1 > kmax) return -1.0;
  double best = 0.0;
  for (int32_t k = M1 + 1; k <= 2 * M1 + 1; ++k) {
    const double v = pnorms[k - 1];
    if (v > 0.0) best = std::max(best, std::exp((std::log(v) - (double)Np * k * std::log(2.0)) / k));
  }
  return best;
}
}  // namespace sexpm
using sexpm::h_refined;

extern "C" int sexpm_alpha_hat(double norm_H, int32_t M, int32_t N, int32_t i, const double* pnorms, int32_t kmax,
                               int32_t* alpha) {
  // Eq. (4.8) (pnorms NULL) or Eq. (4.9): the least M1 2^N1 with 2^N1 rho(M1, x) <= r_i,
  // r_i = 2^i rho(M, ||H 2^-N||) (Eq. 4.6), x = ||H 2^{i-N-N1}|| or h_{M1, N+N1-i}.
  if (!alpha || !(norm_H >= 0.0) || M < 1 || N < 0 || i < 0 || (pnorms && kmax < 3)) return SEXPM_EINVAL;
  const double ri = std::ldexp(sexpm_rho(M, std::ldexp(norm_H, -N)), i);
  long long best = -1;
  for (int32_t N1 = 0; N1 <= 40; ++N1) {
    for (int32_t M1 = 1; M1 <= 1000; ++M1) {
      double x;
      if (!pnorms) {
        x = std::ldexp(norm_H, i - N - N1);
      } else {
        x = h_refined(pnorms, kmax, M1, N + N1 - i);
        if (x < 0.0) break;
      }
      if (std::ldexp(sexpm_rho(M1, x), N1) <= ri) {
        const long long c = (long long)M1 << N1;
        if (best < 0 || c < best) best = c;
        break;
      }
    }
  }
  if (best < 0 || best > INT32_MAX) return SEXPM_ENOPARAM;
  *alpha = (int32_t)best;
  return SEXPM_OK;
}

extern "C" int sexpm_choose_MN_refined(double norm_H, const double* pnorms, int32_t kmax, double eps, int32_t n_extra,
                                       int32_t* M_out, int32_t* N_out) {
  // Eq. (4.20) with the refined norm: minimise M 2^N over N in [0, N0 + n_extra] (N0 from ||H||),
  // M the least positive integer with 2^N rho(M, h_{M,N}) <= eps and h_{M,N} <= 1 (the paper's
  // ||H 2^-N|| <= 1 for the Taylor phase's rounding, read on the refined norm); only M with
  // 2M + 1 <= kmax can be tested.  Ties to the smaller M + N, then the smaller N.
  if (!M_out || !N_out || !pnorms || kmax < 3 || !(eps > 0.0) || !std::isfinite(eps) || !(norm_H >= 0.0) ||
      n_extra < 0)
    return SEXPM_EINVAL;
  if (norm_H == 0.0) {
    *M_out = 0;
    *N_out = 0;
    return SEXPM_OK;
  }
  int e = 0;
  const double m = std::frexp(norm_H, &e);
  const int ceil_log2 = (m == 0.5) ? e - 1 : e;
  const int N0 = ceil_log2 > 0 ? ceil_log2 : 0;
  bool found = false;
  double best_cost = 0.0;
  int best_M = 0, best_N = 0;
  for (int N = 0; N <= N0 + n_extra; ++N) {
    int Mn = -1;
    for (int M = 1; 2 * M + 1 <= kmax; ++M) {
      const double h = h_refined(pnorms, kmax, M, N);
      if (h > 1.0) continue;
      if (std::ldexp(sexpm_rho(M, h), N) <= eps) {
        Mn = M;
        break;
      }
    }
    if (Mn < 0) continue;
    const double cost = std::ldexp((double)Mn, N);
    bool better = !found || cost < best_cost;
    if (found && cost == best_cost) {
      if (Mn + N != best_M + best_N) better = Mn + N < best_M + best_N;
      else better = N < best_N;
    }
    if (better) {
      found = true;
      best_cost = cost;
      best_M = Mn;
      best_N = N;
    }
  }
  if (!found) return SEXPM_ENOPARAM;
  *M_out = best_M;
  *N_out = best_N;
  return SEXPM_OK;
}
