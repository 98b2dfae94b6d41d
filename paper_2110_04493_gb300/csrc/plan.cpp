// Host-side scalar choices of Algorithm 4.2: the Taylor error bound of Eq. (4.5)
// and the (M, N) enumeration of Eq. (4.20).  No GPU is involved.
#include <cmath>
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
