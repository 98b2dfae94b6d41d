// Complex H (the method is stated for C^{n x n}) through the real embedding
//   R(Z) = X (x) I_2 + Y (x) J,  J = [[0, -1], [1, 0]],  for Z = X + iY,
// which maps sums, products, real scalings and the exponential to the same operations on Z
// (J^2 = -I, so R(Z1 Z2) = R(Z1) R(Z2) and e^{R(Z)} = R(e^Z)).  Row 2i of R(Z) holds, for every
// stored z_ij, the pair (column 2j: Re z_ij, column 2j + 1: -Im z_ij); row 2i + 1 holds the same
// columns with each pair (x, -y) turned into (y, x).  Interleaving keeps a row's columns as close
// together as in Z (twice the span), which the bitmap accumulators of the sparse product need.
// The method works on the even rows only: a product T~ = 2 T + T T forms the n even rows of
// R(T) R(T) (A = the even rows, B = all 2n rows, rebuilt from the even rows by a mirror), so each
// complex product costs four real multiply-adds, as in complex arithmetic.
//
// Algorithm 4.1 decides by the modulus: both entries of a pair are kept iff
// |z| = sqrt(re^2 + im^2) > t (computed the same way from either entry, so a pair is never
// split), and every dropped entry adds its square, so a pass sums |z|^2 over the dropped complex
// entries.
//
// Kernels: the embedding of a complex CSR (values re, im interleaved), its validation, the block
// mirror, the complex filter pass and compaction, and the extraction of the complex result.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

int sms_z() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    SX_CUDA(cudaGetDevice(&dev));
    SX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

// First index in [lo, hi) whose column is >= c (columns sorted).
__device__ __forceinline__ int64_t lb(const int32_t* ci, int64_t lo, int64_t hi, int c) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Complex input: rows sorted, columns unique and in [0, n), values finite, row pointers monotone.
// One thread per row.
__global__ void k_valid_z(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* vz, int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == 0 && rp[0] != 0) atomicOr(bad, 1);
  if (i == n) {
    if (rp[n] != nnz) atomicOr(bad, 1);
    return;
  }
  const int64_t p0 = rp[i], p1 = rp[i + 1];
  if (p1 < p0 || p0 < 0 || p1 > nnz) {
    atomicOr(bad, 1);
    return;
  }
  for (int64_t p = p0; p < p1; ++p) {
    const int c = ci[p];
    if (c < 0 || c >= n || (p > p0 && ci[p - 1] >= c) || !isfinite(vz[2 * p]) || !isfinite(vz[2 * p + 1])) {
      atomicOr(bad, 1);
      return;
    }
  }
}

// Even rows of R(Z): row i holds 2 nnz_i entries, the pair (2c: Re z_ic, 2c + 1: -Im z_ic) for
// every stored z_ic, in column order.  One thread per entry.
__global__ void k_embed_even(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* vz,
                             int64_t* rp_t, int32_t* ci_t, double* v_t) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int c = ci[p];
    ci_t[2 * p] = 2 * c;
    v_t[2 * p] = vz[2 * p];
    ci_t[2 * p + 1] = 2 * c + 1;
    v_t[2 * p + 1] = -vz[2 * p + 1];
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) rp_t[i] = 2 * rp[i];
}

// All 2n rows of R(Z) from its even rows: row 2i is even row i, row 2i + 1 holds the same columns
// with each pair (x, -y) turned into (y, x).
__global__ void k_mirror_rp(int64_t n, const int64_t* rp_t, int64_t* rp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  rp[2 * i] = 2 * rp_t[i];
  if (i < n) rp[2 * i + 1] = 2 * rp_t[i] + (rp_t[i + 1] - rp_t[i]);
}

// The value paired with the entry at p of a row [p0, p1) (column c xor 1, next to it when present),
// else 0.
__device__ __forceinline__ double partner(const CsrD& A, int64_t p0, int64_t p1, int64_t p, int c) {
  const int64_t q = (c & 1) ? p - 1 : p + 1;
  return (q >= p0 && q < p1 && A.ci[q] == (c ^ 1)) ? A.v[q] : 0.0;
}

__global__ void k_mirror_rows(int64_t n, CsrD top, const int64_t* rp, int32_t* ci, double* v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < n; i += nw) {
    const int64_t p0 = top.rp[i], p1 = top.rp[i + 1];
    const int64_t o_even = rp[2 * i], o_odd = rp[2 * i + 1];
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      const int c = top.ci[p];
      const double x = top.v[p];
      const double y = partner(top, p0, p1, p, c);
      ci[o_even + (p - p0)] = c;
      v[o_even + (p - p0)] = x;
      ci[o_odd + (p - p0)] = c;
      v[o_odd + (p - p0)] = (c & 1) ? y : -y;  // (x, -y) -> (y, x)
    }
  }
}

// |z| of the complex entry that the entry at p belongs to: sqrt(re^2 + im^2) with (re, -im) the
// pair, evaluated in the same order from either entry (so a pair is never split).
__device__ __forceinline__ double modulus_at(const CsrD& A, int64_t p0, int64_t p1, int64_t p) {
  const int c = A.ci[p];
  const double x = A.v[p];
  const double y = partner(A, p0, p1, p, c);
  const double re = (c & 1) ? y : x, mi = (c & 1) ? x : y;
  return sqrt(__dadd_rn(__dmul_rn(re, re), __dmul_rn(mi, mi)));
}

// One Algorithm 4.1 pass over the even rows: keep[i] = entries of row i whose |z| > t,
// part[i] = sum of v^2 over the others.  One warp per row.
__global__ void k_pass_z(CsrD A, double t, int32_t* keep, double* part) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
    int c = 0;
    double sq = 0.0;
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      if (modulus_at(A, p0, p1, p) > t) ++c;
      else sq = fma(A.v[p], A.v[p], sq);
    }
    for (int o = 16; o > 0; o >>= 1) {
      c += __shfl_xor_sync(FULL, c, o);
      sq += __shfl_xor_sync(FULL, sq, o);
    }
    if (lane_id() == 0) {
      keep[i] = c;
      part[i] = sq;
    }
  }
}

// The kept entries (|z| > t) of every even row, in order, at out_rp[i].
__global__ void k_compact_z(CsrD A, double t, const int64_t* out_rp, int32_t* out_ci, double* out_v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane_id()) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
    int64_t o = out_rp[i];
    for (int64_t pb = p0; pb < p1; pb += 32) {
      const int64_t p = pb + lane_id();
      const bool k = p < p1 && modulus_at(A, p0, p1, p) > t;
      const unsigned m = __ballot_sync(FULL, k);
      if (k) {
        out_ci[o + __popc(m & lt)] = A.ci[p];
        out_v[o + __popc(m & lt)] = A.v[p];
      }
      o += __popc(m);
    }
  }
}

// The identity in the even-row layout: row i holds (2i: 1, 2i + 1: 0).
__global__ void k_eye_pairs(int64_t n, int64_t* rp, int32_t* ci, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  rp[i] = 2 * i;
  if (i < n) {
    ci[2 * i] = (int)(2 * i);
    v[2 * i] = 1.0;
    ci[2 * i + 1] = (int)(2 * i + 1);
    v[2 * i + 1] = 0.0;
  }
}

// d[i] = Re z_ii, the value at column 2i of even row i (0 when absent).
__global__ void k_diag_pairs(CsrD A, double* d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t p1 = A.rp[i + 1];
  const int64_t p = lb(A.ci, A.rp[i], p1, (int)(2 * i));
  d[i] = (p < p1 && A.ci[p] == (int)(2 * i)) ? A.v[p] : 0.0;
}

// Complex entries of each even row: one per column pair j (2j and/or 2j + 1 stored).
// One thread per row.
template <bool WRITE>
__global__ void k_extract_z(CsrD A, int32_t* cnt, const int64_t* out_rp, int32_t* out_ci, double* out_vz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
  int64_t o = WRITE ? out_rp[i] : 0;
  int k = 0;
  for (int64_t p = p0; p < p1;) {
    const int c = A.ci[p];
    double re = 0.0, im = 0.0;
    if ((c & 1) == 0) {
      re = A.v[p];
      if (p + 1 < p1 && A.ci[p + 1] == c + 1) {
        im = -A.v[p + 1];
        p += 2;
      } else {
        p += 1;
      }
    } else {
      im = -A.v[p];
      p += 1;
    }
    if (WRITE) {
      out_ci[o] = c >> 1;
      out_vz[2 * o] = re;
      out_vz[2 * o + 1] = im;
      ++o;
    }
    ++k;
  }
  if (!WRITE) cnt[i] = k;
}

}  // namespace

bool valid_complex(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* vz, cudaStream_t s,
                   HostScalars& hs) {
  DevBuf<int> flag(1, s);
  SX_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  k_valid_z<<<(unsigned)((n + 256) / 256), 256, 0, s>>>(n, nnz, rp, ci, vz, flag.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  int f = 0;
  SX_CUDA(cudaMemcpyAsync(hs.i, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  std::memcpy(&f, hs.i, sizeof(int));
  return f == 0;
}

void embed_top(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* vz, cudaStream_t s,
               CsrOwned& top) {
  top.n = n;
  top.nnz = 2 * nnz;
  top.rp.reset(n + 1, s);
  top.ci.reset(top.nnz, s);
  top.v.reset(top.nnz, s);
  const int blocks = (int)std::min<int64_t>((std::max(nnz, n + 1) + 255) / 256, (int64_t)sms_z() * 16);
  k_embed_even<<<blocks, 256, 0, s>>>(n, nnz, rp, ci, vz, top.rp.p, top.ci.p, top.v.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void block_mirror(const CsrD& top, int64_t n, cudaStream_t s, CsrOwned& full) {
  full.n = 2 * n;
  full.nnz = 2 * top.nnz;
  full.rp.reset(2 * n + 1, s);
  full.ci.reset(full.nnz, s);
  full.v.reset(full.nnz, s);
  k_mirror_rp<<<(unsigned)((n + 256) / 256), 256, 0, s>>>(n, top.rp, full.rp.p);
  if (n) {
    const int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sms_z() * 64);
    k_mirror_rows<<<blocks, 256, 0, s>>>(n, top, full.rp.p, full.ci.p, full.v.p);
  }
  SX_CUDA(cudaGetLastError());
  count_launches(n ? 2 : 1);
}

double pass_complex(const CsrD& top, int64_t n, double t, int32_t* keep, double* part, cudaStream_t s,
                    HostScalars& hs) {
  (void)n;
  if (top.n == 0) return 0.0;
  const int blocks = (int)std::min<int64_t>((top.n + 7) / 8, (int64_t)sms_z() * 64);
  k_pass_z<<<blocks, 256, 0, s>>>(top, t, keep, part);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  return reduce_sum(part, top.n, s, hs);
}

void compact_complex(const CsrD& top, int64_t n, double t, const int32_t* keep, cudaStream_t s, CsrOwned& out,
                     HostScalars& hs) {
  (void)n;
  out.n = top.n;
  out.rp.reset(top.n + 1, s);
  out.nnz = scan_counts(keep, top.n, out.rp.p, s, hs);
  out.ci.reset(out.nnz, s);
  out.v.reset(out.nnz, s);
  if (top.n == 0) return;
  const int blocks = (int)std::min<int64_t>((top.n + 7) / 8, (int64_t)sms_z() * 64);
  k_compact_z<<<blocks, 256, 0, s>>>(top, t, out.rp.p, out.ci.p, out.v.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void identity_pairs(int64_t n, cudaStream_t s, CsrOwned& I) {
  I.n = n;
  I.nnz = 2 * n;
  I.rp.reset(n + 1, s);
  I.ci.reset(I.nnz, s);
  I.v.reset(I.nnz, s);
  k_eye_pairs<<<(unsigned)((n + 256) / 256), 256, 0, s>>>(n, I.rp.p, I.ci.p, I.v.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

double trace_re(const CsrD& top, cudaStream_t s, HostScalars& hs) {
  if (top.n == 0) return 0.0;
  DevBuf<double> d(top.n, s);
  k_diag_pairs<<<(unsigned)((top.n + 255) / 256), 256, 0, s>>>(top, d.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  return reduce_sum(d.p, top.n, s, hs);
}

void extract_complex(const CsrD& top, int64_t n, cudaStream_t s, CsrOwned& pattern, DevBuf<double>& vz,
                     HostScalars& hs) {
  (void)n;
  pattern.n = top.n;
  pattern.rp.reset(top.n + 1, s);
  DevBuf<int32_t> cnt(top.n ? top.n : 1, s);
  const unsigned blocks = (unsigned)((top.n + 255) / 256);
  if (top.n) k_extract_z<false><<<blocks, 256, 0, s>>>(top, cnt.p, nullptr, nullptr, nullptr);
  SX_CUDA(cudaGetLastError());
  pattern.nnz = scan_counts(cnt.p, top.n, pattern.rp.p, s, hs);
  pattern.ci.reset(pattern.nnz, s);
  vz.reset(2 * pattern.nnz, s);
  if (top.n) k_extract_z<true><<<blocks, 256, 0, s>>>(top, nullptr, pattern.rp.p, pattern.ci.p, vz.p);
  SX_CUDA(cudaGetLastError());
  count_launches(top.n ? 2 : 0);
}

}  // namespace sexpm
