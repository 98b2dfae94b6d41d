// Complex H (the method is stated for C^{n x n}) through the real embedding
//   R(Z) = [[X, -Y], [Y, X]]  for Z = X + iY,
// which maps sums, products, real scalings and the exponential to the same operations on Z
// (R(Z1 Z2) = R(Z1) R(Z2), e^{R(Z)} = R(e^Z)).  Row i < n of R(Z) is [X_i | -Y_i]; row n + i is
// the same entries with the halves swapped and the new left half negated.  The method works on
// the top rows only: a product T~ = 2 T + T T forms the n top rows of R(T) R(T) (A = the top
// rows, B = all 2n rows, rebuilt from the top rows by a block mirror), so each complex product
// costs four real multiply-adds, as in complex arithmetic.
//
// Algorithm 4.1 decides by the modulus: complex entry z_ij is stored in top row i as the pair
// (column j: Re z, column n + j: -Im z); both entries are kept iff |z| = sqrt(re^2 + im^2) > t
// (computed the same way from either entry, so a pair is never split), and every dropped entry
// adds its square, so a pass sums |z|^2 over the dropped complex entries.
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

// Top rows of R(Z): row i holds 2 nnz_i entries, columns j (Re z_ij) then n + j (-Im z_ij).
__global__ void k_embed_top(int64_t n, const int64_t* rp, const int32_t* ci, const double* vz, int64_t* rp_t,
                            int32_t* ci_t, double* v_t) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < n; i += nw) {
    const int64_t p0 = rp[i], p1 = rp[i + 1], len = p1 - p0;
    if (lane_id() == 0) {
      rp_t[i] = 2 * p0;
      if (i == n - 1) rp_t[n] = 2 * p1;
    }
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      const int64_t o = 2 * p0 + (p - p0);
      const int c = ci[p];
      ci_t[o] = c;
      v_t[o] = vz[2 * p];
      ci_t[o + len] = c + (int)n;
      v_t[o + len] = -vz[2 * p + 1];
    }
  }
}

// All 2n rows of R(Z) from its top rows (row pointers first, then entries).
__global__ void k_mirror_rp(int64_t n, const int64_t* rp_t, int64_t* rp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  rp[i] = rp_t[i];
  rp[n + i] = rp_t[n] + rp_t[i];
}

__global__ void k_mirror_rows(int64_t n, CsrD top, const int64_t* rp, int32_t* ci, double* v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < n; i += nw) {
    const int64_t p0 = top.rp[i], p1 = top.rp[i + 1];
    const int64_t mid = lb(top.ci, p0, p1, (int)n);
    const int64_t o_top = rp[i], o_bot = rp[n + i];
    const int64_t right = p1 - mid;
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      const int c = top.ci[p];
      const double x = top.v[p];
      ci[o_top + (p - p0)] = c;
      v[o_top + (p - p0)] = x;
      if (p >= mid) {  // -Y entry of the top row: Y at column c - n of the bottom row
        ci[o_bot + (p - mid)] = c - (int)n;
        v[o_bot + (p - mid)] = -x;
      } else {         // X entry: X at column c + n of the bottom row, after the Y entries
        ci[o_bot + right + (p - p0)] = c + (int)n;
        v[o_bot + right + (p - p0)] = x;
      }
    }
  }
}

// |z| of the complex entry that the top-row entry at p belongs to (its pair partner is at
// column c +- n of the same row; an absent partner is 0).  The same value from either entry.
__device__ __forceinline__ double modulus_at(const CsrD& A, int64_t n, int64_t p0, int64_t mid, int64_t p1, int64_t p) {
  const int c = A.ci[p];
  const double x = A.v[p];
  int64_t lo, hi;
  int target;
  if (p < mid) { lo = mid; hi = p1; target = c + (int)n; } else { lo = p0; hi = mid; target = c - (int)n; }
  const int64_t q = lb(A.ci, lo, hi, target);
  const double y = (q < hi && A.ci[q] == target) ? A.v[q] : 0.0;
  const double a = p < mid ? x : y, b = p < mid ? y : x;  // (re, -im) in that order for both entries
  return sqrt(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
}

// One Algorithm 4.1 pass over the top rows: keep[i] = entries of row i whose |z| > t,
// part[i] = sum of v^2 over the others.  One warp per row.
__global__ void k_pass_z(CsrD A, int64_t n, double t, int32_t* keep, double* part) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
    const int64_t mid = lb(A.ci, p0, p1, (int)n);
    int c = 0;
    double sq = 0.0;
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      if (modulus_at(A, n, p0, mid, p1, p) > t) ++c;
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

// The kept entries (|z| > t) of every top row, in order, at out_rp[i].
__global__ void k_compact_z(CsrD A, int64_t n, double t, const int64_t* out_rp, int32_t* out_ci, double* out_v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane_id()) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
    const int64_t mid = lb(A.ci, p0, p1, (int)n);
    int64_t o = out_rp[i];
    for (int64_t pb = p0; pb < p1; pb += 32) {
      const int64_t p = pb + lane_id();
      const bool k = p < p1 && modulus_at(A, n, p0, mid, p1, p) > t;
      const unsigned m = __ballot_sync(FULL, k);
      if (k) {
        out_ci[o + __popc(m & lt)] = A.ci[p];
        out_v[o + __popc(m & lt)] = A.v[p];
      }
      o += __popc(m);
    }
  }
}

// Complex entries of each top row: the union of columns j (left half) and c - n (right half).
// One thread per row (a sequential merge of the two sorted halves).
template <bool WRITE>
__global__ void k_extract_z(CsrD A, int64_t n, int32_t* cnt, const int64_t* out_rp, int32_t* out_ci, double* out_vz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
  const int64_t mid = lb(A.ci, p0, p1, (int)n);
  int64_t l = p0, r = mid, o = WRITE ? out_rp[i] : 0;
  int k = 0;
  while (l < mid || r < p1) {
    const int cl = l < mid ? A.ci[l] : INT_MAX;
    const int cr = r < p1 ? A.ci[r] - (int)n : INT_MAX;
    const int c = min(cl, cr);
    double re = 0.0, im = 0.0;
    if (cl == c) re = A.v[l++];
    if (cr == c) im = -A.v[r++];
    if (WRITE) {
      out_ci[o] = c;
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
  if (n == 0) {
    SX_CUDA(cudaMemsetAsync(top.rp.p, 0, sizeof(int64_t), s));
    return;
  }
  const int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sms_z() * 64);
  k_embed_top<<<blocks, 256, 0, s>>>(n, rp, ci, vz, top.rp.p, top.ci.p, top.v.p);
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
  if (top.n == 0) return 0.0;
  const int blocks = (int)std::min<int64_t>((top.n + 7) / 8, (int64_t)sms_z() * 64);
  k_pass_z<<<blocks, 256, 0, s>>>(top, n, t, keep, part);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  return reduce_sum(part, top.n, s, hs);
}

void compact_complex(const CsrD& top, int64_t n, double t, const int32_t* keep, cudaStream_t s, CsrOwned& out,
                     HostScalars& hs) {
  out.n = top.n;
  out.rp.reset(top.n + 1, s);
  out.nnz = scan_counts(keep, top.n, out.rp.p, s, hs);
  out.ci.reset(out.nnz, s);
  out.v.reset(out.nnz, s);
  if (top.n == 0) return;
  const int blocks = (int)std::min<int64_t>((top.n + 7) / 8, (int64_t)sms_z() * 64);
  k_compact_z<<<blocks, 256, 0, s>>>(top, n, t, out.rp.p, out.ci.p, out.v.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void extract_complex(const CsrD& top, int64_t n, cudaStream_t s, CsrOwned& pattern, DevBuf<double>& vz,
                     HostScalars& hs) {
  pattern.n = top.n;
  pattern.rp.reset(top.n + 1, s);
  DevBuf<int32_t> cnt(top.n ? top.n : 1, s);
  const unsigned blocks = (unsigned)((top.n + 255) / 256);
  if (top.n) k_extract_z<false><<<blocks, 256, 0, s>>>(top, n, cnt.p, nullptr, nullptr, nullptr);
  SX_CUDA(cudaGetLastError());
  pattern.nnz = scan_counts(cnt.p, top.n, pattern.rp.p, s, hs);
  pattern.ci.reset(pattern.nnz, s);
  vz.reset(2 * pattern.nnz, s);
  if (top.n) k_extract_z<true><<<blocks, 256, 0, s>>>(top, n, nullptr, pattern.rp.p, pattern.ci.p, vz.p);
  SX_CUDA(cudaGetLastError());
  count_launches(top.n ? 2 : 0);
}

}  // namespace sexpm
