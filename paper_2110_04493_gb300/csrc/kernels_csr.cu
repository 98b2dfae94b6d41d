// Streaming CSR kernels of the method:
//  * the scan allocator that turns per-row counts into int64 row pointers,
//  * the sparse sum T^_0 += S^_i (Algorithm 4.2 step 3) and e^H = I + T^_N (step 5),
//  * norms, transposition, validation and equality tests used by the plan.
// These are bound by HBM bandwidth; each reads its operands once with coalesced
// warp-per-row accesses.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// |v| > t for finite v and t >= 0, decided on the bit patterns: non-negative doubles are
// ordered as their bit patterns read as unsigned integers, so the test takes no FP64
// instruction (the FP64 pipe is this GPU's scarce unit; the dropped sum of squares keeps it).
__device__ __forceinline__ bool above(double v, unsigned long long tb) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) > tb;
}
__device__ __forceinline__ unsigned long long bits_of(double t) { return (unsigned long long)__double_as_longlong(t); }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

template <typename T>
__device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  __syncthreads();
  if (lane_id() == 0) red[warp_id()] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T t = lane_id() < nw ? red[lane_id()] : T(0);
  return warp_sum(t);
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    SX_CUDA(cudaGetDevice(&dev));
    SX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

// Fixed reduction grid: results do not depend on timing, only on this constant.
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

__global__ void k_final_sum(const double* part, int m, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_partial_sum(const double* x, int64_t n, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_partial_sumsq(const double* x, int64_t n, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ---- scan of int32 counts into int64 row pointers
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_tiles(const int32_t* cnt, int64_t n, int64_t* tile_sum) {
  __shared__ long long red[32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = t0 + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += cnt[i];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
}

__global__ void k_scan_tile_sums(int64_t* tile_sum, int64_t m, int64_t* total) {
  // single block: exclusive scan of m tile sums in chunks of blockDim
  __shared__ long long wsum[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < m; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const long long v = i < m ? tile_sum[i] : 0;
    long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(FULL, incl, o);
      if (lane_id() >= o) incl += y;
    }
    if (lane_id() == 31) wsum[warp_id()] = incl;
    __syncthreads();
    if (warp_id() == 0) {
      const int nw = blockDim.x >> 5;
      long long w = lane_id() < nw ? wsum[lane_id()] : 0;
      long long wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, wi, o);
        if (lane_id() >= o) wi += y;
      }
      if (lane_id() < nw) wsum[lane_id()] = wi - w;
    }
    __syncthreads();
    const long long excl = carry + wsum[warp_id()] + incl - v;
    if (i < m) tile_sum[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int32_t* cnt, int64_t n, const int64_t* tile_off, int64_t* rp) {
  // each thread owns kScanItems consecutive items
  __shared__ long long wsum[32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  const int64_t i0 = t0 + (int64_t)threadIdx.x * kScanItems;
  long long loc[kScanItems];
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = i0 + k;
    loc[k] = i < n ? cnt[i] : 0;
    s += loc[k];
  }
  long long incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(FULL, incl, o);
    if (lane_id() >= o) incl += y;
  }
  if (lane_id() == 31) wsum[warp_id()] = incl;
  __syncthreads();
  if (warp_id() == 0) {
    const int nw = blockDim.x >> 5;
    long long w = lane_id() < nw ? wsum[lane_id()] : 0;
    long long wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(FULL, wi, o);
      if (lane_id() >= o) wi += y;
    }
    if (lane_id() < nw) wsum[lane_id()] = wi - w;
  }
  __syncthreads();
  long long run = tile_off[blockIdx.x] + wsum[warp_id()] + incl - s;
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = i0 + k;
    run += loc[k];
    if (i < n) rp[i + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rp[0] = 0;
}

// ---- C = A + beta B, thread per row merge (rows of the Taylor terms are short)
// A non-null `status` that is set (an operand was not formed) stops the add kernels.
__global__ void k_add_count(CsrD A, CsrD B, int32_t* cnt, const int32_t* status) {
  if (status && *status) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int64_t p = A.rp[i], pe = A.rp[i + 1], q = B.rp[i], qe = B.rp[i + 1];
  int c = 0;
  while (p < pe && q < qe) {
    const int ca = A.ci[p], cb = B.ci[q];
    p += (ca <= cb);
    q += (cb <= ca);
    ++c;
  }
  cnt[i] = c + (int)(pe - p) + (int)(qe - q);
}

__global__ void k_add_write(CsrD A, CsrD B, double beta, const int64_t* rp, int32_t* ci, double* v,
                            const int32_t* status) {
  if (status && *status) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int64_t p = A.rp[i], pe = A.rp[i + 1], q = B.rp[i], qe = B.rp[i + 1];
  int64_t o = rp[i];
  while (p < pe || q < qe) {
    const int ca = p < pe ? A.ci[p] : INT32_MAX;
    const int cb = q < qe ? B.ci[q] : INT32_MAX;
    if (ca < cb) {
      ci[o] = ca; v[o] = A.v[p]; ++p;
    } else if (cb < ca) {
      ci[o] = cb; v[o] = beta * B.v[q]; ++q;
    } else {
      ci[o] = ca; v[o] = A.v[p] + beta * B.v[q]; ++p; ++q;
    }
    ++o;
  }
}

// ---- C = I + A
__device__ __forceinline__ int64_t lower_bound_col(const int32_t* ci, int64_t lo, int64_t hi, int c) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_eye_count(CsrD A, int32_t* cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
  const int64_t p = lower_bound_col(A.ci, p0, p1, (int)i);
  cnt[i] = (int)(p1 - p0) + ((p < p1 && A.ci[p] == (int)i) ? 0 : 1);
}

__global__ void k_eye_write(CsrD A, const int64_t* rp, int32_t* ci, double* v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
    const int64_t pos = lower_bound_col(A.ci, p0, p1, (int)i);
    const bool has = pos < p1 && A.ci[pos] == (int)i;
    const int64_t o = rp[i];
    for (int64_t q = p0 + lane_id(); q < p1; q += 32) {
      const int64_t d = o + (q - p0) + ((!has && q >= pos) ? 1 : 0);
      ci[d] = A.ci[q];
      v[d] = (has && q == pos) ? 1.0 + A.v[q] : A.v[q];
    }
    if (!has && lane_id() == 0) {
      ci[o + (pos - p0)] = (int)i;
      v[o + (pos - p0)] = 1.0;
    }
  }
}

__global__ void k_scale(const double* x, double alpha, int64_t n, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = alpha * x[i];
}

// ---- transpose: column counts, scan, scatter with atomic cursors, per-row sort
__global__ void k_col_count(CsrD A, int32_t* cnt) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < A.nnz; q += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[A.ci[q]], 1);
}

__global__ void k_transpose_scatter(CsrD A, const int64_t* rp_t, int32_t* cursor, int32_t* ci_t, double* v_t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
    const int c = A.ci[q];
    const int64_t d = rp_t[c] + atomicAdd(&cursor[c], 1);
    ci_t[d] = (int)i;
    v_t[d] = A.v[q];
  }
}

// ---- batched (block-diagonal) helpers: inst[i] is the instance of row i; instances own
//      contiguous row ranges seg[b] .. seg[b+1]

// Algorithm 4.1 pass with a threshold per instance: row_part[i] = sum_{|v| <= t_inst} v^2 over
// row i, keep[i] = #{|v| > t_inst}.  One warp per row.
// A non-null `status` that is set means A was not formed (a capacity was exceeded): nothing runs.
__global__ void k_filter_pass_seg(CsrD A, const int32_t* inst, const double* t_inst, int32_t* keep, double* row_part,
                                  const int32_t* status) {
  if (status && *status) return;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const unsigned long long tb = bits_of(t_inst[inst[i]]);
    int c = 0;
    double sq = 0.0;
    for (int64_t q = A.rp[i] + lane_id(); q < A.rp[i + 1]; q += 32) {
      const double v = A.v[q];
      if (above(v, tb)) ++c; else sq = fma(v, v, sq);
    }
    c = warp_sum(c);
    sq = warp_sum(sq);
    if (lane_id() == 0) {
      keep[i] = c;
      row_part[i] = sq;
    }
  }
}

// out[b] = sum of x over the rows of instance b (one block per instance, fixed order).
__global__ void k_seg_sum(const double* x, const int64_t* seg, double* out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int64_t i = seg[b] + threadIdx.x; i < seg[b + 1]; i += blockDim.x) s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[b] = s;
}

__global__ void k_compact_seg(CsrD A, const int32_t* inst, const double* t_inst, const int64_t* rp_out, int32_t* ci_out,
                              double* v_out, const int32_t* status) {
  if (status && *status) return;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane_id()) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const unsigned long long tb = bits_of(t_inst[inst[i]]);
    const int64_t q0 = A.rp[i], q1 = A.rp[i + 1];
    int64_t o = rp_out[i];
    // four chunks of 32 per round: every load of the round is issued before the first store
    for (int64_t qb = q0; qb < q1; qb += 128) {
      double v[4];
      int c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t q = qb + 32 * u + lane_id();
        v[u] = q < q1 ? A.v[q] : 0.0;
        c[u] = q < q1 ? A.ci[q] : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool keep = qb + 32 * u + lane_id() < q1 && above(v[u], tb);
        const unsigned m = __ballot_sync(FULL, keep);
        if (keep) {
          const int64_t d = o + __popc(m & lt);
          ci_out[d] = c[u];
          v_out[d] = v[u];
        }
        o += __popc(m);
      }
    }
  }
}

// out_v = factor[inst[row]] * v, one warp per row.
__global__ void k_scale_rows(CsrD A, const int32_t* inst, const double* factor, double* out_v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const double f = factor[inst[i]];
    for (int64_t q = A.rp[i] + lane_id(); q < A.rp[i + 1]; q += 32) out_v[q] = f * A.v[q];
  }
}

// Instance of every row: the largest b with seg[b] <= i.
__global__ void k_instance_of_row(const int64_t* seg, int count, int64_t n, int32_t* inst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg[mid] <= i) lo = mid; else hi = mid - 1;
  }
  inst[i] = lo;
}

// Row flag from an instance flag.
__global__ void k_row_flags(const int32_t* inst, const uint8_t* inst_flag, int64_t n, uint8_t* row_flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) row_flag[i] = inst_flag[inst[i]];
}

// Copy instance block X (n_b rows) into the block-diagonal arrays at (row0, nnz0).
__global__ void k_block_put(CsrD X, int64_t row0, int64_t nnz0, int64_t* rp, int32_t* ci, double* v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < X.n; i += stride) rp[row0 + i] = X.rp[i] + nnz0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < X.nnz; q += stride) {
    ci[nnz0 + q] = X.ci[q] + (int)row0;
    v[nnz0 + q] = X.v[q];
  }
}

// Rows [row0, row0 + nb) of E as an nb x nb CSR (columns shifted by -row0).
__global__ void k_block_get(CsrD E, int64_t row0, int64_t nb, int64_t* rp, int32_t* ci, double* v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nnz0 = E.rp[row0];
  const int64_t nnz1 = E.rp[row0 + nb];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nb; i += stride) rp[i] = E.rp[row0 + i] - nnz0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz1 - nnz0; q += stride) {
    ci[q] = E.ci[nnz0 + q] - (int)row0;
    v[q] = E.v[nnz0 + q];
  }
}

__global__ void k_gather_rp(const int64_t* rp, const int64_t* seg, int count, int64_t* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b <= count) out[b] = rp[seg[b]];
}

// ---- symmetric part: (A + A^T)/2 on the pattern of A; entries whose mirror is absent are flagged
__device__ __forceinline__ int64_t lb_col(const int32_t* ci, int64_t lo, int64_t hi, int c) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_sym_gather(CsrD A, double* out_v, uint8_t* lone, unsigned long long* n_lone) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      const int j = A.ci[p];
      const double a = A.v[p];
      if (j == (int)i) {
        out_v[p] = a;
        lone[p] = 0;
        continue;
      }
      const int64_t q0 = A.rp[j], q1 = A.rp[j + 1];
      const int64_t q = lb_col(A.ci, q0, q1, (int)i);
      if (q < q1 && A.ci[q] == (int)i) {
        out_v[p] = 0.5 * (a + A.v[q]);
        lone[p] = 0;
      } else {
        out_v[p] = 0.5 * a;
        lone[p] = 1;
        atomicAdd(n_lone, 1ull);
      }
    }
  }
}

// Per-row count and compaction of the flagged entries (warp per row).
__global__ void k_flag_count(CsrD A, const uint8_t* flag, int32_t* cnt) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    int c = 0;
    for (int64_t p = A.rp[i] + lane_id(); p < A.rp[i + 1]; p += 32) c += flag[p];
    c = warp_sum(c);
    if (lane_id() == 0) cnt[i] = c;
  }
}

__global__ void k_flag_compact(CsrD A, const double* vals, const uint8_t* flag, const int64_t* rp_out, int32_t* ci_out,
                               double* v_out) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane_id()) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    const int64_t q0 = A.rp[i], q1 = A.rp[i + 1];
    int64_t o = rp_out[i];
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane_id();
      const bool keep = q < q1 && flag[q];
      const unsigned m = __ballot_sync(FULL, keep);
      if (keep) {
        const int64_t d = o + __popc(m & lt);
        ci_out[d] = A.ci[q];
        v_out[d] = vals[q];
      }
      o += __popc(m);
    }
  }
}

// ---- equality (B == sign * A, same pattern) and validation; flag[0] set on mismatch / invalid
__global__ void k_equal(CsrD A, CsrD B, double sign, int* flag) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < A.nnz; q += (int64_t)gridDim.x * blockDim.x)
    if (A.ci[q] != B.ci[q] || A.v[q] != sign * B.v[q]) atomicOr(flag, 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= A.n; i += (int64_t)gridDim.x * blockDim.x)
    if (A.rp[i] != B.rp[i]) atomicOr(flag, 1);
}

__global__ void k_valid(CsrD A, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
  if (i == 0 && p0 != 0) atomicOr(flag, 1);
  if (i == A.n - 1 && p1 != A.nnz) atomicOr(flag, 1);
  if (p0 < 0 || p1 < p0 || p1 > A.nnz) { atomicOr(flag, 1); return; }
  int prev = -1;
  for (int64_t p = p0; p < p1; ++p) {
    const int c = A.ci[p];
    if (c <= prev || c >= A.n || !isfinite(A.v[p])) atomicOr(flag, 1);
    prev = c;
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

HostScalars::HostScalars() {
  SX_CUDA(cudaMallocHost(&d, 8 * sizeof(double)));
  SX_CUDA(cudaMallocHost(&i, 8 * sizeof(int64_t)));
}
HostScalars::~HostScalars() {
  if (d) cudaFreeHost(d);
  if (i) cudaFreeHost(i);
}

static double finish_partials(const double* part, int m, cudaStream_t s, HostScalars& hs) {
  DevBuf<double> out(1, s);
  k_final_sum<<<1, 1024, 0, s>>>(part, m, out.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(hs.d, out.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return hs.d[0];
}

double reduce_sum(const double* x, int64_t n, cudaStream_t s, HostScalars& hs) {
  if (n == 0) return 0.0;
  DevBuf<double> part(kRedBlocks, s);
  k_partial_sum<<<kRedBlocks, kRedThreads, 0, s>>>(x, n, part.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  return finish_partials(part.p, kRedBlocks, s, hs);
}

double sum_squares(const CsrD& A, cudaStream_t s, HostScalars& hs) {
  if (A.nnz == 0) return 0.0;
  DevBuf<double> part(kRedBlocks, s);
  k_partial_sumsq<<<kRedBlocks, kRedThreads, 0, s>>>(A.v, A.nnz, part.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  return finish_partials(part.p, kRedBlocks, s, hs);
}

int64_t scan_counts(const int32_t* cnt, int64_t n, int64_t* rp, cudaStream_t s, HostScalars& hs) {
  if (n == 0) {
    SX_CUDA(cudaMemsetAsync(rp, 0, sizeof(int64_t), s));
    return 0;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  DevBuf<int64_t> ts(tiles + 1, s);
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, ts.p);
  k_scan_tile_sums<<<1, 1024, 0, s>>>(ts.p, tiles, ts.p + tiles);
  k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, ts.p, rp);
  SX_CUDA(cudaGetLastError());
  count_launches(3);
  SX_CUDA(cudaMemcpyAsync(hs.i, ts.p + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return hs.i[0];
}

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

void scan_counts_dev(const int32_t* cnt, int64_t n, int64_t* rp, int64_t* ts, cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, ts);
  k_scan_tile_sums<<<1, 1024, 0, s>>>(ts, tiles, ts + tiles);
  k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, ts, rp);
  SX_CUDA(cudaGetLastError());
  count_launches(3);
}

void add(const CsrD& A, const CsrD& B, double beta, cudaStream_t s, CsrOwned& C, HostScalars& hs) {
  const int64_t n = A.n;
  C.n = n;
  C.rp.reset(n + 1, s);
  DevBuf<int32_t> cnt(n ? n : 1, s);
  const unsigned g = (unsigned)((n + 255) / 256);
  if (n) k_add_count<<<g, 256, 0, s>>>(A, B, cnt.p, nullptr);
  SX_CUDA(cudaGetLastError());
  count_launches(n ? 1 : 0);
  C.nnz = scan_counts(cnt.p, n, C.rp.p, s, hs);
  C.ci.reset(C.nnz, s);
  C.v.reset(C.nnz, s);
  if (n) k_add_write<<<g, 256, 0, s>>>(A, B, beta, C.rp.p, C.ci.p, C.v.p, nullptr);
  SX_CUDA(cudaGetLastError());
  count_launches(n ? 1 : 0);
}

void add_identity(const CsrD& A, cudaStream_t s, CsrOwned& C, HostScalars& hs) {
  const int64_t n = A.n;
  C.n = n;
  C.rp.reset(n + 1, s);
  DevBuf<int32_t> cnt(n ? n : 1, s);
  if (n) k_eye_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, cnt.p);
  SX_CUDA(cudaGetLastError());
  count_launches(n ? 1 : 0);
  C.nnz = scan_counts(cnt.p, n, C.rp.p, s, hs);
  C.ci.reset(C.nnz, s);
  C.v.reset(C.nnz, s);
  if (n) {
    const int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sm_count() * 64);
    k_eye_write<<<blocks, 256, 0, s>>>(A, C.rp.p, C.ci.p, C.v.p);
    count_launches(1);
  }
  SX_CUDA(cudaGetLastError());
}

void scale_values(const double* x, double alpha, int64_t n, double* y, cudaStream_t s) {
  if (!n) return;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
  k_scale<<<blocks, 256, 0, s>>>(x, alpha, n, y);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void transpose(const CsrD& A, cudaStream_t s, CsrOwned& T, HostScalars& hs) {
  const int64_t n = A.n;
  T.n = n;
  T.rp.reset(n + 1, s);
  DevBuf<int32_t> cnt(n ? n : 1, s);
  SX_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.count * sizeof(int32_t), s));
  if (A.nnz) k_col_count<<<(unsigned)std::min<int64_t>((A.nnz + 255) / 256, 65535), 256, 0, s>>>(A, cnt.p);
  SX_CUDA(cudaGetLastError());
  count_launches(A.nnz ? 1 : 0);
  T.nnz = scan_counts(cnt.p, n, T.rp.p, s, hs);
  T.ci.reset(T.nnz, s);
  T.v.reset(T.nnz, s);
  SX_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.count * sizeof(int32_t), s));
  if (n) {
    k_transpose_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, T.rp.p, cnt.p, T.ci.p, T.v.p);
    count_launches(1);
    sort_rows(n, T.rp.p, T.ci.p, T.v.p, s);
  }
  SX_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- batched helpers (host)

void seg_sums(const double* x, const int64_t* seg, int count, double* out_host, cudaStream_t s) {
  if (count == 0) return;
  DevBuf<double> out(count, s);
  k_seg_sum<<<count, 256, 0, s>>>(x, seg, out.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(out_host, out.p, count * sizeof(double), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
}

void filter_pass_seg(const CsrD& A, const int32_t* inst, const double* t_inst, int32_t* keep, double* row_part,
                     const int64_t* seg, int count, double* sums_host, cudaStream_t s) {
  if (A.n) {
    const int blocks = (int)std::min<int64_t>((A.n + 7) / 8, (int64_t)sm_count() * 64);
    k_filter_pass_seg<<<blocks, 256, 0, s>>>(A, inst, t_inst, keep, row_part, nullptr);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
  }
  seg_sums(row_part, seg, count, sums_host, s);
}

// status |= bit when the size at *rp_n exceeds cap (need = the largest size asked for); skipped
// once the status is set.
__global__ void k_csr_cap_check(const int64_t* rp_n, int64_t cap, int32_t* status, unsigned long long* need,
                                int32_t bit) {
  if (*status) return;
  const long long total = *rp_n;
  atomicMax(need, (unsigned long long)total);
  if (total > cap) atomicOr(status, bit);
}

void add_dev(const CsrD& A, const CsrD& B, double beta, int32_t* cnt, int64_t* rp_out, int64_t* ts, int32_t* ci_out,
             double* v_out, int64_t cap, int32_t* status, unsigned long long* need, int32_t bit, cudaStream_t s) {
  const int64_t n = A.n;
  const unsigned g = (unsigned)((n + 255) / 256);
  k_add_count<<<g, 256, 0, s>>>(A, B, cnt, status);
  scan_counts_dev(cnt, n, rp_out, ts, s);
  k_csr_cap_check<<<1, 1, 0, s>>>(rp_out + n, cap, status, need, bit);
  k_add_write<<<g, 256, 0, s>>>(A, B, beta, rp_out, ci_out, v_out, status);
  check_cuda(cudaGetLastError(), "add_dev");
  count_launches(3);
}

void seg_sums_dev(const double* x, const int64_t* seg, int count, double* out, cudaStream_t s) {
  k_seg_sum<<<count, 256, 0, s>>>(x, seg, out);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void filter_pass_seg_dev(const CsrD& A, const int32_t* inst, const double* t_inst, int32_t* keep, double* row_part,
                         const int32_t* status, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((A.n + 7) / 8, (int64_t)sm_count() * 64);
  k_filter_pass_seg<<<blocks, 256, 0, s>>>(A, inst, t_inst, keep, row_part, status);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void compact_seg_dev(const CsrD& A, const int32_t* inst, const double* t_inst, const int64_t* rp_out, int32_t* ci_out,
                     double* v_out, const int32_t* status, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((A.n + 7) / 8, (int64_t)sm_count() * 64);
  k_compact_seg<<<blocks, 256, 0, s>>>(A, inst, t_inst, rp_out, ci_out, v_out, status);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void compact_seg(const CsrD& A, const int32_t* inst, const double* t_inst, CsrOwned& C, cudaStream_t s) {
  if (A.n == 0) return;
  const int blocks = (int)std::min<int64_t>((A.n + 7) / 8, (int64_t)sm_count() * 64);
  k_compact_seg<<<blocks, 256, 0, s>>>(A, inst, t_inst, C.rp.p, C.ci.p, C.v.p, nullptr);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void scale_rows(const CsrD& A, const int32_t* inst, const double* factor, double* out_v, cudaStream_t s) {
  if (A.n == 0) return;
  const int blocks = (int)std::min<int64_t>((A.n + 7) / 8, (int64_t)sm_count() * 64);
  k_scale_rows<<<blocks, 256, 0, s>>>(A, inst, factor, out_v);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void instance_of_row(const int64_t* seg, int count, int64_t n, int32_t* inst, cudaStream_t s) {
  if (n == 0) return;
  k_instance_of_row<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seg, count, n, inst);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void row_flags(const int32_t* inst, const uint8_t* inst_flag, int64_t n, uint8_t* row_flag, cudaStream_t s) {
  if (n == 0) return;
  k_row_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(inst, inst_flag, n, row_flag);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void block_put(const CsrD& X, int64_t row0, int64_t nnz0, int64_t* rp, int32_t* ci, double* v, cudaStream_t s) {
  const int64_t work = std::max<int64_t>(X.n, X.nnz);
  if (work == 0) return;
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 16);
  k_block_put<<<blocks, 256, 0, s>>>(X, row0, nnz0, rp, ci, v);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void block_get(const CsrD& E, int64_t row0, int64_t nb, int64_t nnz_b, CsrOwned& out, cudaStream_t s) {
  out.n = nb;
  out.nnz = nnz_b;
  out.rp.reset(nb + 1, s);
  out.ci.reset(nnz_b, s);
  out.v.reset(nnz_b, s);
  const int64_t work = std::max<int64_t>(nb + 1, nnz_b);
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 16);
  k_block_get<<<blocks, 256, 0, s>>>(E, row0, nb, out.rp.p, out.ci.p, out.v.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

void gather_row_ptr(const int64_t* rp, const int64_t* seg, int count, int64_t* out_host, cudaStream_t s) {
  DevBuf<int64_t> out(count + 1, s);
  k_gather_rp<<<(count + 256) / 256, 256, 0, s>>>(rp, seg, count, out.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(out_host, out.p, (count + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
}

void symmetric_part(const CsrD& A, cudaStream_t s, CsrOwned& S, HostScalars& hs) {
  const int64_t n = A.n;
  S.n = n;
  S.nnz = A.nnz;
  S.rp.reset(n + 1, s);
  S.ci.reset(A.nnz, s);
  S.v.reset(A.nnz, s);
  if (n == 0) {
    SX_CUDA(cudaMemsetAsync(S.rp.p, 0, sizeof(int64_t), s));
    return;
  }
  SX_CUDA(cudaMemcpyAsync(S.rp.p, A.rp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (A.nnz) SX_CUDA(cudaMemcpyAsync(S.ci.p, A.ci, A.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  DevBuf<uint8_t> lone(A.nnz ? A.nnz : 1, s);
  DevBuf<unsigned long long> cntr(1, s);
  SX_CUDA(cudaMemsetAsync(cntr.p, 0, sizeof(unsigned long long), s));
  const int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sm_count() * 64);
  k_sym_gather<<<blocks, 256, 0, s>>>(A, S.v.p, lone.p, cntr.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(hs.i, cntr.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  unsigned long long nl;
  std::memcpy(&nl, hs.i, sizeof(nl));
  if (nl == 0) return;
  // entries whose mirror is absent: U (halved values) ; S <- S_avg + U^T
  CsrOwned U, Ut, R;
  U.n = n;
  U.rp.reset(n + 1, s);
  DevBuf<int32_t> cnt(n, s);
  k_flag_count<<<blocks, 256, 0, s>>>(A, lone.p, cnt.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  U.nnz = scan_counts(cnt.p, n, U.rp.p, s, hs);
  U.ci.reset(U.nnz, s);
  U.v.reset(U.nnz, s);
  k_flag_compact<<<blocks, 256, 0, s>>>(A, S.v.p, lone.p, U.rp.p, U.ci.p, U.v.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  transpose(U.view(), s, Ut, hs);
  add(S.view(), Ut.view(), 1.0, s, R, hs);
  S = std::move(R);
}

bool csr_equal(const CsrD& A, const CsrD& B, double sign, cudaStream_t s, HostScalars& hs) {
  if (A.n != B.n || A.nnz != B.nnz) return false;
  DevBuf<int> flag(1, s);
  SX_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  k_equal<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((std::max(A.nnz, A.n + 1) + 255) / 256, 65535)), 256, 0, s>>>(
      A, B, sign, flag.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(hs.i, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  int f;
  std::memcpy(&f, hs.i, sizeof(int));
  return f == 0;
}

bool csr_valid(const CsrD& A, cudaStream_t s, HostScalars& hs) {
  if (A.n == 0) return A.nnz == 0;
  DevBuf<int> flag(1, s);
  SX_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  k_valid<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A, flag.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(hs.i, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  int f;
  std::memcpy(&f, hs.i, sizeof(int));
  return f == 0;
}

}  // namespace sexpm
