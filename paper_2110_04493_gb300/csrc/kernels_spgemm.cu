// Sparse product of Algorithm 4.2 with its fused scaling and sum:
//     C = (A B) / div + beta D
// used for the Taylor terms S~_i = S^_{i-1} H_0 / i (Eq. 4.10) and the squaring
// steps T~_i = 2 T^_{i-1} + T^_{i-1}^2 (Eq. 4.15).
//
// Row-wise (Gustavson) product, one thread block per output row.  The output
// pattern of a row is held as a bitmap over the row's column span
// [base, hi] (base rounded down to a multiple of 32).  A symbolic pass builds
// the bitmap and counts its bits; the numeric pass rebuilds it, turns it into
// per-word prefix counts, and uses rank(c) = pre[c/32] + popc(bm[c/32] & below(c))
// as a perfect hash into a dense accumulator of exactly nnz(row) doubles.  The
// accumulator is therefore already in sorted column order and is written out
// with coalesced stores; no hash probing and no sort are needed.
//
// Rows are binned by the shared memory they need (bitmap, prefix counts and
// accumulator); the widest rows use a per-block global-memory scratch slice.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kClasses = 5;
// Shared-memory budget and block size of each row class; the last class uses global scratch.
constexpr int kClassBytes[kClasses] = {4 << 10, 16 << 10, 64 << 10, 200 << 10, INT_MAX};
constexpr int kClassThreads[kClasses] = {64, 128, 256, 512, 512};

__host__ __device__ constexpr int class_limit(int c) {
  return c == 0 ? (4 << 10) : c == 1 ? (16 << 10) : c == 2 ? (64 << 10) : c == 3 ? (200 << 10) : INT_MAX;
}

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Block-wide sum; every thread receives the total.  `red` is a 32-entry shared scratch.
template <typename T>
__device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  __syncthreads();
  if (lane_id() == 0) red[warp_id()] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T t = lane_id() < nw ? red[lane_id()] : T(0);
  t = warp_sum(t);
  return t;
}

// Sets the bits of column offsets c (relative to the row's base) held by the active lanes.
// Active lanes form a prefix of the warp and their offsets increase with the lane index,
// so lanes hitting the same 32-bit word are contiguous: OR them together with a segmented
// down-sweep and let the first lane of each segment issue one atomicOr.
__device__ __forceinline__ void warp_set_bits(uint32_t* bm, int c, bool act) {
  const int lane = lane_id();
  int w = act ? (c >> 5) : -1;
  uint32_t bits = act ? (1u << (c & 31)) : 0u;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t ob = __shfl_down_sync(FULL, bits, off);
    int ow = __shfl_down_sync(FULL, w, off);
    if (lane + off < 32 && ow == w) bits |= ob;
  }
  int pw = __shfl_up_sync(FULL, w, 1);
  if (act && (lane == 0 || pw != w)) atomicOr(&bm[w], bits);
}

// Position of the r-th (0-based) set bit of m; m has more than r set bits.
__device__ __forceinline__ int select_bit(uint32_t m, int r) {
  int pos = 0;
  int c = __popc(m & 0xffffu);
  if (r >= c) { r -= c; m >>= 16; pos += 16; }
  c = __popc(m & 0xffu);
  if (r >= c) { r -= c; m >>= 8; pos += 8; }
  c = __popc(m & 0xfu);
  if (r >= c) { r -= c; m >>= 4; pos += 4; }
  c = __popc(m & 0x3u);
  if (r >= c) { r -= c; m >>= 2; pos += 2; }
  c = int(m & 1u);
  if (r >= c) pos += 1;
  return pos;
}

// Per row: column span of the product row (A B plus the pattern of D) and its product count.
// One warp per row.
__global__ void k_analysis(CsrD A, CsrD B, CsrD D, int32_t* base, int32_t* words, int64_t* flops) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    int lo = INT_MAX, hi = -1;
    int64_t f = 0;
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    for (int64_t p = a0 + lane_id(); p < a1; p += 32) {
      const int k = A.ci[p];
      const int64_t b0 = B.rp[k], b1 = B.rp[k + 1];
      if (b1 > b0) {
        lo = min(lo, B.ci[b0]);
        hi = max(hi, B.ci[b1 - 1]);
        f += b1 - b0;
      }
    }
    if (D.n > 0 && lane_id() == 0) {
      const int64_t d0 = D.rp[i], d1 = D.rp[i + 1];
      if (d1 > d0) {
        lo = min(lo, D.ci[d0]);
        hi = max(hi, D.ci[d1 - 1]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(FULL, lo, o));
      hi = max(hi, __shfl_xor_sync(FULL, hi, o));
      f += __shfl_xor_sync(FULL, f, o);
    }
    if (lane_id() == 0) {
      if (hi < 0) {
        base[i] = 0;
        words[i] = 0;
      } else {
        const int b = lo & ~31;
        base[i] = b;
        words[i] = ((hi - b) >> 5) + 1;
      }
      flops[i] = f;
    }
  }
}

// Assign each row to a class by its shared-memory need (bytes); append row ids per class.
// mode 0: symbolic need 4 W; mode 1: numeric need 8 W + 8 cnt.
__global__ void k_classify(int64_t n, const int32_t* words, const int64_t* rp_out, int mode,
                           int32_t* lists, int64_t list_stride, unsigned long long* counts,
                           unsigned long long* maxneed) {
  __shared__ unsigned int cnt[kClasses];
  __shared__ unsigned long long off[kClasses];
  if (threadIdx.x < kClasses) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int cls = -1;
  unsigned int slot = 0;
  long long need = 0;
  if (i < n) {
    const long long W = words[i];
    if (mode == 0) {
      need = 4 * W;
    } else {
      need = 8 * W + 8 * (rp_out[i + 1] - rp_out[i]);
    }
    if (W > 0) {
      cls = 0;
      while (cls < kClasses - 1 && need > class_limit(cls)) ++cls;
      slot = atomicAdd(&cnt[cls], 1u);
      if (cls == kClasses - 1) atomicMax(maxneed, (unsigned long long)need);
    }
  }
  __syncthreads();
  if (threadIdx.x < kClasses) off[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], (unsigned long long)cnt[threadIdx.x]) : 0ull;
  __syncthreads();
  if (cls >= 0) lists[cls * list_stride + off[cls] + slot] = (int32_t)i;
}

// Symbolic pass: cnt[i] = number of distinct columns of row i of A B (+ pattern of D).
template <bool GLOBAL>
__global__ void k_symbolic(CsrD A, CsrD B, CsrD D, const int32_t* rows, int64_t nrows, const int32_t* base,
                           const int32_t* words, int32_t* cnt, uint32_t* gscratch, int64_t gstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int red[32];
  uint32_t* bm = GLOBAL ? gscratch + (int64_t)blockIdx.x * gstride : reinterpret_cast<uint32_t*>(smem);
  const int nwarps = blockDim.x >> 5;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int W = words[i];
    const int b = base[i];
    for (int w = threadIdx.x; w < W; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    for (int64_t p = a0 + warp_id(); p < a1; p += nwarps) {
      const int k = A.ci[p];
      const int64_t b0 = B.rp[k], b1 = B.rp[k + 1];
      for (int64_t q0 = b0; q0 < b1; q0 += 32) {
        const int64_t q = q0 + lane_id();
        const bool act = q < b1;
        warp_set_bits(bm, act ? B.ci[q] - b : 0, act);
      }
    }
    if (D.n > 0 && warp_id() == 0) {
      const int64_t d0 = D.rp[i], d1 = D.rp[i + 1];
      for (int64_t q0 = d0; q0 < d1; q0 += 32) {
        const int64_t q = q0 + lane_id();
        const bool act = q < d1;
        warp_set_bits(bm, act ? D.ci[q] - b : 0, act);
      }
    }
    __syncthreads();
    int c = 0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) c += __popc(bm[w]);
    c = block_sum(c, red);
    if (threadIdx.x == 0) cnt[i] = c;
    __syncthreads();
  }
}

// Numeric pass.  Shared layout per row: acc[cnt] doubles, bm[W] words, pre[W] prefix counts.
template <bool GLOBAL>
__global__ void k_numeric(CsrD A, CsrD B, CsrD D, double div, double beta, const int32_t* rows, int64_t nrows,
                          const int32_t* base, const int32_t* words, const int64_t* rp_out, int32_t* ci_out,
                          double* v_out, double* row_sq, double* row_diag, unsigned char* gscratch,
                          int64_t gstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int ired[32];
  __shared__ double dred[32];
  unsigned char* mem = GLOBAL ? gscratch + (int64_t)blockIdx.x * gstride : smem;
  const int nwarps = blockDim.x >> 5;
  const int T = blockDim.x;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int W = words[i];
    const int b = base[i];
    const int64_t o0 = rp_out[i];
    const int cnt = (int)(rp_out[i + 1] - o0);
    double* acc = reinterpret_cast<double*>(mem);
    uint32_t* bm = reinterpret_cast<uint32_t*>(acc + cnt);
    int* pre = reinterpret_cast<int*>(bm + W);
    for (int w = threadIdx.x; w < W; w += T) bm[w] = 0u;
    for (int k = threadIdx.x; k < cnt; k += T) acc[k] = 0.0;
    if (row_diag && threadIdx.x == 0) row_diag[i] = 0.0;
    __syncthreads();
    // 1. pattern bitmap (as in the symbolic pass)
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    for (int64_t p = a0 + warp_id(); p < a1; p += nwarps) {
      const int k = A.ci[p];
      const int64_t b0 = B.rp[k], b1 = B.rp[k + 1];
      for (int64_t q0 = b0; q0 < b1; q0 += 32) {
        const int64_t q = q0 + lane_id();
        const bool act = q < b1;
        warp_set_bits(bm, act ? B.ci[q] - b : 0, act);
      }
    }
    if (D.n > 0 && warp_id() == 0) {
      const int64_t d0 = D.rp[i], d1 = D.rp[i + 1];
      for (int64_t q0 = d0; q0 < d1; q0 += 32) {
        const int64_t q = q0 + lane_id();
        const bool act = q < d1;
        warp_set_bits(bm, act ? D.ci[q] - b : 0, act);
      }
    }
    __syncthreads();
    // 2. exclusive prefix of the per-word popcounts: each thread scans a contiguous chunk
    {
      const int ch = (W + T - 1) / T;
      const int w0 = min(W, threadIdx.x * ch), w1 = min(W, w0 + ch);
      int s = 0;
      for (int w = w0; w < w1; ++w) s += __popc(bm[w]);
      // block exclusive scan of s
      int incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, incl, o);
        if (lane_id() >= o) incl += y;
      }
      if (lane_id() == 31) ired[warp_id()] = incl;
      __syncthreads();
      if (warp_id() == 0) {
        int v = lane_id() < nwarps ? ired[lane_id()] : 0;
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(FULL, vi, o);
          if (lane_id() >= o) vi += y;
        }
        if (lane_id() < nwarps) ired[lane_id()] = vi - v;
      }
      __syncthreads();
      int run = ired[warp_id()] + incl - s;
      for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bm[w]);
      }
    }
    __syncthreads();
    // 3. accumulate the products a_ik b_kj at rank(j)
    for (int64_t p = a0 + warp_id(); p < a1; p += nwarps) {
      const int k = A.ci[p];
      const double a = A.v[p];
      const int64_t b0 = B.rp[k], b1 = B.rp[k + 1];
      for (int64_t q = b0 + lane_id(); q < b1; q += 32) {
        const int c = B.ci[q] - b;
        const int w = c >> 5;
        const int pos = pre[w] + __popc(bm[w] & ((1u << (c & 31)) - 1u));
        atomicAdd(&acc[pos], a * B.v[q]);
      }
    }
    __syncthreads();
    // 4. scaling (Taylor /i) and the fused beta D term (squaring +2T), in that order
    if (div != 1.0)
      for (int k = threadIdx.x; k < cnt; k += T) acc[k] = acc[k] / div;
    __syncthreads();
    if (D.n > 0) {
      const int64_t d0 = D.rp[i], d1 = D.rp[i + 1];
      for (int64_t q = d0 + threadIdx.x; q < d1; q += T) {
        const int c = D.ci[q] - b;
        const int w = c >> 5;
        const int pos = pre[w] + __popc(bm[w] & ((1u << (c & 31)) - 1u));
        acc[pos] += beta * D.v[q];
      }
    }
    __syncthreads();
    // 5. write the row in column order; per-row sum of squares and diagonal
    double sq = 0.0;
    for (int k = threadIdx.x; k < cnt; k += T) {
      int lo = 0, hi = W - 1;  // largest w with pre[w] <= k
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= k) lo = mid; else hi = mid - 1;
      }
      const int col = b + lo * 32 + select_bit(bm[lo], k - pre[lo]);
      const double v = acc[k];
      ci_out[o0 + k] = col;
      v_out[o0 + k] = v;
      sq += v * v;
      if (row_diag && col == i) row_diag[i] = v;
    }
    if (row_sq) {
      sq = block_sum(sq, dred);
      if (threadIdx.x == 0) row_sq[i] = sq;
    }
    __syncthreads();
  }
}

__global__ void k_zero_rows(const int32_t* words, int64_t n, double* row_sq, double* row_diag, int32_t* cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && words[i] == 0) {
    if (row_sq) row_sq[i] = 0.0;
    if (row_diag) row_diag[i] = 0.0;
    cnt[i] = 0;
  }
}

__global__ void k_sum_i64(const int64_t* x, int64_t n, unsigned long long* out) {
  __shared__ long long red[32];
  long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) atomicAdd(out, (unsigned long long)s);
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    SX_CUDA(cudaGetDevice(&dev));
    SX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

void set_smem_limits() {
  static bool done = false;
  if (done) return;
  int cap = kClassBytes[kClasses - 2];
  SX_CUDA(cudaFuncSetAttribute(k_symbolic<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  SX_CUDA(cudaFuncSetAttribute(k_numeric<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  done = true;
}

}  // namespace

namespace {
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  bool on;
  cudaStream_t s;
  EventPair(bool enable, cudaStream_t st) : on(enable), s(st) {
    if (on) {
      SX_CUDA(cudaEventCreate(&a));
      SX_CUDA(cudaEventCreate(&b));
    }
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  void start() { if (on) SX_CUDA(cudaEventRecord(a, s)); }
  double stop() {
    if (!on) return 0.0;
    SX_CUDA(cudaEventRecord(b, s));
    SX_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    SX_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
};
}  // namespace

int64_t spgemm(const CsrD& A, const CsrD& B, const CsrD& D, double div, double beta, cudaStream_t s, CsrOwned& C,
               RowStats* stats, HostScalars& hs, SpgemmTimes* times) {
  const int64_t n = A.n;
  EventPair ev_sym(times != nullptr, s), ev_num(times != nullptr, s);
  set_smem_limits();
  C.n = n;
  C.rp.reset(n + 1, s);
  if (stats) {
    stats->sq.reset(n, s);
    stats->diag.reset(n, s);
  }
  if (n == 0) {
    SX_CUDA(cudaMemsetAsync(C.rp.p, 0, sizeof(int64_t), s));
    C.nnz = 0;
    return 0;
  }
  DevBuf<int32_t> base(n, s), words(n, s), cnt(n, s), lists((size_t)n * kClasses, s);
  DevBuf<int64_t> flops(n, s);
  DevBuf<unsigned long long> ctr(2 * kClasses + 4, s);
  SX_CUDA(cudaMemsetAsync(ctr.p, 0, ctr.count * sizeof(unsigned long long), s));
  const int sms = num_sms();
  ev_sym.start();
  {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + 7) / 8, (int64_t)sms * 64);
    k_analysis<<<(unsigned)blocks, threads, 0, s>>>(A, B, D, base.p, words.p, flops.p);
    SX_CUDA(cudaGetLastError());
    k_sum_i64<<<std::min<int64_t>((n + 255) / 256, sms * 8), 256, 0, s>>>(flops.p, n, ctr.p + 2 * kClasses + 2);
    k_classify<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, words.p, nullptr, 0, lists.p, n, ctr.p, ctr.p + 2 * kClasses);
    k_zero_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(words.p, n, stats ? stats->sq.p : nullptr,
                                                         stats ? stats->diag.p : nullptr, cnt.p);
    SX_CUDA(cudaGetLastError());
    count_launches(4);
  }
  unsigned long long h[2 * kClasses + 4];
  SX_CUDA(cudaMemcpyAsync(h, ctr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  const int64_t products = (int64_t)h[2 * kClasses + 2];
  // symbolic pass per class
  {
    DevBuf<uint32_t> gs;
    for (int c = 0; c < kClasses; ++c) {
      const int64_t nr = (int64_t)h[c];
      if (!nr) continue;
      const int threads = kClassThreads[c];
      if (c < kClasses - 1) {
        const int64_t grid = std::min<int64_t>(nr, (int64_t)sms * 32);
        k_symbolic<false><<<(unsigned)grid, threads, kClassBytes[c], s>>>(A, B, D, lists.p + c * n, nr, base.p,
                                                                        words.p, cnt.p, nullptr, 0);
      } else {
        const int64_t stride = ((int64_t)h[2 * kClasses] / 4 + 63) & ~63ll;
        const int64_t grid = std::min<int64_t>(nr, (int64_t)sms * 2);
        gs.reset((size_t)(stride * grid), s);
        k_symbolic<true><<<(unsigned)grid, threads, 0, s>>>(A, B, D, lists.p + c * n, nr, base.p, words.p, cnt.p,
                                                          gs.p, stride);
      }
      SX_CUDA(cudaGetLastError());
      count_launches(1);
    }
  }
  // row pointers of C
  SX_CUDA(cudaMemsetAsync(ctr.p, 0, ctr.count * sizeof(unsigned long long), s));
  const int64_t total = scan_counts(cnt.p, n, C.rp.p, s, hs);
  if (total > (int64_t)INT32_MAX * 64) fail(SEXPM_EOVERFLOW, "product too large");
  C.nnz = total;
  C.ci.reset(total, s);
  C.v.reset(total, s);
  k_classify<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, words.p, C.rp.p, 1, lists.p, n, ctr.p, ctr.p + 2 * kClasses);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(h, ctr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  if (times) times->ms_symbolic += ev_sym.stop();
  ev_num.start();
  {
    DevBuf<unsigned char> gs;
    for (int c = 0; c < kClasses; ++c) {
      const int64_t nr = (int64_t)h[c];
      if (!nr) continue;
      const int threads = kClassThreads[c];
      if (c < kClasses - 1) {
        const int64_t grid = std::min<int64_t>(nr, (int64_t)sms * 32);
        k_numeric<false><<<(unsigned)grid, threads, kClassBytes[c], s>>>(
            A, B, D, div, beta, lists.p + c * n, nr, base.p, words.p, C.rp.p, C.ci.p, C.v.p,
            stats ? stats->sq.p : nullptr, stats ? stats->diag.p : nullptr, nullptr, 0);
      } else {
        const int64_t stride = ((int64_t)h[2 * kClasses] + 255) & ~255ll;
        const int64_t grid = std::min<int64_t>(nr, (int64_t)sms * 2);
        gs.reset((size_t)(stride * grid), s);
        k_numeric<true><<<(unsigned)grid, threads, 0, s>>>(A, B, D, div, beta, lists.p + c * n, nr, base.p, words.p,
                                                         C.rp.p, C.ci.p, C.v.p, stats ? stats->sq.p : nullptr,
                                                         stats ? stats->diag.p : nullptr, gs.p, stride);
      }
      SX_CUDA(cudaGetLastError());
      count_launches(1);
    }
  }
  if (times) times->ms_numeric += ev_num.stop();
  return products;
}

}  // namespace sexpm
