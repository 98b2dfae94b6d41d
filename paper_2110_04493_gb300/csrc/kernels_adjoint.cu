// Kernels of the reverse pass of Algorithm 4.2 (masks frozen):
//  * k_sddmm: out[p] = acc * out[p] + alpha * sum_l A_il B_jl + beta * A_ij for every stored
//    (i, j) of a pattern P, i.e. P o (alpha A B^T + beta A).  With A = Y and B = T this is
//    mask(Y T^T) (and 2Y), with A = T^T, B = Y^T it is mask(T^T Y): the two products of the
//    squaring adjoint  dL/dT_{k-1} = mask(2Y + Y T^T + T^T Y).
//    One block per row i: row A_i is held as a bitmap over its column span plus per-word
//    prefix counts (rank = position in the row), warps take the entries (i, j) of P_i and
//    stream row B_j, looking each column up in the bitmap; a warp reduction gives the dot
//    product.  No atomics; one FMA per matching pair.
//  * k_sort_rows_block / k_sort_long: per-row sorts used by the transpose: a bitonic sort in
//    shared memory for rows of up to 4096 entries; longer rows sort their 4096-entry chunks the
//    same way and merge the sorted runs pairwise (merge-path co-ranks) through a scratch array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kSddmmMaxWords = 12288;  // 96 KB of bitmap + prefix per block
constexpr int kSortMax = 4096;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Row span of A in 32-column words: base[i] (multiple of 32) and words[i]; maxw gets the largest.
__global__ void k_row_words(CsrD A, int32_t* base, int32_t* words, unsigned* maxw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
  if (a1 == a0) {
    base[i] = 0;
    words[i] = 0;
    return;
  }
  const int b = A.ci[a0] & ~31;
  const int w = ((A.ci[a1 - 1] - b) >> 5) + 1;
  base[i] = b;
  words[i] = w;
  atomicMax(maxw, (unsigned)w);
}

// BITMAP = true: A_i held as bitmap + prefix in shared memory (rows with words <= the launch's
// capacity); false: binary search in A_i (any row).
template <bool BITMAP>
__global__ void k_sddmm(CsrD P, CsrD A, CsrD B, double alpha, double beta, int accumulate, const int32_t* base,
                        const int32_t* words, int cap_words, double* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned red[32];
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem);
  unsigned* pre = bm + cap_words;
  const int nwarps = blockDim.x >> 5;
  for (int64_t i = blockIdx.x; i < P.n; i += gridDim.x) {
    const int64_t p0 = P.rp[i], p1 = P.rp[i + 1];
    if (p1 == p0) continue;
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    const int W = words[i];
    const int b = base[i];
    if (BITMAP && W > cap_words) continue;      // handled by the binary-search launch
    if (!BITMAP && W <= cap_words && cap_words > 0) continue;
    if (BITMAP) {
      for (int w = threadIdx.x; w < W; w += blockDim.x) bm[w] = 0u;
      __syncthreads();
      for (int64_t q = a0 + threadIdx.x; q < a1; q += blockDim.x) {
        const int c = A.ci[q] - b;
        atomicOr(&bm[c >> 5], 1u << (c & 31));
      }
      __syncthreads();
      // exclusive prefix of popcounts (per-thread chunks, then a block scan)
      const int T = blockDim.x;
      const int ch = (W + T - 1) / T;
      const int w0 = min(W, (int)threadIdx.x * ch), w1 = min(W, w0 + ch);
      unsigned s = 0;
      for (int w = w0; w < w1; ++w) s += __popc(bm[w]);
      unsigned incl = s;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(FULL, incl, o);
        if (lane_id() >= o) incl += y;
      }
      if (lane_id() == 31) red[warp_id()] = incl;
      __syncthreads();
      if (warp_id() == 0) {
        const unsigned v = lane_id() < nwarps ? red[lane_id()] : 0u;
        unsigned vi = v;
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(FULL, vi, o);
          if (lane_id() >= o) vi += y;
        }
        if (lane_id() < nwarps) red[lane_id()] = vi - v;
      }
      __syncthreads();
      unsigned run = red[warp_id()] + incl - s;
      for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bm[w]);
      }
      __syncthreads();
    }
    for (int64_t p = p0 + warp_id(); p < p1; p += nwarps) {
      const int j = P.ci[p];
      double acc = 0.0;
      if (alpha != 0.0 && a1 > a0) {
        const int64_t q0 = B.rp[j], q1 = B.rp[j + 1];
        for (int64_t q = q0 + lane_id(); q < q1; q += 32) {
          const int c = B.ci[q];
          int64_t pos = -1;
          if (BITMAP) {
            const int r = c - b;
            if (r >= 0 && r < 32 * W) {
              const uint32_t m = bm[r >> 5];
              if (m & (1u << (r & 31))) pos = a0 + pre[r >> 5] + __popc(m & ((1u << (r & 31)) - 1u));
            }
          } else {
            int64_t lo = a0, hi = a1;
            while (lo < hi) {
              const int64_t mid = (lo + hi) >> 1;
              if (A.ci[mid] < c) lo = mid + 1; else hi = mid;
            }
            if (lo < a1 && A.ci[lo] == c) pos = lo;
          }
          if (pos >= 0) acc = fma(A.v[pos], B.v[q], acc);
        }
        acc = warp_sum(acc);
      }
      if (lane_id() == 0) {
        double own = 0.0;
        if (beta != 0.0 && a1 > a0) {
          int64_t lo = a0, hi = a1;
          while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (A.ci[mid] < j) lo = mid + 1; else hi = mid;
          }
          if (lo < a1 && A.ci[lo] == j) own = A.v[lo];
        }
        const double v = alpha * acc + beta * own;
        out[p] = accumulate ? out[p] + v : v;
      }
    }
    __syncthreads();
  }
}

// Bitonic sort of entries [p0, p0 + len) (len <= kSortMax) by column, in shared memory, by the
// whole block.
__device__ void sort_chunk(int32_t* ci, double* v, int64_t p0, int len, int* sk, double* sv) {
  int size = 1;
  while (size < len) size <<= 1;
  for (int k = threadIdx.x; k < size; k += blockDim.x) {
    sk[k] = k < len ? ci[p0 + k] : INT_MAX;
    sv[k] = k < len ? v[p0 + k] : 0.0;
  }
  __syncthreads();
  for (int kk = 2; kk <= size; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < size; t += blockDim.x) {
        const int partner = t ^ jj;
        if (partner > t) {
          const bool up = (t & kk) == 0;
          const int a = sk[t], bq = sk[partner];
          if ((a > bq) == up) {
            sk[t] = bq;
            sk[partner] = a;
            const double x = sv[t];
            sv[t] = sv[partner];
            sv[partner] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int k = threadIdx.x; k < len; k += blockDim.x) {
    ci[p0 + k] = sk[k];
    v[p0 + k] = sv[k];
  }
  __syncthreads();
}

// Rows of at most kSortMax entries, one block per row (longer rows are left to k_sort_long).
__global__ void k_sort_rows_block(int64_t n, const int64_t* rp, int32_t* ci, double* v) {
  __shared__ int sk[kSortMax];
  __shared__ double sv[kSortMax];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int64_t p0 = rp[i], p1 = rp[i + 1];
    const int len = (int)(p1 - p0);
    if (len <= 1 || len > kSortMax) continue;
    sort_chunk(ci, v, p0, len, sk, sv);
  }
}

// Rows longer than kSortMax, one block per row (rows[b], scratch slice at off[b] of the row's
// length): chunks of kSortMax sorted in shared memory, then passes that merge pairs of sorted
// runs of width w into runs of 2w, alternating between the row and the scratch.  Output
// position k of a merge takes its element from the co-rank i(k) (the number of elements of the
// left run among the first k outputs, found by binary search); columns within a row are unique.
__global__ void k_sort_long(const int64_t* rows, const int64_t* rp, int32_t* ci, double* v, const int64_t* off,
                            int32_t* sci, double* sv_g) {
  __shared__ int sk[kSortMax];
  __shared__ double sv[kSortMax];
  const int64_t i = rows[blockIdx.x];
  const int64_t p0 = rp[i];
  const int64_t len = rp[i + 1] - p0;
  for (int64_t c0 = 0; c0 < len; c0 += kSortMax)
    sort_chunk(ci, v, p0 + c0, (int)(len - c0 < kSortMax ? len - c0 : kSortMax), sk, sv);
  int32_t* srcc = ci + p0;
  double* srcv = v + p0;
  int32_t* dstc = sci + off[blockIdx.x];
  double* dstv = sv_g + off[blockIdx.x];
  for (int64_t w = kSortMax; w < len; w <<= 1) {
    for (int64_t a0 = 0; a0 < len; a0 += 2 * w) {
      const int64_t na = w < len - a0 ? w : len - a0;
      const int64_t rest = len - a0 - w > 0 ? len - a0 - w : 0;
      const int64_t nb = w < rest ? w : rest;
      const int32_t* A = srcc + a0;
      const int32_t* B = A + na;
      for (int64_t k = threadIdx.x; k < na + nb; k += blockDim.x) {
        int64_t lo = k - nb > 0 ? k - nb : 0, hi = k < na ? k : na;
        while (lo < hi) {  // smallest i with A[i] > B[k - i - 1]
          const int64_t mid = (lo + hi) >> 1;
          if (A[mid] <= B[k - mid - 1]) lo = mid + 1; else hi = mid;
        }
        const int64_t ia = lo, ib = k - lo;
        const bool take_a = ia < na && (ib >= nb || A[ia] <= B[ib]);
        const int64_t src = take_a ? a0 + ia : a0 + na + ib;
        dstc[a0 + k] = srcc[src];
        dstv[a0 + k] = srcv[src];
      }
    }
    __syncthreads();
    int32_t* tc = srcc; srcc = dstc; dstc = tc;
    double* tv = srcv; srcv = dstv; dstv = tv;
  }
  if (srcc != ci + p0) {
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
      ci[p0 + k] = srcc[k];
      v[p0 + k] = srcv[k];
    }
  }
}

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    SX_CUDA(cudaGetDevice(&dev));
    SX_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

}  // namespace

// Rows longer than kSortMax: their ids and lengths (n_long entries; synchronises s).
__global__ void k_count_long(int64_t n, const int64_t* rp, unsigned long long* cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && rp[i + 1] - rp[i] > kSortMax) atomicAdd(cnt, 1ull);
}

void sort_rows(int64_t n, const int64_t* rp, int32_t* ci, double* v, cudaStream_t s) {
  if (n == 0) return;
  const int64_t grid = std::min<int64_t>(n, (int64_t)sms() * 16);
  k_sort_rows_block<<<(unsigned)grid, 256, 0, s>>>(n, rp, ci, v);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  // rows longer than kSortMax: found on the host from the row pointers when any exists
  DevBuf<unsigned long long> cnt(1, s);
  SX_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
  k_count_long<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, rp, cnt.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  unsigned long long h = 0;
  SX_CUDA(cudaMemcpyAsync(&h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  if (h == 0) return;
  std::vector<int64_t> rph(n + 1);
  SX_CUDA(cudaMemcpyAsync(rph.data(), rp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> rows, off;
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t len = rph[i + 1] - rph[i];
    if (len > kSortMax) {
      rows.push_back(i);
      off.push_back(total);
      total += len;
    }
  }
  DevBuf<int64_t> drows(rows.size(), s), doff(off.size(), s);
  DevBuf<int32_t> sci(total, s);
  DevBuf<double> sv(total, s);
  SX_CUDA(cudaMemcpyAsync(drows.p, rows.data(), rows.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  SX_CUDA(cudaMemcpyAsync(doff.p, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_sort_long<<<(unsigned)rows.size(), 256, 0, s>>>(drows.p, rp, ci, v, doff.p, sci.p, sv.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaStreamSynchronize(s));
}

void sddmm(const CsrD& P, const CsrD& A, const CsrD& B, double alpha, double beta, bool accumulate, double* out,
           cudaStream_t s, HostScalars& hs) {
  const int64_t n = P.n;
  if (n == 0 || P.nnz == 0) return;
  static bool attr[64] = {};
  once_per_device(attr, [] {
    SX_CUDA(cudaFuncSetAttribute(k_sddmm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kSddmmMaxWords));
  });
  DevBuf<int32_t> base(n, s), words(n, s);
  DevBuf<unsigned> maxw(1, s);
  SX_CUDA(cudaMemsetAsync(maxw.p, 0, sizeof(unsigned), s));
  k_row_words<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, base.p, words.p, maxw.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(hs.i, maxw.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  unsigned mw = 0;
  std::memcpy(&mw, hs.i, sizeof(unsigned));
  const int cap = (int)std::min<unsigned>(mw, (unsigned)kSddmmMaxWords);
  const int64_t grid = std::min<int64_t>(n, (int64_t)sms() * 8);
  k_sddmm<true><<<(unsigned)grid, 256, (size_t)8 * std::max(cap, 1), s>>>(P, A, B, alpha, beta, accumulate ? 1 : 0,
                                                                        base.p, words.p, cap, out);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  if ((int)mw > cap) {
    k_sddmm<false><<<(unsigned)grid, 256, 0, s>>>(P, A, B, alpha, beta, accumulate ? 1 : 0, base.p, words.p, cap, out);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
  }
}

}  // namespace sexpm
