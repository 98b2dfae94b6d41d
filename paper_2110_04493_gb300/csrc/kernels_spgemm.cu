// Sparse product of Algorithm 4.2 with its fused scaling and sum:
//     C = (A B) / div + beta D
// used for the Taylor terms S~_i = S^_{i-1} H_0 / i (Eq. 4.10) and the squaring
// steps T~_i = 2 T^_{i-1} + T^_{i-1}^2 (Eq. 4.15).
//
// Row-wise (Gustavson) product, one thread block per output row; each size class
// of rows is one persistent launch of the resident blocks, which take rows from an
// atomic counter in schedule order.
//
// Pattern.  The output pattern of row i is a bitmap over the row's column span
// [base_i, hi_i] (base_i a multiple of 32).  B and D are first compressed to
// "word patterns": for every row, the distinct 32-column words it touches and
// the bit mask inside each word.  The row bitmap is then the OR of the word
// patterns of the rows B_k, k in A_i (plus D_i), which costs one shared-memory
// atomicOr per (k, word) instead of one per scalar product.  The symbolic pass
// counts the bits; the numeric pass rebuilds the bitmap the same cheap way.
//
// Values.  Each bitmap word is kept with its position prefix, and
// rank(c) = prefix[c/32] + popc(mask[c/32] & below(c)) maps a column to its
// position in the sorted output row, so an accumulator is a dense array of
// exactly nnz(row) doubles already in column order.  The block's warps form
// groups that split the row's columns (equal shares of its products); the
// members of a group split the k's of A_i and accumulate the part of B_k inside
// the group's columns into accumulators of their own, summed in member order.
// Every product is one FP64 FMA on a shared-memory accumulator (no atomics).
//
// Rows are binned by the shared memory they need (accumulators, bitmap words and
// prefixes); the widest rows use a per-block global-memory scratch slice.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <cstdlib>
#include <string>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kClasses = kProductClasses;
// Shared-memory budget and block size of each row class; the last class uses global scratch.
// The symbolic pass uses blocks of at most 256 threads.  The numeric kernel is compiled for
// 32 resident warps per SM (its register budget: SEXPM_NUMERIC_BLOCKS blocks of 256 threads).
// Rows of the global-scratch class (accumulators in L2) run on blocks of 1024 threads, one per
// SM, which keeps those 32 warps there (measured on the 3-D 64^3 grid: its last squaring 118 s ->
// 82 s); the 112 KB and 220 KB classes measured 5-18% slower on 512 or 1024 threads than on 256
// (more column groups, each searching every B row) and stay at 256.  SEXPM_WIDE_BLOCKS=0 in the
// environment keeps 256 threads for the global class too.
constexpr int kClassBytes[kClasses] = {8 << 10, 24 << 10, 56 << 10, 112 << 10, 220 << 10, INT_MAX};
constexpr int kClassThreads[kClasses] = {64, 128, 256, 256, 256, 256};      // symbolic pass
constexpr int kNumThreadsWide[kClasses] = {64, 128, 256, 256, 256, 1024};  // numeric pass

__host__ __device__ constexpr int class_limit(int c) {
  return c == 0 ? (8 << 10) : c == 1 ? (24 << 10) : c == 2 ? (56 << 10) : c == 3 ? (112 << 10)
       : c == 4 ? (220 << 10) : INT_MAX;
}

// Warps of the numeric pass's blocks in class c.
__host__ __device__ constexpr int class_warps(int c, bool wide) {
  return wide ? (c == 0 ? 2 : c == 1 ? 4 : c <= 4 ? 8 : 32) : (c == 0 ? 2 : c == 1 ? 4 : 8);
}
static_assert(class_warps(0, true) * 32 == kNumThreadsWide[0] && class_warps(3, true) * 32 == kNumThreadsWide[3] &&
                  class_warps(4, true) * 32 == kNumThreadsWide[4] && class_warps(5, true) * 32 == kNumThreadsWide[5] &&
                  class_warps(2, false) * 32 == kClassThreads[2] && class_warps(5, false) * 32 == kClassThreads[5],
              "class_warps must match the block sizes");

// Shared bytes of the numeric pass for a row with W bitmap words, cnt outputs of which cacc
// are accumulated (the upper part in the symmetric mode), and q accumulators: the
// accumulators (8 cacc bytes each; the region first holds the per-word product counts,
// 4 W bytes) and the bitmap words with their position prefixes (8 W bytes).
__host__ __device__ __forceinline__ long long acc_bytes(long long W, long long cacc, int q) {
  const long long a = 8 * cacc * q, w = 4 * W;
  return ((a > w ? a : w) + 15) & ~15ll;
}
__host__ __device__ __forceinline__ long long need_bytes(long long W, long long cnt, long long cacc, int q) {
  return acc_bytes(W, cacc, q) + 8 * W;
}

// Resident 256-thread blocks per SM the numeric kernel is compiled for (its register budget).
#ifndef SEXPM_NUMERIC_BLOCKS
#define SEXPM_NUMERIC_BLOCKS 4
#endif
constexpr int kNumericWarpsPerSM = 8 * SEXPM_NUMERIC_BLOCKS;

// Accumulation layout of a row: the block's warps form groups of `members` warps.  The
// groups split the row's columns (equal shares of its products); the members of a group
// split the k's of A_i (member q takes every members-th k) and accumulate into accumulator q
// of their own; the members' accumulators are summed in member order.  members = 1 is a pure
// column split (every warp searches each B_k for its columns); members = nwarps is a pure
// k split (whole rows B_k, no search).  More members means fewer, longer segments and fewer
// searches, at 8 bytes per accumulated entry and member.  The numeric kernel holds
// kNumericWarpsPerSM warps per SM (its register budget), so a block of nwarps warps may use
// that fraction of the SM's shared memory without lowering the occupancy: members is the
// largest power of two whose row fits in that share of sm_bytes (sm_bytes = 0: column split).
constexpr int kKsplitBytesDefault = 220 << 10;
__host__ __device__ __forceinline__ int ks_members(long long W, long long cnt, long long cacc, int nwarps,
                                                   int sm_bytes) {
  const long long budget = (long long)sm_bytes * nwarps / kNumericWarpsPerSM;
  int q = nwarps;
  while (q > 1 && need_bytes(W, cnt, cacc, q) > budget) q >>= 1;
  return q;
}
__host__ __device__ __forceinline__ long long acc_region(long long W, long long cnt, long long cacc, int nwarps,
                                                         int sm_bytes) {
  return acc_bytes(W, cacc, ks_members(W, cnt, cacc, nwarps, sm_bytes));
}
__host__ __device__ __forceinline__ long long numeric_need(long long W, long long cnt, long long cacc, int nwarps,
                                                           int sm_bytes) {
  return need_bytes(W, cnt, cacc, ks_members(W, cnt, cacc, nwarps, sm_bytes));
}

// (WPat, the word pattern of a CSR matrix, is declared in sexpm_internal.cuh.)

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

// Row bitmap with position prefixes: word w of the row is bp[w] = {mask, prefix}, the mask of
// the row's columns b + 32 w .. b + 32 w + 31 and the number of the row's columns before it.
// Column (relative to the row base) of output position k: the largest word w with
// prefix <= k, then the (k - prefix)-th set bit of that word.
__device__ __forceinline__ int column_at(const uint2* bp, int W, int k) {
  int lo = 0, hi = W - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)bp[mid].y <= k) lo = mid; else hi = mid - 1;
  }
  const uint2 e = bp[lo];
  return lo * 32 + select_bit(e.x, k - (int)e.y);
}

// Output position of column c (relative to the row base): the prefix of its word plus the
// set bits below it ((mask << (31 - r)) << 1 keeps bits 0 .. r-1 of the mask, r = c mod 32).
__device__ __forceinline__ unsigned rank_of(const uint2* bp, int c) {
  const uint2 e = bp[c >> 5];
  return e.y + __popc((e.x << (~c & 31)) << 1);
}

__device__ __forceinline__ int64_t lower_bound_col(const int32_t* ci, int64_t lo, int64_t hi, int c) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- word patterns
// Number of distinct words per row (one warp per row; rows are sorted).
__global__ void k_wcount(CsrD X, int32_t* cnt) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < X.n; i += nw) {
    const int64_t p0 = X.rp[i], p1 = X.rp[i + 1];
    int c = 0;
    int prev = -1;
    for (int64_t q0 = p0; q0 < p1; q0 += 32) {
      const int64_t q = q0 + lane_id();
      const bool act = q < p1;
      const int w = act ? (X.ci[q] >> 5) : -2;
      int pw = __shfl_up_sync(FULL, w, 1);
      if (lane_id() == 0) pw = prev;
      c += __popc(__ballot_sync(FULL, act && w != pw));
      prev = __shfl_sync(FULL, w, (int)(p1 - q0 - 1 < 31 ? p1 - q0 - 1 : 31));
    }
    if (lane_id() == 0) cnt[i] = c;
  }
}

// Writes the word pattern: distinct words and the OR of their column bits.
// A non-null status that is set (the pattern exceeds its capacity) stops the kernel.
__global__ void k_wwrite(CsrD X, const int64_t* wrp, int32_t* wi, uint32_t* wb, const int32_t* status) {
  if (status && *status) return;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane_id()) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < X.n; i += nw) {
    const int64_t p0 = X.rp[i], p1 = X.rp[i + 1];
    int64_t o = wrp[i];
    int prev = -1;
    for (int64_t q0 = p0; q0 < p1; q0 += 32) {
      __syncwarp();
      const int64_t q = q0 + lane_id();
      const bool act = q < p1;
      const int col = act ? X.ci[q] : 0;
      const int w = act ? (col >> 5) : -2;
      uint32_t bits = act ? (1u << (col & 31)) : 0u;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t ob = __shfl_down_sync(FULL, bits, off);
        const int ow = __shfl_down_sync(FULL, w, off);
        if (lane_id() + off < 32 && ow == w) bits |= ob;
      }
      int pw = __shfl_up_sync(FULL, w, 1);
      if (lane_id() == 0) pw = prev;
      const bool head = act && w != pw;
      const unsigned hm = __ballot_sync(FULL, head);
      if (head) {
        const int64_t d = o + __popc(hm & lt);
        wi[d] = w;
        wb[d] = bits;
      }
      if (lane_id() == 0 && act && w == prev) wb[o - 1] |= bits;  // word continued from the previous chunk
      o += __popc(hm);
      prev = __shfl_sync(FULL, w, (int)(p1 - q0 - 1 < 31 ? p1 - q0 - 1 : 31));
    }
  }
}

// ---------------------------------------------------------------- row analysis and binning
// Per row: column span of the product row (A B plus the pattern of D) and its product count.
// One warp per row.
__global__ void k_analysis(CsrD A, CsrD B, CsrD D, const uint8_t* frozen, int32_t* base, int32_t* words,
                           int64_t* flops) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    int lo = INT_MAX, hi = -1;
    int64_t f = 0;
    const bool fz = frozen && frozen[i];
    const int64_t a0 = A.rp[i], a1 = fz ? a0 : A.rp[i + 1];
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

// Assign each row to a class by its shared-memory need (bytes); append row ids per class and
// record the largest need of each class (maxneed[class]).
// mode 0: symbolic need 4 W; mode 1: numeric need 12 W + 8 cnt.
__global__ void k_classify(int64_t n, const int32_t* sched, const int32_t* words, const int64_t* rp_out,
                           const int32_t* cnt_up, int mode, int ks_bytes, int32_t* lists, int64_t list_stride,
                           unsigned long long* counts, unsigned long long* maxneed, int64_t r0, int64_t r1,
                           bool wide) {
  __shared__ unsigned int cnt[kClasses];
  __shared__ unsigned long long off[kClasses];
  if (threadIdx.x < kClasses) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = (t < n && sched) ? (int64_t)sched[t] : t;  // rows enter the lists in schedule order
  int cls = -1;
  unsigned int slot = 0;
  long long need = 0;
  if (t < n && i >= r0 && i < r1) {  // only the rows of [r0, r1) enter the lists
    const long long W = words[i];
    const long long full = mode == 0 ? 0 : rp_out[i + 1] - rp_out[i];
    const long long cacc = cnt_up ? (long long)cnt_up[i] : full;
    if (W > 0) {
      cls = 0;
      for (;;) {
        need = mode == 0 ? 4 * W : numeric_need(W, full, cacc, class_warps(cls, wide), ks_bytes);
        if (cls == kClasses - 1 || need <= class_limit(cls)) break;
        ++cls;
      }
      slot = atomicAdd(&cnt[cls], 1u);
      atomicMax(&maxneed[cls], (unsigned long long)need);
    }
  }
  __syncthreads();
  if (threadIdx.x < kClasses)
    off[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], (unsigned long long)cnt[threadIdx.x]) : 0ull;
  __syncthreads();
  if (cls >= 0) lists[cls * list_stride + off[cls] + slot] = (int32_t)i;
}

// OR the word patterns of the rows B_k (k in A_i) and of D_i into the row bitmap bm
// (word wlo of the row is bm[0]; word w at bm[w * STRIDE]).  When work != nullptr, work[w] also
// receives the number of scalar products that land in word w (the popcount of every B_k mask
// ORed into it); with upper set, only products at columns >= i are counted.
// Each warp takes batches of 32 k's (one per lane: the k's a0 + 32 (w + nwarps m) + lane) and
// streams the concatenation of their word patterns 32 entries at a time; lane l finds the k of
// its entry by a binary search over the lanes' exclusive prefix of pattern lengths.  All
// loads of a batch are independent (an OR does not depend on its order).  Batches whose
// patterns average kLongPattern entries or more are streamed one k at a time instead (the
// search would cost more than the latency it hides).
// Block-wide; the caller synchronises afterwards.
constexpr int kLongPattern = 48;

template <int STRIDE>
__device__ __forceinline__ void build_row_bitmap(const CsrD& A, const WPat& WB, const WPat& WD, bool hasD, int64_t i,
                                                 int wlo, uint32_t* bm, unsigned* work, bool upper, bool fz) {
  const int nwarps = blockDim.x >> 5, lane = lane_id();
  const int64_t a0 = A.rp[i], a1 = fz ? a0 : A.rp[i + 1];
  const int iw = (int)(i >> 5);
  const uint32_t imask = ~((1u << (i & 31)) - 1u);
  for (int64_t kb = a0 + 32 * warp_id(); kb < a1; kb += 32 * nwarps) {
    int64_t e0 = 0;
    int len = 0;
    if (kb + lane < a1) {
      const int k = A.ci[kb + lane];
      e0 = WB.rp[k];
      len = (int)(WB.rp[k + 1] - e0);
    }
    int excl = len;  // inclusive, then exclusive prefix of the lengths over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, excl, o);
      if (lane >= o) excl += y;
    }
    const int total = __shfl_sync(FULL, excl, 31);
    excl -= len;
    if (total >= 32 * kLongPattern) {
      // long patterns (rows of B spread over many words): one k at a time, 32 entries a round
      for (int j = 0; j < 32; ++j) {
        const int64_t ej = __shfl_sync(FULL, e0, j);
        const int lj = __shfl_sync(FULL, len, j);
        for (int f = lane; f < lj; f += 32) {
          const int wa = WB.wi[ej + f];
          const int w = wa - wlo;
          const uint32_t bits = WB.wb[ej + f];
          atomicOr(&bm[w * STRIDE], bits);
          if (work) {
            const uint32_t wbits = !upper || wa > iw ? bits : (wa == iw ? (bits & imask) : 0u);
            if (wbits) atomicAdd(&work[w], (unsigned)__popc(wbits));
          }
        }
      }
      continue;
    }
#pragma unroll 2
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      // the last lane j with excl_j <= f holds f (lanes with an empty pattern share the
      // prefix of the next lane, so the last such lane has a non-empty one)
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int ex = __shfl_sync(FULL, excl, j + step);
        if (ex <= f) j += step;
      }
      const int64_t ej = __shfl_sync(FULL, e0, j);
      const int xj = __shfl_sync(FULL, excl, j);
      if (f < total) {
        const int64_t e = ej + (f - xj);
        const int wa = WB.wi[e];
        const int w = wa - wlo;
        const uint32_t bits = WB.wb[e];
        atomicOr(&bm[w * STRIDE], bits);
        if (work) {
          const uint32_t wbits = !upper || wa > iw ? bits : (wa == iw ? (bits & imask) : 0u);
          if (wbits) atomicAdd(&work[w], (unsigned)__popc(wbits));
        }
      }
    }
  }
  if (hasD) {
    const int64_t e1 = WD.rp[i + 1];
    for (int64_t e = WD.rp[i] + threadIdx.x; e < e1; e += blockDim.x) atomicOr(&bm[(WD.wi[e] - wlo) * STRIDE], WD.wb[e]);
  }
}

// In-place exclusive scan of x[0..W) by the whole block; returns the total to every thread.
// Each thread scans a contiguous chunk; `red` is a 33-entry shared scratch.
__device__ unsigned block_exclusive_scan(unsigned* x, int W, unsigned* red) {
  const int T = blockDim.x, nwarps = T >> 5, lane = lane_id();
  const int ch = (W + T - 1) / T;
  const int w0 = min(W, (int)threadIdx.x * ch), w1 = min(W, w0 + ch);
  unsigned s = 0;
  for (int w = w0; w < w1; ++w) s += x[w];
  unsigned incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) red[warp_id()] = incl;
  __syncthreads();
  if (warp_id() == 0) {
    const unsigned v = lane < nwarps ? red[lane] : 0u;
    unsigned vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nwarps) red[lane] = vi - v;
    if (lane == 31) red[32] = vi;  // block total (red has 33 entries)
  }
  __syncthreads();
  unsigned run = red[warp_id()] + incl - s;
  for (int w = w0; w < w1; ++w) {
    const unsigned v = x[w];
    x[w] = run;
    run += v;
  }
  const unsigned total = red[32];
  __syncthreads();
  return total;
}

// Symbolic pass: cnt[i] = number of distinct columns of row i of A B (+ pattern of D).
// Dynamic row assignment for the persistent row kernels: block b first takes row b of its
// list, then the rows gridDim.x, gridDim.x + 1, ... in the order blocks ask for them, so the
// rows in flight stay a window of consecutive list entries (the list follows the row
// schedule, which keeps the rows of B they read resident in L2).  Thread 0 asks at the start
// of a row and publishes the answer after the row, so the atomic's latency is hidden; every
// row body has a block barrier between the read of s_next and its next write.
__device__ __forceinline__ long long next_row(unsigned long long* ctr) {
  return (long long)gridDim.x + (long long)atomicAdd(ctr, 1ull);
}

template <bool GLOBAL>
__global__ void k_symbolic(CsrD A, WPat WB, WPat WD, bool hasD, const uint8_t* frozen, const int32_t* rows,
                           int64_t nrows, const unsigned long long* nrows_dev, const int32_t* base,
                           const int32_t* words, int32_t* cnt, int32_t* cnt_up, uint32_t* gscratch, int64_t gstride,
                           unsigned long long* row_ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int red[32];
  __shared__ long long s_next;
  uint32_t* bm = GLOBAL ? gscratch + (int64_t)blockIdx.x * gstride : reinterpret_cast<uint32_t*>(smem);
  if (nrows_dev) nrows = min(nrows, (int64_t)*nrows_dev);  // list length decided on the device
  long long nxt = 0;
  for (int64_t r = blockIdx.x; r < nrows;) {
    if (threadIdx.x == 0) nxt = next_row(row_ctr);
    const int i = rows[r];
    const int W = words[i];
    const int wlo = base[i] >> 5;
    for (int w = threadIdx.x; w < W; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    build_row_bitmap<1>(A, WB, WD, hasD, i, wlo, bm, nullptr, false, frozen && frozen[i]);
    __syncthreads();
    int c = 0, cu = 0;
    const int iw = i >> 5;
    const uint32_t imask = ~((1u << (i & 31)) - 1u);
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      const uint32_t m = bm[w];
      c += __popc(m);
      if (cnt_up) {
        const int wa = wlo + w;
        cu += wa > iw ? __popc(m) : (wa == iw ? __popc(m & imask) : 0);
      }
    }
    c = block_sum(c, red);
    if (threadIdx.x == 0) cnt[i] = c;
    if (cnt_up) {
      cu = block_sum(cu, red);
      if (threadIdx.x == 0) cnt_up[i] = cu;
    }
    if (threadIdx.x == 0) s_next = nxt;
    __syncthreads();
    r = s_next;
  }
}

// Exclusive prefix of the popcounts of the masks bp[0..W).x into bp[0..W).y, by the whole block.
__device__ void block_popc_prefix(uint2* bp, int W, unsigned* red) {
  const int T = blockDim.x, nwarps = T >> 5, lane = lane_id();
  const int ch = (W + T - 1) / T;
  const int w0 = min(W, (int)threadIdx.x * ch), w1 = min(W, w0 + ch);
  unsigned s = 0;
  for (int w = w0; w < w1; ++w) s += __popc(bp[w].x);
  unsigned incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) red[warp_id()] = incl;
  __syncthreads();
  if (warp_id() == 0) {
    const unsigned v = lane < nwarps ? red[lane] : 0u;
    unsigned vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nwarps) red[lane] = vi - v;
  }
  __syncthreads();
  unsigned run = red[warp_id()] + incl - s;
  for (int w = w0; w < w1; ++w) {
    bp[w].y = run;
    run += __popc(bp[w].x);
  }
  __syncthreads();
}

// Rows of B up to this length are masked below the diagonal instead of searched (upper mode,
// whole rows).
constexpr int kMaskMax = 16;

// One quad of a segment: up to 128 consecutive entries of one row B_k, entry 32 t + lane of
// the quad in chunk t of this lane.  s is the quad's first entry, len the entries left in the
// segment from s, a the factor A_ik.
struct Quad {
  int64_t s;
  int len;
  double a;
  int c[4];
  double v[4];
};

// Loads the quad's four chunks.  Lanes past the segment's end read its last entry instead,
// so every load is in bounds and none is conditional; such a lane repeats the last entry's
// update (the same value, from the same accumulator load), which is harmless.
__device__ __forceinline__ void load_quad(const CsrD& B, int lane, Quad& q) {
  const int32_t* cb = B.ci + q.s;
  const double* vb = B.v + q.s;
  const int last = q.len - 1;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int e = min(lane + 32 * t, last);
    q.c[t] = __ldg(cb + e);
    q.v[t] = __ldg(vb + e);
  }
}

// Shared-memory accesses through 32-bit shared-window addresses (the accumulators and the
// bitmap words of the shared-memory classes).
__device__ __forceinline__ uint2 lds_u2(uint32_t a) {
  uint2 r;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(a));
  return r;
}
__device__ __forceinline__ double lds_f64(uint32_t a) {
  double r;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(r) : "r"(a));
  return r;
}
__device__ __forceinline__ void sts_f64(uint32_t a, double x) {
  asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(x) : "memory");
}

// Addresses of the accumulation: generic pointers (global-scratch rows) and, for rows held in
// shared memory, the same arrays as 32-bit shared-window addresses.
struct AccPtrs {
  double* acc;
  double* sink;
  const uint2* bp;
  uint32_t acc_s, sink_s, bp_s;
  int c_lo;  // with MASK, entries below this column go to the sink
};

// acc[rank(c_t)] += a v_t for the NC chunks of quad q; with MASK an entry with a column below
// P.c_lo (the upper mode's entries below the diagonal) is sent to the warp's sink slot instead
// (only rows whose k's are not split into column groups need it: short rows of B are masked
// rather than searched).
// The columns of a quad are distinct (one row of B; repeated last entries aside), so every rank
// and accumulator load is issued before the first store and the chunks' DFMAs overlap.  The
// code is branch-free; every chunk has a lane inside the segment, so no DFMA is issued for a
// chunk without work.  SH: the accumulators and bitmap are in shared memory (32-bit addresses).
template <int NC, bool MASK, bool SH>
__device__ __forceinline__ void accumulate_chunks(const AccPtrs& P, int b, const Quad& q) {
  double x[NC];
  if (SH) {
    uint32_t ad[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      const int c = q.c[t];
      const unsigned rel = (unsigned)(c - b);
      const uint2 e = lds_u2(P.bp_s + (rel >> 5) * 8u);
      const uint32_t at = P.acc_s + (e.y + __popc((e.x << (~rel & 31u)) << 1)) * 8u;
      ad[t] = (!MASK || c >= P.c_lo) ? at : P.sink_s;
    }
#pragma unroll
    for (int t = 0; t < NC; ++t) x[t] = lds_f64(ad[t]);
#pragma unroll
    for (int t = 0; t < NC; ++t) x[t] = fma(q.a, q.v[t], x[t]);
#pragma unroll
    for (int t = 0; t < NC; ++t) sts_f64(ad[t], x[t]);
  } else {
    double* ad[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      const int c = q.c[t];
      double* const at = P.acc + rank_of(P.bp, c - b);
      ad[t] = (!MASK || c >= P.c_lo) ? at : P.sink;
    }
#pragma unroll
    for (int t = 0; t < NC; ++t) x[t] = *ad[t];
#pragma unroll
    for (int t = 0; t < NC; ++t) x[t] = fma(q.a, q.v[t], x[t]);
#pragma unroll
    for (int t = 0; t < NC; ++t) *ad[t] = x[t];
  }
}

template <bool MASK, bool SH>
__device__ __forceinline__ void accumulate_quad_m(const AccPtrs& P, int b, const Quad& q) {
  if (q.len > 96) accumulate_chunks<4, MASK, SH>(P, b, q);
  else if (q.len > 64) accumulate_chunks<3, MASK, SH>(P, b, q);
  else if (q.len > 32) accumulate_chunks<2, MASK, SH>(P, b, q);
  else accumulate_chunks<1, MASK, SH>(P, b, q);
}

// One stage of the accumulation pipeline: fix the quad after `cur` (the next 128 entries of
// its segment, else the first quad of the next non-empty segment of the batch, from the
// lanes' s, len, a and the mask `live` of segments not yet started), start its loads, then
// accumulate `cur`.  Returns false when `cur` was the batch's last quad.  Between two
// segments the warp synchronises: rows B_k and B_k' may share columns.
template <bool MASK, bool SH>
__device__ __forceinline__ bool pipe_stage(const CsrD& B, const AccPtrs& P, int b, int lane, int64_t s, int len,
                                           double a, unsigned& live, const Quad& cur, Quad& nxt) {
  bool more = true, fresh = false;
  if (cur.len > 128) {
    nxt.s = cur.s + 128;
    nxt.len = cur.len - 128;
    nxt.a = cur.a;
  } else if (live) {
    const int j = __ffs(live) - 1;
    live &= live - 1u;
    nxt.s = __shfl_sync(FULL, s, j);
    nxt.len = __shfl_sync(FULL, len, j);
    nxt.a = __shfl_sync(FULL, a, j);
    fresh = true;
  } else {
    more = false;
  }
  if (more) load_quad(B, lane, nxt);
  accumulate_quad_m<MASK, SH>(P, b, cur);
  if (fresh) __syncwarp();
  return more;
}

// Numeric pass, one row: prefixes, accumulation, fused scaling and beta D, and the ordered
// write.  The accumulator region first holds wk (products per word); bp holds the row's
// bitmap words with their position prefixes.
template <bool SH>
__device__ void numeric_row(const CsrD& A, const CsrD& B, const CsrD& D, double div, double beta, bool upper, bool fz,
                            int i, int W, int b, int64_t o0, int cnt, int lo_pos, double* acc, unsigned* wk,
                            uint2* bp, double* sink, int32_t* ci_out, double* v_out, double* row_sq,
                            double* row_diag, unsigned* ured, double* dred, unsigned long long* work_total,
                            int ks_bytes) {
  const int nwarps = blockDim.x >> 5;
  const int T = blockDim.x;
  const int lane = lane_id();
  const bool hasD = D.n > 0;
  // 2. exclusive prefixes: output positions (bp[].y) and products (wk) per word
  block_popc_prefix(bp, W, ured);
  const unsigned work = block_exclusive_scan(wk, W, ured);
  if (threadIdx.x == 0) atomicAdd(work_total, (unsigned long long)work);
  // 3. accumulation.  Warp w is member q = w % members of group g = w / members; group g owns
  //    the words [wa, wb) that hold the g-th equal share of the row's products, i.e. the
  //    columns [b + 32 wa, b + 32 wb); member q visits the k's a0 + q, a0 + q + members, ...,
  //    takes the part of B_k inside the group's columns (the whole row when there is one
  //    group) and accumulates it into accumulator q (acc + q cacc), one quad of 128 entries
  //    at a time, loading the next quad while the current one is accumulated.
  {
    const int cacc = cnt - lo_pos;
    const int members = ks_members(W, cnt, cacc, nwarps, ks_bytes);
    const int groups = nwarps / members;
    const int g = warp_id() / members, q = warp_id() % members;
    int wa = 0, wb = W;
    if (groups > 1) {
      const unsigned t0 = (unsigned)(((unsigned long long)g * work) / groups);
      const unsigned t1 = (unsigned)(((unsigned long long)(g + 1) * work) / groups);
      // first word whose prefix is >= target (words before it end before the target)
      int lo = 0, hi = W;
      while (lo < hi) { const int mid = (lo + hi) >> 1; if (wk[mid] < t0) lo = mid + 1; else hi = mid; }
      wa = lo;
      lo = wa; hi = W;
      while (lo < hi) { const int mid = (lo + hi) >> 1; if (wk[mid] < t1) lo = mid + 1; else hi = mid; }
      wb = (g == groups - 1) ? W : lo;
    }
    __syncthreads();  // every warp has read wk: the region now becomes the accumulators
    const int zend = lo_pos + members * cacc;
    for (int k = lo_pos + threadIdx.x; k < zend; k += T) acc[k] = 0.0;
    __syncthreads();
    if (wa < wb && !fz) {
      const int c_lo = upper ? max(b + 32 * wa, i) : b + 32 * wa;
      const int c_hi = b + 32 * wb - 1;
      double* const accw = acc + q * cacc;
      // short rows of B are masked entry by entry (upper mode, one column group)
      const bool mask_row = upper && groups == 1;
      AccPtrs P;
      P.c_lo = c_lo;
      P.acc = accw;
      P.sink = sink;
      P.bp = bp;
      if (SH) {
        // 32-bit shared addresses; acc is indexed by full-row position and may start before the
        // region (modular arithmetic brings every accessed position back inside)
        P.acc_s = (uint32_t)__cvta_generic_to_shared(acc + lo_pos) - 8u * (uint32_t)lo_pos + 8u * (uint32_t)(q * cacc);
        P.sink_s = (uint32_t)__cvta_generic_to_shared(sink);
        P.bp_s = (uint32_t)__cvta_generic_to_shared(bp);
      }
      const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
      for (int64_t kb = a0 + q; kb < a1; kb += 32 * members) {
        const int64_t p = kb + lane * members;
        int64_t s = 0;
        int len = 0;
        double a = 0.0;
        if (p < a1) {
          const int k = A.ci[p];
          a = A.v[p];
          const int64_t b0 = B.rp[k], b1 = B.rp[k + 1];
          int64_t e = b1;
          s = b0;
          if (groups == 1) {
            // whole row; in the upper mode rows of more than kMaskMax entries start at the first
            // column >= c_lo (a DFMA lane costs more than the search), shorter ones are masked
            // entry by entry
            if (upper && b1 - b0 > kMaskMax && B.ci[b0] < c_lo) s = lower_bound_col(B.ci, b0, b1, c_lo);
          } else if (b1 > b0) {
            const int f = B.ci[b0], l = B.ci[b1 - 1];
            if (f <= c_hi && l >= c_lo) {
              s = f >= c_lo ? b0 : lower_bound_col(B.ci, b0, b1, c_lo);
              e = l <= c_hi ? b1 : lower_bound_col(B.ci, s, b1, c_hi + 1);
            } else {
              e = s;
            }
          }
          len = (int)(e - s);
        }
        // the non-empty segments of this batch of 32 k's (ballot), in lane order
        unsigned live = __ballot_sync(FULL, len > 0);
        if (!live) continue;
        Quad qa, qb;
        {
          const int j = __ffs(live) - 1;
          live &= live - 1u;
          qa.s = __shfl_sync(FULL, s, j);
          qa.len = __shfl_sync(FULL, len, j);
          qa.a = __shfl_sync(FULL, a, j);
          load_quad(B, lane, qa);
        }
        if (mask_row) {
          while (pipe_stage<true, SH>(B, P, b, lane, s, len, a, live, qa, qb) &&
                 pipe_stage<true, SH>(B, P, b, lane, s, len, a, live, qb, qa)) {
          }
        } else {
          while (pipe_stage<false, SH>(B, P, b, lane, s, len, a, live, qa, qb) &&
                 pipe_stage<false, SH>(B, P, b, lane, s, len, a, live, qb, qa)) {
          }
        }
        __syncwarp();
      }
    }
    if (members > 1) {
      __syncthreads();
      for (int k = lo_pos + threadIdx.x; k < cnt; k += T) {
        double v = acc[k];
        for (int w = 1; w < members; ++w) v += acc[k + w * cacc];
        acc[k] = v;
      }
    }
  }
  __syncthreads();  // every accumulation (and the members' sum) is complete
  // 4. scaling (Taylor /i) and the fused beta D term (squaring +2T), in that order;
  //    a frozen row is a plain copy of D
  if (div != 1.0)
    for (int k = lo_pos + threadIdx.x; k < cnt; k += T) acc[k] = acc[k] / div;
  __syncthreads();
  if (hasD) {
    const double coef = fz ? 1.0 : beta;
    const int64_t d0 = D.rp[i], d1 = D.rp[i + 1];
    for (int64_t q = d0 + threadIdx.x; q < d1; q += T) {
      const int c = D.ci[q];
      if (upper && c < i) continue;
      const int pos = (int)rank_of(bp, c - b);
      acc[pos] += coef * D.v[q];
    }
  }
  __syncthreads();
  // 5. write the row in column order; per-row sum of squares and diagonal
  //    (upper: values below the diagonal are filled afterwards from the mirror entries, and an
  //    off-diagonal entry stands for itself and its mirror in the sum of squares)
  double sq = 0.0;
  for (int k = threadIdx.x; k < cnt; k += T) {
    const int col = b + column_at(bp, W, k);
    ci_out[o0 + k] = col;
    if (k < lo_pos) continue;
    const double v = acc[k];
    v_out[o0 + k] = v;
    sq += (upper && col != i) ? 2.0 * v * v : v * v;
    if (row_diag && col == i) row_diag[i] = v;
  }
  if (row_sq) {
    sq = block_sum(sq, dred);
    if (threadIdx.x == 0) row_sq[i] = sq;
  }
  __syncthreads();
}

// Numeric pass.  Layout per row: an accumulator region (the members' accumulators of cacc
// doubles each; before the accumulation it holds wk[W], the prefix product counts), then
// bp[W], the bitmap words with their position prefixes.
template <bool GLOBAL, int NT>
__global__ void __launch_bounds__(NT, (8 * SEXPM_NUMERIC_BLOCKS * 32) / NT) k_numeric(CsrD A, CsrD B, CsrD D, WPat WB, WPat WD, double div, double beta, bool upper,
                          const uint8_t* frozen, const int32_t* cnt_up, const int32_t* rows,
                          int64_t nrows, const unsigned long long* nrows_dev, const int32_t* base,
                          const int32_t* words, const int64_t* rp_out,
                          int32_t* ci_out, double* v_out, double* row_sq, double* row_diag, unsigned char* gscratch,
                          int64_t gstride, unsigned long long* work_total, unsigned long long* row_ctr,
                          int ks_bytes, int64_t out_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned ured[33];
  __shared__ double dred[32];
  __shared__ long long s_next;
  __shared__ double sink[NT / 32];  // per-warp target of masked accumulator updates (never read back)
  unsigned char* mem = GLOBAL ? gscratch + (int64_t)blockIdx.x * gstride : smem;
  const int T = blockDim.x;
  const bool hasD = D.n > 0;
  if (nrows_dev) nrows = min(nrows, (int64_t)*nrows_dev);  // list length decided on the device
  long long nxt = 0;
  for (int64_t r = blockIdx.x; r < nrows;) {
    if (threadIdx.x == 0) nxt = next_row(row_ctr);
    const int i = rows[r];
    const int W = words[i];
    const int b = base[i];
    const int64_t o0 = rp_out[i] - out_base;  // row i's entries go to ci_out/v_out at rp_out[i] - out_base
    const int cnt = (int)(rp_out[i + 1] - rp_out[i]);
    const int cacc = upper ? cnt_up[i] : cnt;   // entries accumulated: positions cnt - cacc .. cnt
    double* acc = reinterpret_cast<double*>(mem) - (cnt - cacc);  // indexed by full-row position
    unsigned* wk = reinterpret_cast<unsigned*>(mem);
    uint2* bp = reinterpret_cast<uint2*>(mem + acc_region(W, cnt, cacc, T >> 5, ks_bytes));
    for (int w = threadIdx.x; w < W; w += T) {
      bp[w].x = 0u;
      wk[w] = 0u;
    }
    if (row_diag && threadIdx.x == 0) row_diag[i] = 0.0;
    __syncthreads();
    // 1. pattern bitmap and products per word, from the word patterns
    const bool fz = frozen && frozen[i];
    build_row_bitmap<2>(A, WB, WD, hasD, i, b >> 5, reinterpret_cast<uint32_t*>(bp), wk, upper, fz);
    __syncthreads();
    numeric_row<!GLOBAL>(A, B, D, div, beta, upper, fz, i, W, b, o0, cnt, cnt - cacc, acc, wk, bp, &sink[threadIdx.x >> 5],
                ci_out, v_out, row_sq, row_diag, ured, dred, work_total, ks_bytes);
    if (threadIdx.x == 0) s_next = nxt;
    __syncthreads();
    r = s_next;
  }
}

// Fills the entries below the diagonal of a structurally symmetric product whose upper part
// (columns >= row) was computed: C[i][j] = C[j][i] for j < i, found in row j.
// One warp per row.  A partner that is absent (the pattern was not symmetric) counts a miss.
__global__ void k_mirror(int64_t n, const int64_t* rp, const int32_t* ci, double* v, unsigned long long* misses,
                         const int32_t* status) {
  if (status && *status) return;  // the product was not formed (capacity exceeded)
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < n; i += nw) {
    const int64_t p0 = rp[i], p1 = rp[i + 1];
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      const int j = ci[p];
      if (j >= i) break;
      const int64_t q0 = rp[j], q1 = rp[j + 1];
      // first probe: the point-mirrored index (rows that are translates of one symmetric
      // offset set hold column i of row j at index cnt_j - 1 - t when column j sits at
      // index t of row i), else binary search
      int64_t q = q1 - 1 - (p - p0);
      if (q < q0 || ci[q] != (int)i) q = lower_bound_col(ci, q0, q1, (int)i);
      if (q < q1 && ci[q] == (int)i) {
        v[p] = v[q];
      } else {
        v[p] = 0.0;
        atomicAdd(misses, 1ull);
      }
    }
  }
}

__global__ void k_zero_rows(const int32_t* words, int64_t n, double* row_sq, double* row_diag, int32_t* cnt,
                            int32_t* cnt_up) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && words[i] == 0) {
    if (row_sq) row_sq[i] = 0.0;
    if (row_diag) row_diag[i] = 0.0;
    cnt[i] = 0;
    if (cnt_up) cnt_up[i] = 0;
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

// Wide numeric blocks for the wide classes (SEXPM_WIDE_BLOCKS=0 turns them off; read per product).
bool wide_blocks() {
  const char* e = std::getenv("SEXPM_WIDE_BLOCKS");
  return !(e && *e == '0');
}

// Byte limit of the k split's accumulators: SEXPM_KSPLIT_BYTES from the environment (read on
// every product, so a process can compare the two accumulation modes), else the default.
int ksplit_bytes() {
  const char* e = std::getenv("SEXPM_KSPLIT_BYTES");
  if (!e || !*e) return kKsplitBytesDefault;
  const long v = std::strtol(e, nullptr, 10);
  return v < 0 ? 0 : (int)std::min<long>(v, 1l << 20);
}

// Blocks of `kernel` that are resident at once on the whole GPU (at least one per SM).
template <typename K>
int64_t resident_blocks(K kernel, int threads, int bytes) {
  int per_sm = 0;
  SX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, (size_t)bytes));
  return (int64_t)std::max(per_sm, 1) * num_sms();
}

// Dynamic shared-memory limit of the row kernels, once per device.
void set_smem_limits() {
  static bool done[64] = {};
  once_per_device(done, [] {
    const int cap = kClassBytes[kClasses - 2];
    SX_CUDA(cudaFuncSetAttribute(k_symbolic<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    SX_CUDA(cudaFuncSetAttribute(k_numeric<false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    SX_CUDA(cudaFuncSetAttribute(k_numeric<false, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    SX_CUDA(cudaFuncSetAttribute(k_numeric<false, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  });
}

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
  void start() {
    if (on) SX_CUDA(cudaEventRecord(a, s));
  }
  double stop() {
    if (!on) return 0.0;
    SX_CUDA(cudaEventRecord(b, s));
    SX_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    SX_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
};

// Owned word pattern.
struct WPatOwned {
  DevBuf<int64_t> rp;
  DevBuf<int32_t> wi;
  DevBuf<uint32_t> wb;
  WPat view() const {
    WPat w;
    w.rp = rp.p; w.wi = wi.p; w.wb = wb.p;
    return w;
  }
};

void word_pattern(const CsrD& X, cudaStream_t s, WPatOwned& out, HostScalars& hs) {
  const int64_t n = X.n;
  out.rp.reset(n + 1, s);
  DevBuf<int32_t> cnt(n, s);
  const int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)num_sms() * 64);
  k_wcount<<<blocks, 256, 0, s>>>(X, cnt.p);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  const int64_t total = scan_counts(cnt.p, n, out.rp.p, s, hs);
  out.wi.reset(total, s);
  out.wb.reset(total, s);
  k_wwrite<<<blocks, 256, 0, s>>>(X, out.rp.p, out.wi.p, out.wb.p, nullptr);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

// ---- device-sized products (the captured batched step)
// status |= bit when the size at *rp_n exceeds cap; need = the largest size requested.  Skipped
// once the status is set (an earlier step stopped the run: its sizes are not this run's).
__global__ void k_dev_cap_check(const int64_t* rp_n, int64_t cap, int32_t* status, unsigned long long* need,
                                int32_t bit) {
  if (*status) return;
  const long long total = *rp_n;
  atomicMax(need, (unsigned long long)total);
  if (total > cap) atomicOr(status, bit);
}

// Before a pass over the row lists: a row whose need exceeds the global class's scratch stride
// (a bound the buffers were sized by) stops the step; when the step is stopped every list is
// emptied so the row kernels form nothing.
// (A step already stopped -- its sizes come from skipped kernels -- is not judged.)
__global__ void k_dev_gate(unsigned long long* counts, const unsigned long long* maxneed, long long global_cap,
                           int32_t* status) {
  if (threadIdx.x != 0) return;
  if (*status == 0 && counts[kClasses - 1] > 0 && maxneed[kClasses - 1] > (unsigned long long)global_cap)
    atomicOr(status, kStBound);
  if (*status)
    for (int c = 0; c < kClasses; ++c) counts[c] = 0;
}

// Sets status bit `bit` when *x != 0.
__global__ void k_dev_flag_nonzero(const unsigned long long* x, int32_t* status, int32_t bit) {
  if (threadIdx.x == 0 && *x) atomicOr(status, bit);
}

// Arguments of one numeric launch (one size class).
struct NumericArgs {
  CsrD A, B, D;
  WPat WB, WD;
  double div, beta;
  bool upper;
  const uint8_t* frozen;
  const int32_t* cnt_up;
  const int32_t* rows;
  int64_t nrows;
  const unsigned long long* nrows_dev;  // non-null: the list length is read on the device
  const int32_t* base;
  const int32_t* words;
  const int64_t* rp_out;
  int32_t* ci_out;
  double* v_out;
  double* row_sq;
  double* row_diag;
  unsigned char* gscratch;
  int64_t gstride;
  unsigned long long* work_total;
  unsigned long long* row_ctr;
  int ks_bytes;
  int64_t out_base;
};

// Launches the numeric kernel instance for blocks of NT threads: a persistent grid of the blocks
// that are resident at once (grid > 0: that many).
template <bool GLOBAL, int NT>
void launch_numeric(const NumericArgs& a, int threads, int bytes, cudaStream_t s, int64_t grid = 0) {
  // (the 64- and 128-thread classes run the 256-thread instance with fewer threads)
  if (grid == 0) grid = std::min<int64_t>(a.nrows, resident_blocks(k_numeric<GLOBAL, NT>, threads, bytes));
  k_numeric<GLOBAL, NT><<<(unsigned)grid, threads, bytes, s>>>(
      a.A, a.B, a.D, a.WB, a.WD, a.div, a.beta, a.upper, a.frozen, a.cnt_up, a.rows, a.nrows, a.nrows_dev, a.base,
      a.words,
      a.rp_out, a.ci_out, a.v_out, a.row_sq, a.row_diag, a.gscratch, a.gstride, a.work_total, a.row_ctr,
      a.ks_bytes, a.out_base);
}

}  // namespace

void product_symbolic(const CsrD& A, const CsrD& B, const CsrD& D, bool upper, const uint8_t* frozen,
                      const int32_t* sched, RowStats* stats, cudaStream_t s, HostScalars& hs, ProductSym& ps) {
  const int64_t n = A.n;
  set_smem_limits();
  ps.n = n;
  ps.upper = upper;
  ps.frozen = frozen;
  ps.sched = sched;
  ps.hasD = D.n > 0;
  ps.ks_bytes = ksplit_bytes();
  ps.rp.reset(n + 1, s);
  if (stats) {
    stats->sq.reset(n, s);
    stats->diag.reset(n, s);
  }
  if (n == 0) {
    SX_CUDA(cudaMemsetAsync(ps.rp.p, 0, sizeof(int64_t), s));
    ps.nnz = 0;
    ps.products = 0;
    return;
  }
  const int sms = num_sms();
  WPatOwned wB, wD;
  word_pattern(B, s, wB, hs);
  ps.sameD = ps.hasD && D.rp == B.rp && D.ci == B.ci;
  if (ps.hasD && !ps.sameD) word_pattern(D, s, wD, hs);
  ps.wB_rp = std::move(wB.rp); ps.wB_wi = std::move(wB.wi); ps.wB_wb = std::move(wB.wb);
  ps.wD_rp = std::move(wD.rp); ps.wD_wi = std::move(wD.wi); ps.wD_wb = std::move(wD.wb);
  const WPat WB = ps.wpat_B(), WD = ps.wpat_D();
  ps.base.reset(n, s);
  ps.words.reset(n, s);
  ps.cnt.reset(n, s);
  ps.lists.reset((size_t)n * kClasses, s);
  ps.cnt_up.reset(upper ? n : 0, s);
  DevBuf<int64_t> flops(n, s);
  ps.ctr.reset(2 * kClasses + 4, s);
  SX_CUDA(cudaMemsetAsync(ps.ctr.p, 0, ps.ctr.count * sizeof(unsigned long long), s));
  {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + 7) / 8, (int64_t)sms * 64);
    k_analysis<<<(unsigned)blocks, threads, 0, s>>>(A, B, D, frozen, ps.base.p, ps.words.p, flops.p);
    SX_CUDA(cudaGetLastError());
    k_sum_i64<<<(unsigned)std::min<int64_t>((n + 255) / 256, sms * 8), 256, 0, s>>>(flops.p, n,
                                                                                 ps.ctr.p + 2 * kClasses + 2);
    k_classify<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, sched, ps.words.p, nullptr, nullptr, 0, ps.ks_bytes,
                                                         ps.lists.p, n, ps.ctr.p, ps.ctr.p + kClasses, 0, n, false);
    k_zero_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ps.words.p, n, stats ? stats->sq.p : nullptr,
                                                         stats ? stats->diag.p : nullptr, ps.cnt.p,
                                                         upper ? ps.cnt_up.p : nullptr);
    SX_CUDA(cudaGetLastError());
    count_launches(4);
  }
  ps.row_ctr.reset(2 * kClasses, s);
  SX_CUDA(cudaMemsetAsync(ps.row_ctr.p, 0, ps.row_ctr.count * sizeof(unsigned long long), s));
  unsigned long long h[2 * kClasses + 4];
  SX_CUDA(cudaMemcpyAsync(h, ps.ctr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  ps.products = (int64_t)h[2 * kClasses + 2];
  for (int c = 0; c < kClasses; ++c) ps.rows_symbolic[c] = (int64_t)h[c];
  // symbolic pass per class
  {
    DevBuf<uint32_t> gs;
    for (int c = 0; c < kClasses; ++c) {
      const int64_t nr = (int64_t)h[c];
      if (!nr) continue;
      const int threads = kClassThreads[c];
      const int64_t need = (int64_t)h[kClasses + c];
      if (c < kClasses - 1) {
        const int bytes = (int)((need + 1023) & ~1023ll);
        const int64_t grid = std::min<int64_t>(nr, resident_blocks(k_symbolic<false>, threads, bytes));
        k_symbolic<false><<<(unsigned)grid, threads, bytes, s>>>(A, WB, WD, ps.hasD, frozen, ps.lists.p + c * n, nr,
                                                               nullptr, ps.base.p, ps.words.p, ps.cnt.p,
                                                               upper ? ps.cnt_up.p : nullptr, nullptr, 0,
                                                               ps.row_ctr.p + c);
      } else {
        const int64_t stride = (need / 4 + 63) & ~63ll;
        const int64_t grid = std::min<int64_t>(nr, (int64_t)sms * 2);
        gs.reset((size_t)(stride * grid), s);
        k_symbolic<true><<<(unsigned)grid, threads, 0, s>>>(A, WB, WD, ps.hasD, frozen, ps.lists.p + c * n, nr,
                                                          nullptr, ps.base.p, ps.words.p, ps.cnt.p,
                                                          upper ? ps.cnt_up.p : nullptr, gs.p, stride,
                                                          ps.row_ctr.p + c);
      }
      SX_CUDA(cudaGetLastError());
      count_launches(1);
    }
  }
  // row pointers of the unfiltered product
  ps.nnz = scan_counts(ps.cnt.p, n, ps.rp.p, s, hs);
}

int64_t product_numeric(ProductSym& ps, const CsrD& A, const CsrD& B, const CsrD& D, double div, double beta,
                        int64_t r0, int64_t r1, int64_t out_base, int32_t* ci_out, double* v_out, RowStats* stats,
                        cudaStream_t s, HostScalars& hs) {
  const int64_t n = ps.n;
  if (n == 0 || r1 <= r0) return 0;
  const int sms = num_sms();
  const WPat WB = ps.wpat_B(), WD = ps.wpat_D();
  const bool upper = ps.upper;
  SX_CUDA(cudaMemsetAsync(ps.ctr.p, 0, ps.ctr.count * sizeof(unsigned long long), s));
  SX_CUDA(cudaMemsetAsync(ps.row_ctr.p + kClasses, 0, kClasses * sizeof(unsigned long long), s));
  const bool wide = wide_blocks();
  k_classify<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, ps.sched, ps.words.p, ps.row_ptr(),
                                                       upper ? ps.cnt_up.p : nullptr, 1, ps.ks_bytes, ps.lists.p, n,
                                                       ps.ctr.p, ps.ctr.p + kClasses, r0, r1, wide);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  unsigned long long h[2 * kClasses + 4];
  SX_CUDA(cudaMemcpyAsync(h, ps.ctr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < kClasses; ++c) ps.rows_numeric[c] += (int64_t)h[c];
  DevBuf<unsigned char> gs;
  for (int c = 0; c < kClasses; ++c) {
    const int64_t nr = (int64_t)h[c];
    if (!nr) continue;
    const int threads = wide ? kNumThreadsWide[c] : kClassThreads[c];
    const int64_t need = (int64_t)h[kClasses + c];
    NumericArgs na{A, B, D, WB, WD, div, beta, upper, ps.frozen, upper ? ps.cnt_up.p : nullptr, ps.lists.p + c * n, nr,
                   nullptr, ps.base.p, ps.words.p, ps.row_ptr(), ci_out, v_out, stats ? stats->sq.p : nullptr,
                   stats ? stats->diag.p : nullptr, nullptr, 0, ps.ctr.p + 2 * kClasses + 3,
                   ps.row_ctr.p + kClasses + c, ps.ks_bytes, out_base};
    if (c < kClasses - 1) {
      const int bytes = (int)((need + 1023) & ~1023ll);
      if (threads <= 256) launch_numeric<false, 256>(na, threads, bytes, s);
      else if (threads == 512) launch_numeric<false, 512>(na, threads, bytes, s);
      else launch_numeric<false, 1024>(na, threads, bytes, s);
    } else {
      const int64_t stride = (need + 255) & ~255ll;
      // two resident blocks per SM up to 512 threads, one at 1024 (the register budget); the
      // scratch slices of one wave of blocks then stay within L2 for rows up to ~800 KB
      const int64_t grid = std::min<int64_t>(nr, (int64_t)sms * (threads >= 1024 ? 1 : 2));
      gs.reset((size_t)(stride * grid), s);
      na.gscratch = gs.p;
      na.gstride = stride;
      if (threads <= 256) launch_numeric<true, 256>(na, threads, 0, s, grid);
      else if (threads == 512) launch_numeric<true, 512>(na, threads, 0, s, grid);
      else launch_numeric<true, 1024>(na, threads, 0, s, grid);
    }
    SX_CUDA(cudaGetLastError());
    count_launches(1);
  }
  SX_CUDA(cudaMemcpyAsync(h + 2 * kClasses + 3, ps.ctr.p + 2 * kClasses + 3, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return (int64_t)h[2 * kClasses + 3];
}

void mirror_lower(const CsrOwned& C, cudaStream_t s, HostScalars& hs) {
  const int64_t n = C.n;
  if (n == 0) return;
  DevBuf<unsigned long long> miss(1, s);
  SX_CUDA(cudaMemsetAsync(miss.p, 0, sizeof(unsigned long long), s));
  const int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)num_sms() * 64);
  k_mirror<<<blocks, 256, 0, s>>>(n, C.rp.p, C.ci.p, C.v.p, miss.p, nullptr);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  unsigned long long h = 0;
  SX_CUDA(cudaMemcpyAsync(hs.i, miss.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  std::memcpy(&h, hs.i, sizeof(h));
  if (h != 0) fail(SEXPM_ECUDA, "symmetric product: " + std::to_string(h) + " entries without a mirror partner");
}

int64_t spgemm(const CsrD& A, const CsrD& B, const CsrD& D, double div, double beta, cudaStream_t s, CsrOwned& C,
               RowStats* stats, HostScalars& hs, SpgemmTimes* times, bool upper, int64_t* done,
               const uint8_t* frozen, const int32_t* sched, int64_t* rows_class) {
  const int64_t n = A.n;
  EventPair ev_sym(times != nullptr, s), ev_num(times != nullptr, s);
  ev_sym.start();
  ProductSym ps;
  product_symbolic(A, B, D, upper, frozen, sched, stats, s, hs, ps);
  C.n = n;
  C.nnz = ps.nnz;
  C.rp = std::move(ps.rp);
  ps.rp_ext = C.rp.p;  // the numeric pass reads the row pointers from C now
  C.ci.reset(C.nnz, s);
  C.v.reset(C.nnz, s);
  if (times) times->ms_symbolic += ev_sym.stop();
  ev_num.start();
  const int64_t formed = product_numeric(ps, A, B, D, div, beta, 0, n, 0, C.ci.p, C.v.p, stats, s, hs);
  if (done) *done = formed;
  if (rows_class)
    for (int c = 0; c < kClasses; ++c) rows_class[c] = ps.rows_numeric[c];
  if (upper) mirror_lower(C, s, hs);
  if (times) times->ms_numeric += ev_num.stop();
  return ps.products;
}

// ---------------------------------------------------------------- device-sized product
// The same kernels as spgemm, launched with grids and shared-memory sizes that do not depend on
// the data: the size classes use their class's full shared-memory budget, the persistent
// row kernels read their list lengths on the device, and the global-memory class uses scratch
// sized for the widest row an instance of n_max rows can have.  Nothing is read back, so the
// sequence can be captured into a CUDA graph.  Results equal spgemm's bit for bit (the
// accumulation layout of a row depends only on the row and its class).

namespace {
constexpr int kCtrHalf = 2 * kClasses + 4;  // counters per half of DevProduct::ctr
}  // namespace

int default_ks_bytes() { return ksplit_bytes(); }
bool default_wide_blocks() { return wide_blocks(); }

int dev_product_products_index() { return 2 * kClasses + 2; }
int dev_product_formed_index() { return kCtrHalf + 2 * kClasses + 3; }

void dev_product_scratch(int64_t n_max, int ks_bytes, bool wide, int64_t& sym_stride, int64_t& sym_grid,
                         int64_t& num_stride, int64_t& num_grid) {
  // A row of an instance with n_max rows spans at most n_max columns from a 32-aligned base:
  // W <= n_max / 32 + 2 bitmap words and at most n_max entries.
  const int64_t W = n_max / 32 + 2;
  sym_stride = (W + 63) & ~63ll;  // uint32 words (the symbolic need is 4 W bytes)
  sym_grid = (int64_t)num_sms() * 2;
  // numeric: the k split keeps a row within ks_bytes * warps / 32 unless one accumulator does
  // not fit, so the need is at most max(that budget, the need of one accumulator)
  const int threads = wide ? kNumThreadsWide[kClasses - 1] : kClassThreads[kClasses - 1];
  const long long one = need_bytes(W, n_max, n_max, 1);
  const long long need = std::max<long long>((long long)ks_bytes * (threads / 32) / kNumericWarpsPerSM, one);
  num_stride = (need + 255) & ~255ll;
  num_grid = (int64_t)num_sms() * (threads >= 1024 ? 1 : 2);
}

void dev_product_prepare(DevProduct& P) {
  set_smem_limits();
  for (int c = 0; c < kClasses - 1; ++c) {
    const int bytes = class_limit(c);
    P.grid_sym[c] = resident_blocks(k_symbolic<false>, kClassThreads[c], bytes);
    const int threads = P.wide ? kNumThreadsWide[c] : kClassThreads[c];
    P.grid_num[c] = threads <= 256   ? resident_blocks(k_numeric<false, 256>, threads, bytes)
                    : threads == 512 ? resident_blocks(k_numeric<false, 512>, threads, bytes)
                                     : resident_blocks(k_numeric<false, 1024>, threads, bytes);
  }
  P.grid_sym[kClasses - 1] = P.gs_sym_grid;
  P.grid_num[kClasses - 1] = P.gs_num_grid;
  P.prepared = true;
}

void dev_product(const CsrD& A, const CsrD& B, bool hasD, double div, double beta, bool upper, const uint8_t* frozen,
                 const DevProduct& P, cudaStream_t s) {
  const int64_t n = P.n;
  if (!P.prepared) fail(SEXPM_ECUDA, "dev_product: launch shapes not prepared");
  const int sms = num_sms();
  CsrD D;
  if (hasD) D = B;
  WPat WB;
  WB.rp = P.wrp; WB.wi = P.wi; WB.wb = P.wb;
  const WPat WD = hasD ? WB : WPat();
  unsigned long long* cs = P.ctr;             // symbolic half
  unsigned long long* cn = P.ctr + kCtrHalf;  // numeric half
  SX_CUDA(cudaMemsetAsync(P.ctr, 0, 2 * kCtrHalf * sizeof(unsigned long long), s));
  SX_CUDA(cudaMemsetAsync(P.row_ctr, 0, 2 * kClasses * sizeof(unsigned long long), s));
  const int rblocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sms * 64);
  // word pattern of B, within its capacity
  k_wcount<<<rblocks, 256, 0, s>>>(B, P.cnt);
  SX_CUDA(cudaGetLastError());
  scan_counts_dev(P.cnt, n, P.wrp, P.scan_ts, s);
  k_dev_cap_check<<<1, 1, 0, s>>>(P.wrp + n, P.wcap, P.status, P.need_w, kStWords);
  k_wwrite<<<rblocks, 256, 0, s>>>(B, P.wrp, P.wi, P.wb, P.status);
  // analysis and symbolic classes
  k_analysis<<<rblocks, 256, 0, s>>>(A, B, D, frozen, P.base, P.words, P.flops);
  k_sum_i64<<<(unsigned)std::min<int64_t>((n + 255) / 256, sms * 8), 256, 0, s>>>(P.flops, n,
                                                                               cs + dev_product_products_index());
  k_classify<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nullptr, P.words, nullptr, nullptr, 0, P.ks_bytes, P.lists,
                                                       n, cs, cs + kClasses, 0, n, false);
  k_zero_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P.words, n, P.row_sq, P.row_diag, P.cnt,
                                                       upper ? P.cnt_up : nullptr);
  k_dev_gate<<<1, 32, 0, s>>>(cs, cs + kClasses, 4 * P.gs_sym_stride, P.status);
  SX_CUDA(cudaGetLastError());
  count_launches(8);
  for (int c = 0; c < kClasses; ++c) {
    const int threads = kClassThreads[c];
    if (c < kClasses - 1) {
      const int bytes = class_limit(c);
      k_symbolic<false><<<(unsigned)P.grid_sym[c], threads, bytes, s>>>(A, WB, WD, hasD, frozen, P.lists + c * n, n,
                                                                       cs + c, P.base, P.words, P.cnt,
                                                                       upper ? P.cnt_up : nullptr, nullptr, 0,
                                                                       P.row_ctr + c);
    } else {
      k_symbolic<true><<<(unsigned)P.gs_sym_grid, threads, 0, s>>>(A, WB, WD, hasD, frozen, P.lists + c * n, n, cs + c,
                                                                  P.base, P.words, P.cnt, upper ? P.cnt_up : nullptr,
                                                                  P.gs_sym, P.gs_sym_stride, P.row_ctr + c);
    }
    SX_CUDA(cudaGetLastError());
    count_launches(1);
  }
  // row pointers of the unfiltered product and its capacity
  scan_counts_dev(P.cnt, n, P.rp_out, P.scan_ts, s);
  k_dev_cap_check<<<1, 1, 0, s>>>(P.rp_out + n, P.cap_out, P.status, P.need, kStProduct);
  const bool wide = P.wide;
  k_classify<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nullptr, P.words, P.rp_out, upper ? P.cnt_up : nullptr, 1,
                                                       P.ks_bytes, P.lists, n, cn, cn + kClasses, 0, n, wide);
  k_dev_gate<<<1, 32, 0, s>>>(cn, cn + kClasses, P.gs_num_stride, P.status);
  SX_CUDA(cudaGetLastError());
  count_launches(3);
  for (int c = 0; c < kClasses; ++c) {
    const int threads = wide ? kNumThreadsWide[c] : kClassThreads[c];
    NumericArgs na{A, B, D, WB, WD, div, beta, upper, frozen, upper ? P.cnt_up : nullptr, P.lists + c * n, n, cn + c,
                   P.base, P.words, P.rp_out, P.ci_out, P.v_out, P.row_sq, P.row_diag, nullptr, 0,
                   cn + 2 * kClasses + 3, P.row_ctr + kClasses + c, P.ks_bytes, 0};
    if (c < kClasses - 1) {
      const int bytes = class_limit(c);
      if (threads <= 256) launch_numeric<false, 256>(na, threads, bytes, s, P.grid_num[c]);
      else if (threads == 512) launch_numeric<false, 512>(na, threads, bytes, s, P.grid_num[c]);
      else launch_numeric<false, 1024>(na, threads, bytes, s, P.grid_num[c]);
    } else {
      na.gscratch = P.gs_num;
      na.gstride = P.gs_num_stride;
      if (threads <= 256) launch_numeric<true, 256>(na, threads, 0, s, P.gs_num_grid);
      else if (threads == 512) launch_numeric<true, 512>(na, threads, 0, s, P.gs_num_grid);
      else launch_numeric<true, 1024>(na, threads, 0, s, P.gs_num_grid);
    }
    SX_CUDA(cudaGetLastError());
    count_launches(1);
  }
  if (upper) {
    unsigned long long* miss = cn + 2 * kClasses + 2;  // unused by the numeric classification
    k_mirror<<<rblocks, 256, 0, s>>>(n, P.rp_out, P.ci_out, P.v_out, miss, P.status);
    k_dev_flag_nonzero<<<1, 32, 0, s>>>(miss, P.status, kStMirror);
    SX_CUDA(cudaGetLastError());
    count_launches(2);
  }
}

}  // namespace sexpm
