// Algorithm 4.1 (forward-error filter) kernels over the stored values of a sparse matrix held
// as one or more row-range "pieces" (CSR blocks with local row pointers):
//
//  * k_pass_flat: one reduction pass, sum of v^2 over |v| <= t, streaming the value array as
//    16-byte pairs in tiles of kTile entries; it also writes the number of kept entries
//    (|v| > t) that each warp saw in each tile, so that the compaction after the last pass needs
//    no count pass.
//  * k_compact_flat: A~ = A - b_n, the kept entries of a tile go to the output at the tile's
//    scanned offset plus their rank inside the tile; the rows that start inside the tile get
//    their output row pointers from the same ranks.  Neither kernel looks at row boundaries
//    while streaming, so both run at the bandwidth of a plain copy whatever the row lengths.
//  * k_drop_rows / k_compact_rows: the exact streaming step used when a squaring product is
//    formed in row chunks.  Every threshold Algorithm 4.1 visits is at least
//    eps_g / sqrt(nnz) (t_0 = eps_g; b_j <= sqrt(nnz) t_j since every dropped entry is <= t_j;
//    t_{j+1} = eps_g t_j / b_j), so entries at or below a lower bound L of that value are
//    dropped by every pass: a chunk keeps only its entries above L (plus the sum of squares
//    of the others) and is freed, and Algorithm 4.1 then runs on the kept pieces.
//
// All sums have an order fixed by the input and the launch shapes.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kTile = 2048;          // entries per tile: 256 threads x 4 pairs
constexpr int kFlatThreads = 256;
constexpr int kWarpsPerTile = kFlatThreads / 32;  // kept counts per tile (one per warp)
constexpr int kFlatBlocks = 1024;    // fixed reduction grid of a pass (sums do not depend on timing)
constexpr int kRowBlocks = 1024;     // fixed grid of the row-wise chunk kernels

// |v| > t for finite v and t >= 0, on the bit patterns (non-negative doubles are ordered as
// unsigned integers), so the test takes no FP64 instruction.
__device__ __forceinline__ bool above(double v, unsigned long long tb) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) > tb;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Bits 0..15 of x moved to the even positions 0, 2, .., 30.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Loads pair j (entries 2j, 2j+1) of tile k: 16-byte loads when the pair is complete and the
// array is 16-byte aligned, else element loads; entries past nnz read as 0 (dropped, adding 0).
template <bool VEC>
__device__ __forceinline__ double2 load_pair(const double* v, int64_t e, int64_t nnz) {
  if (VEC && e + 1 < nnz) return __ldg(reinterpret_cast<const double2*>(v + e));
  double2 r;
  r.x = e < nnz ? __ldg(v + e) : 0.0;
  r.y = e + 1 < nnz ? __ldg(v + e + 1) : 0.0;
  return r;
}
template <bool VEC>
__device__ __forceinline__ int2 load_pair_i(const int32_t* c, int64_t e, int64_t nnz) {
  if (VEC && e + 1 < nnz) return __ldg(reinterpret_cast<const int2*>(c + e));
  int2 r;
  r.x = e < nnz ? __ldg(c + e) : 0;
  r.y = e + 1 < nnz ? __ldg(c + e + 1) : 0;
  return r;
}

// One Algorithm 4.1 pass: part[block] = sum over the block's tiles of v^2 for |v| <= t, and
// wcnt[8 k + w] = #{|v| > t} among the entries warp w reads in tile k (its four 64-entry
// groups).  Block b takes tiles b, b + grid, ...; each thread loads the next tile's four 16-byte
// pairs before it works on the current ones, and no barrier is taken per tile, so the loads of
// two tiles are in flight while the block computes (the stream would otherwise be latency-bound).
template <bool VEC>
__device__ __forceinline__ void load_tile(const double* v, int64_t nnz, int64_t e0, double2 (&x)[4]) {
  if (VEC && e0 + kTile <= nnz) {
    const double2* p = reinterpret_cast<const double2*>(v + e0) + threadIdx.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = __ldg(p + u * kFlatThreads);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = load_pair<false>(v, e0 + 2 * (u * kFlatThreads + threadIdx.x), nnz);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kFlatThreads) k_pass_flat(const double* __restrict__ v, int64_t nnz,
                                                            unsigned long long tb, int32_t* __restrict__ wcnt,
                                                            double* __restrict__ part) {
  __shared__ double red_s[kFlatThreads / 32];
  const int64_t tiles = (nnz + kTile - 1) / kTile;
  double s = 0.0;
  double2 x[4], y[4];
  int64_t k = blockIdx.x;
  if (k < tiles) load_tile<VEC>(v, nnz, k * kTile, x);
  for (; k < tiles; k += gridDim.x) {
    const int64_t kn = k + gridDim.x;
    if (kn < tiles) load_tile<VEC>(v, nnz, kn * kTile, y);
    int c = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool a0 = above(x[u].x, tb), a1 = above(x[u].y, tb);
      c += __popc(__ballot_sync(FULL, a0)) + __popc(__ballot_sync(FULL, a1));
      if (!a0) s = fma(x[u].x, x[u].x, s);
      if (!a1) s = fma(x[u].y, x[u].y, s);
    }
    if (lane_id() == 0) wcnt[k * kWarpsPerTile + warp_id()] = c;
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = y[u];
  }
  s = warp_sum(s);
  if (lane_id() == 0) red_s[warp_id()] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kFlatThreads / 32; ++w) t += red_s[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_sum_parts(const double* part, int m, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if (lane_id() == 0) red[warp_id()] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// First index i in [0, n] with rp[i] >= x (rp non-decreasing, n + 1 entries), by one warp:
// a 32-way search, each round one load per lane.
__device__ int64_t warp_lower_bound(const int64_t* rp, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n + 1;  // the answer lies in [lo, hi) (it exists: x <= rp[n])
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t idx = lo + (int64_t)lane_id() * step;
    const bool less = idx < hi && __ldg(rp + idx) < x;
    const int c = __popc(__ballot_sync(FULL, less));
    if (c == 0) { hi = lo; break; }
    // lanes 0..c-1 are below x: the answer lies after lane c-1's index and at or before lane c's
    const int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
    const int64_t nhi = min(hi, lo + (int64_t)c * step + 1);
    lo = nlo;
    hi = nhi;
  }
  if (hi > lo) {
    const int64_t idx = lo + lane_id();
    const bool less = idx < hi && __ldg(rp + idx) < x;
    lo += __popc(__ballot_sync(FULL, less));
  }
  return lo;
}

// Compaction of one piece by tiles (one block per tile).  Kept entries (|v| > t) of tile k go
// to out_ci/out_v at tile_off[8 k] (the scan of the pass's per-warp counts at the tile's first
// warp) + their rank among the tile's kept entries; rows of the piece whose first entry lies in
// tile k (for the last tile also the rows that start at nnz) get out_rp[i] = that offset + the
// number of kept entries of the tile before that entry.
template <bool VEC>
__global__ void __launch_bounds__(kFlatThreads) k_compact_flat(const int64_t* __restrict__ rp, int64_t nrows,
                                                               const int32_t* __restrict__ ci,
                                                               const double* __restrict__ v, int64_t nnz,
                                                               unsigned long long tb, const int64_t* __restrict__ tile_off,
                                                               int64_t* __restrict__ out_rp, int32_t* __restrict__ out_ci,
                                                               double* __restrict__ out_v) {
  constexpr int NW = kFlatThreads / 32;
  __shared__ uint32_t bits[kTile / 32];  // kept flags of the tile, entry order
  __shared__ unsigned wpre[kTile / 32];  // kept entries before each word
  __shared__ unsigned seg[4][NW];        // kept entries before (pair group u, warp w)
  __shared__ int64_t s_row0;
  const int64_t k = blockIdx.x;
  const int64_t e0 = k * kTile;
  const int64_t tiles = (nnz + kTile - 1) / kTile;
  const bool last = k == tiles - 1;
  const int lane = lane_id(), w = warp_id();
  if (w == NW - 1) {
    const int64_t r = warp_lower_bound(rp, nrows, e0);
    if (lane == 0) s_row0 = r;
  }
  double2 x[4];
  int2 c[4];
  unsigned b0[4], b1[4];
  if (VEC && e0 + kTile <= nnz) {
    // a full tile: eight unconditional 16- and 8-byte loads in flight per thread
    const double2* pv = reinterpret_cast<const double2*>(v + e0) + threadIdx.x;
    const int2* pc = reinterpret_cast<const int2*>(ci + e0) + threadIdx.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[u] = __ldg(pv + u * kFlatThreads);
      c[u] = __ldg(pc + u * kFlatThreads);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + 2 * (u * kFlatThreads + threadIdx.x);
      x[u] = load_pair<false>(v, e, nnz);
      c[u] = load_pair_i<false>(ci, e, nnz);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    b0[u] = __ballot_sync(FULL, above(x[u].x, tb));
    b1[u] = __ballot_sync(FULL, above(x[u].y, tb));
  }
  if (lane == 0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      seg[u][w] = __popc(b0[u]) + __popc(b1[u]);
      // entries 512 u + 64 w + 2 l + {0, 1} (lane l): words 16 u + 2 w (lanes 0..15) and + 1
      bits[16 * u + 2 * w] = spread16(b0[u]) | (spread16(b1[u]) << 1);
      bits[16 * u + 2 * w + 1] = spread16(b0[u] >> 16) | (spread16(b1[u] >> 16) << 1);
    }
  }
  __syncthreads();
  if (w == 0) {
    // exclusive scan of the 32 group counts in (u, w) order, and of the 64 word counts
    unsigned* sflat = &seg[0][0];
    const unsigned val = sflat[lane];
    unsigned inc = val;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    sflat[lane] = inc - val;
    const unsigned p0 = __popc(bits[2 * lane]), p1 = __popc(bits[2 * lane + 1]);
    unsigned wi = p0 + p1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, wi, o);
      if (lane >= o) wi += y;
    }
    wpre[2 * lane] = wi - p0 - p1;
    wpre[2 * lane + 1] = wi - p1;
  }
  __syncthreads();
  const int64_t base = tile_off[k * kWarpsPerTile];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t pos = base + seg[u][w] + __popc(b0[u] & lt) + __popc(b1[u] & lt);
    if ((b0[u] >> lane) & 1u) {
      out_ci[pos] = c[u].x;
      out_v[pos] = x[u].x;
      ++pos;
    }
    if ((b1[u] >> lane) & 1u) {
      out_ci[pos] = c[u].y;
      out_v[pos] = x[u].y;
    }
  }
  // row pointers of the rows that start in this tile
  const unsigned tile_total = wpre[kTile / 32 - 1] + __popc(bits[kTile / 32 - 1]);
  const int64_t e_hi = last ? nnz + 1 : e0 + kTile;
  for (int64_t i = s_row0 + threadIdx.x; i < nrows; i += kFlatThreads) {
    const int64_t r = rp[i];
    if (r >= e_hi) break;
    const int64_t pos = r - e0;
    unsigned rank;
    if (pos >= kTile) {
      rank = tile_total;
    } else {
      const int wd = (int)(pos >> 5);
      rank = wpre[wd] + __popc(bits[wd] & ((1u << (pos & 31)) - 1u));
    }
    out_rp[i] = base + rank;
  }
}

__global__ void k_fill_i64(int64_t* out, int64_t count, const int64_t* val) {
  const int64_t x = *val;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x;
}

// ---------------------------------------------------------------- exact streaming of a chunk

__device__ __forceinline__ int64_t lb_col(const int32_t* ci, int64_t lo, int64_t hi, int c) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Value of entry (j, c) stored in the earlier pieces (rows < the current chunk); found = false
// when it was dropped.
__device__ __forceinline__ double piece_lookup(const Piece* pieces, int np, int64_t j, int c, bool& found) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pieces[mid].r0 <= j) lo = mid; else hi = mid - 1;
  }
  const Piece P = pieces[lo];
  const int64_t q0 = P.rp[j - P.r0], q1 = P.rp[j - P.r0 + 1];
  const int64_t q = lb_col(P.ci, q0, q1, c);
  found = q < q1 && P.ci[q] == c;
  return found ? P.v[q] : 0.0;
}

// Rows [r0, r1) of a chunk of an unfiltered product (row i at rp[i] - base .. rp[i+1] - base of
// ci/v).  Upper entries (col >= row; every entry when !sym) are kept iff |v| > L; a dropped one
// adds v^2 to the block's partial sum, twice for an off-diagonal entry in the symmetric mode (it
// stands for its mirror too).  In the symmetric mode a lower entry (col < row) takes the value of
// its mirror (col, row) and that entry's decision: from this chunk when col >= r0, else from the
// earlier pieces; v is written (0 when the pair was dropped).  keep[i - r0] = kept entries of row i.
__global__ void __launch_bounds__(256) k_drop_rows(int64_t r0, int64_t r1, const int64_t* __restrict__ rp,
                                                   int64_t base, const int32_t* __restrict__ ci, double* v, int sym,
                                                   unsigned long long Lb, const Piece* __restrict__ pieces, int npieces,
                                                   int32_t* __restrict__ keep, double* __restrict__ part) {
  __shared__ double red[8];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  double s = 0.0;
  for (int64_t i = r0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < r1; i += nw) {
    const int64_t p0 = rp[i] - base, p1 = rp[i + 1] - base;
    int cnt = 0;
    for (int64_t p = p0 + lane_id(); p < p1; p += 32) {
      const int c = ci[p];
      if (sym && c < i) {
        double x = 0.0;
        bool kept = false;
        if (c >= r0) {
          const int64_t q0 = rp[c] - base, q1 = rp[c + 1] - base;
          int64_t q = q1 - 1 - (p - p0);  // point-mirrored position (exact for translated symmetric rows)
          if (q < q0 || q >= q1 || ci[q] != (int)i) q = lb_col(ci, q0, q1, (int)i);
          if (q < q1 && ci[q] == (int)i) {
            x = v[q];
            kept = above(x, Lb);
          }
        } else {
          x = piece_lookup(pieces, npieces, c, (int)i, kept);
        }
        v[p] = kept ? x : 0.0;
        cnt += kept;
      } else {
        const double x = v[p];
        if (above(x, Lb)) {
          ++cnt;
        } else {
          const double w = (sym && c != i) ? 2.0 : 1.0;
          s = fma(w * x, x, s);
        }
      }
    }
    cnt = warp_sum(cnt);
    if (lane_id() == 0) keep[i - r0] = cnt;
  }
  s = warp_sum(s);
  if (lane_id() == 0) red[warp_id()] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// Copies the entries k_drop_rows kept into a piece (local row pointers out_rp, r1 - r0 + 1).
__global__ void __launch_bounds__(256) k_compact_rows(int64_t r0, int64_t r1, const int64_t* __restrict__ rp,
                                                      int64_t base, const int32_t* __restrict__ ci,
                                                      const double* __restrict__ v, int sym, unsigned long long Lb,
                                                      const int64_t* __restrict__ out_rp, int32_t* __restrict__ out_ci,
                                                      double* __restrict__ out_v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane_id()) - 1u;
  for (int64_t i = r0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < r1; i += nw) {
    const int64_t q0 = rp[i] - base, q1 = rp[i + 1] - base;
    int64_t o = out_rp[i - r0];
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane_id();
      bool k = false;
      int c = 0;
      double x = 0.0;
      if (q < q1) {
        c = ci[q];
        x = v[q];
        k = (sym && c < i) ? (x != 0.0) : above(x, Lb);
      }
      const unsigned m = __ballot_sync(FULL, k);
      if (k) {
        const int64_t d = o + __popc(m & lt);
        out_ci[d] = c;
        out_v[d] = x;
      }
      o += __popc(m);
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// part[block] = sum over the block's rows r0 <= i < r1 of sum_j (delta_ij + a_ij)^2 (one warp per row).
__global__ void k_norm2_I_plus_rows(CsrD A, int64_t r0, int64_t r1, double* part) {
  __shared__ double red[8];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  double s = 0.0;
  for (int64_t i = r0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < r1; i += nw) {
    bool diag = false;
    for (int64_t p = A.rp[i] + lane_id(); p < A.rp[i + 1]; p += 32) {
      const double x = A.v[p];
      if (A.ci[p] == (int)i) {
        diag = true;
        s = fma(1.0 + x, 1.0 + x, s);
      } else {
        s = fma(x, x, s);
      }
    }
    if (!__any_sync(FULL, diag) && lane_id() == 0) s += 1.0;
  }
  s = warp_sum(s);
  if (lane_id() == 0) red[warp_id()] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

}  // namespace

double norm2_I_plus_rows(const CsrD& A, int64_t r0, int64_t r1, cudaStream_t s, HostScalars& hs) {
  if (r1 <= r0) return 0.0;
  const int grid = (int)std::min<int64_t>(kRowBlocks, (r1 - r0 + 7) / 8);
  DevBuf<double> part(grid + 1, s);
  k_norm2_I_plus_rows<<<grid, 256, 0, s>>>(A, r0, r1, part.p);
  k_sum_parts<<<1, 1024, 0, s>>>(part.p, grid, part.p + grid);
  SX_CUDA(cudaGetLastError());
  count_launches(2);
  SX_CUDA(cudaMemcpyAsync(hs.d, part.p + grid, sizeof(double), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return hs.d[0];
}

// ---------------------------------------------------------------- host side

int64_t tiles_of(int64_t nnz) { return (nnz + kTile - 1) / kTile; }
int64_t counts_of(int64_t nnz) { return tiles_of(nnz) * kWarpsPerTile; }

double pass_pieces(const std::vector<Piece>& P, const std::vector<int64_t>& tile_base, double t, int32_t* tile_cnt,
                   cudaStream_t s, HostScalars& hs) {
  int64_t nparts = 0;
  std::vector<int> grids(P.size(), 0);
  for (size_t p = 0; p < P.size(); ++p) {
    grids[p] = (int)std::min<int64_t>(kFlatBlocks, tiles_of(P[p].nnz));
    nparts += grids[p];
  }
  if (nparts == 0) return 0.0;
  DevBuf<double> part(nparts + 1, s);
  unsigned long long tb;
  std::memcpy(&tb, &t, sizeof(tb));
  int64_t off = 0;
  for (size_t p = 0; p < P.size(); ++p) {
    if (!grids[p]) continue;
    if (aligned16(P[p].v))
      k_pass_flat<true><<<grids[p], kFlatThreads, 0, s>>>(P[p].v, P[p].nnz, tb, tile_cnt + tile_base[p], part.p + off);
    else
      k_pass_flat<false><<<grids[p], kFlatThreads, 0, s>>>(P[p].v, P[p].nnz, tb, tile_cnt + tile_base[p], part.p + off);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
    off += grids[p];
  }
  k_sum_parts<<<1, 1024, 0, s>>>(part.p, (int)nparts, part.p + nparts);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
  SX_CUDA(cudaMemcpyAsync(hs.d, part.p + nparts, sizeof(double), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return hs.d[0];
}

void compact_pieces(const std::vector<Piece>& P, const std::vector<int64_t>& tile_base, double t,
                    const int64_t* tile_off, int64_t n, CsrOwned& out, cudaStream_t s) {
  unsigned long long tb;
  std::memcpy(&tb, &t, sizeof(tb));
  for (size_t p = 0; p < P.size(); ++p) {
    const Piece& Q = P[p];
    const int64_t tiles = tiles_of(Q.nnz);
    const int64_t nrows = Q.r1 - Q.r0;
    if (tiles == 0) {
      if (nrows > 0) {
        const int g = (int)std::min<int64_t>((nrows + 255) / 256, 4096);
        k_fill_i64<<<g, 256, 0, s>>>(out.rp.p + Q.r0, nrows, tile_off + tile_base[p]);
        SX_CUDA(cudaGetLastError());
        count_launches(1);
      }
      continue;
    }
    const bool vec = aligned16(Q.v) && (reinterpret_cast<uintptr_t>(Q.ci) & 7u) == 0;
    if (vec)
      k_compact_flat<true><<<(unsigned)tiles, kFlatThreads, 0, s>>>(Q.rp, nrows, Q.ci, Q.v, Q.nnz, tb,
                                                                   tile_off + tile_base[p], out.rp.p + Q.r0, out.ci.p,
                                                                   out.v.p);
    else
      k_compact_flat<false><<<(unsigned)tiles, kFlatThreads, 0, s>>>(Q.rp, nrows, Q.ci, Q.v, Q.nnz, tb,
                                                                    tile_off + tile_base[p], out.rp.p + Q.r0, out.ci.p,
                                                                    out.v.p);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
  }
  // out.rp[n] = total kept (the scan's last entry)
  const int64_t total_counts = tile_base.empty() ? 0 : tile_base.back();
  SX_CUDA(cudaMemcpyAsync(out.rp.p + n, tile_off + total_counts, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
}

double drop_rows(int64_t r0, int64_t r1, const int64_t* rp, int64_t base, const int32_t* ci, double* v, bool sym,
                 double L, const Piece* pieces, int npieces, int32_t* keep, cudaStream_t s, HostScalars& hs) {
  if (r1 <= r0) return 0.0;
  unsigned long long Lb;
  std::memcpy(&Lb, &L, sizeof(Lb));
  const int grid = (int)std::min<int64_t>(kRowBlocks, (r1 - r0 + 7) / 8);
  DevBuf<double> part(grid + 1, s);
  k_drop_rows<<<grid, 256, 0, s>>>(r0, r1, rp, base, ci, v, sym ? 1 : 0, Lb, pieces, npieces, keep, part.p);
  k_sum_parts<<<1, 1024, 0, s>>>(part.p, grid, part.p + grid);
  SX_CUDA(cudaGetLastError());
  count_launches(2);
  SX_CUDA(cudaMemcpyAsync(hs.d, part.p + grid, sizeof(double), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return hs.d[0];
}

void compact_rows(int64_t r0, int64_t r1, const int64_t* rp, int64_t base, const int32_t* ci, const double* v, bool sym,
                  double L, const int64_t* out_rp, int32_t* out_ci, double* out_v, cudaStream_t s) {
  if (r1 <= r0) return;
  unsigned long long Lb;
  std::memcpy(&Lb, &L, sizeof(Lb));
  const int grid = (int)std::min<int64_t>(kRowBlocks * 8, (r1 - r0 + 7) / 8);
  k_compact_rows<<<grid, 256, 0, s>>>(r0, r1, rp, base, ci, v, sym ? 1 : 0, Lb, out_rp, out_ci, out_v);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

}  // namespace sexpm
