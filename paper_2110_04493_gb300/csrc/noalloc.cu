// sexpm_filter_noalloc: Algorithm 4.1 and the compaction of the kept entries on a
// caller-owned device CSR, writing into caller-owned output arrays, without allocating
// any memory.
//
// Some callers cannot allocate device memory at the moment they need the filter: a
// framework may have reserved all of the GPU's memory for its own allocator up front,
// or the caller runs under a fixed memory budget where a cudaMalloc (or a pool growth)
// could fail or stall.  This entry point serves them: its scratch space (per-row kept
// counts, per-block partial sums, scan tile sums and a validation flag) lives in one
// file-scope __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that first
// call before any stream capture.  The address is cached for the life of the process:
// after a cudaDeviceReset the cache is stale, so a caller that resets a device must not
// call this entry point on that device again.  `stream` must belong to the current
// device (checked).  Every call shares the array, so calls that overlap on the GPU
// (different streams, different host threads) race on it and must be serialised by the
// caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>

#include "sexpm_internal.cuh"

namespace sexpm_noalloc {
namespace {

// |v| > t for finite v and t >= 0, decided on the bit patterns: non-negative doubles are
// ordered as their bit patterns read as unsigned integers, so the test takes no FP64
// instruction (the FP64 pipe is this GPU's scarce unit; the dropped sum of squares keeps it).
__device__ __forceinline__ bool above(double v, unsigned long long tb) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) > tb;
}
__device__ __forceinline__ unsigned long long bits_of(double t) { return (unsigned long long)__double_as_longlong(t); }

constexpr unsigned FULL = 0xffffffffu;
constexpr int64_t kMaxRows = SEXPM_NOALLOC_MAX_ROWS;
constexpr int kBlocks = 1024;      // fixed reduction grid: sums do not depend on timing
constexpr int kThreads = 256;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int64_t kMaxTiles = (kMaxRows + kScanTile - 1) / kScanTile;

// Scratch layout (bytes): kept counts | block partials | tile sums | total | flag.
constexpr size_t kOffKeep = 0;
constexpr size_t kOffPart = kOffKeep + sizeof(int32_t) * kMaxRows;
constexpr size_t kOffTile = kOffPart + sizeof(double) * (kBlocks + 1);
constexpr size_t kOffFlag = kOffTile + sizeof(int64_t) * (kMaxTiles + 1);
constexpr size_t kScratchBytes = kOffFlag + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct View {
  int64_t n, nnz;
  const int64_t* rp;
  const int32_t* ci;
  const double* v;
};

__device__ __forceinline__ int lane() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T wsum(T x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

template <typename T>
__device__ T bsum(T x, T* red) {
  x = wsum(x);
  __syncthreads();
  if (lane() == 0) red[warp()] = x;
  __syncthreads();
  T t = lane() < (int)(blockDim.x >> 5) ? red[lane()] : T(0);
  return wsum(t);
}

// Row pointers monotone and in range, columns sorted, unique and in range, values finite.
__global__ void k_check(View A, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t p0 = A.rp[i], p1 = A.rp[i + 1];
  if ((i == 0 && p0 != 0) || (i == A.n - 1 && p1 != A.nnz) || p0 < 0 || p1 < p0 || p1 > A.nnz) {
    atomicOr(flag, 1);
    return;
  }
  int prev = -1;
  for (int64_t p = p0; p < p1; ++p) {
    const int c = A.ci[p];
    if (c <= prev || c >= A.n || !isfinite(A.v[p])) atomicOr(flag, 1);
    prev = c;
  }
}

// One pass: per-block partial sums of v^2 over |v| <= t, and keep[i] = #{|v| > t}.
__global__ void k_pass(View A, double t, int32_t* keep, double* part) {
  __shared__ double red[32];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  double s = 0.0;
  const unsigned long long tb = bits_of(t);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp(); i < A.n; i += nw) {
    int c = 0;
    for (int64_t q = A.rp[i] + lane(); q < A.rp[i + 1]; q += 32) {
      const double x = A.v[q];
      if (above(x, tb)) ++c; else s = fma(x, x, s);
    }
    c = wsum(c);
    if (lane() == 0) keep[i] = c;
  }
  s = bsum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_total(const double* part, int m, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  s = bsum(s, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_tiles(const int32_t* cnt, int64_t n, int64_t* tile) {
  __shared__ long long red[32];
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = (int64_t)blockIdx.x * kScanTile + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += cnt[i];
  }
  s = bsum(s, red);
  if (threadIdx.x == 0) tile[blockIdx.x] = s;
}

__global__ void k_tile_scan(int64_t* tile, int64_t m) {
  // single thread: at most kMaxTiles + 1 entries; the last receives the total
  if (threadIdx.x != 0) return;
  long long run = 0;
  for (int64_t k = 0; k < m; ++k) {
    const long long v = tile[k];
    tile[k] = run;
    run += v;
  }
  tile[m] = run;
}

__global__ void k_rows(const int32_t* cnt, int64_t n, const int64_t* tile, int64_t* rp) {
  __shared__ long long ws[32];
  const int64_t i0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  long long loc[kScanItems];
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = i0 + k < n ? cnt[i0 + k] : 0;
    s += loc[k];
  }
  long long incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(FULL, incl, o);
    if (lane() >= o) incl += y;
  }
  if (lane() == 31) ws[warp()] = incl;
  __syncthreads();
  if (warp() == 0) {
    const int nw = blockDim.x >> 5;
    const long long w = lane() < nw ? ws[lane()] : 0;
    long long wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(FULL, wi, o);
      if (lane() >= o) wi += y;
    }
    if (lane() < nw) ws[lane()] = wi - w;
  }
  __syncthreads();
  long long run = tile[blockIdx.x] + ws[warp()] + incl - s;
  for (int k = 0; k < kScanItems; ++k) {
    run += loc[k];
    if (i0 + k < n) rp[i0 + k + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rp[0] = 0;
}

__global__ void k_keep(View A, double t, const int64_t* rp, int32_t* ci, double* v) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lt = (1u << lane()) - 1u;
  const unsigned long long tb = bits_of(t);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp(); i < A.n; i += nw) {
    int64_t o = rp[i];
    for (int64_t qb = A.rp[i]; qb < A.rp[i + 1]; qb += 32) {
      const int64_t q = qb + lane();
      const bool act = q < A.rp[i + 1];
      const double x = act ? A.v[q] : 0.0;
      const bool k = act && above(x, tb);
      const unsigned m = __ballot_sync(FULL, k);
      if (k) {
        const int64_t d = o + __popc(m & lt);
        ci[d] = A.ci[q];
        v[d] = x;
      }
      o += __popc(m);
    }
  }
}

std::mutex g_mu;
unsigned char* g_addr[64] = {};

// Failures are reported through the library's sexpm_last_error().
int err(int code, const std::string& m) {
  sexpm::set_last_error(m);
  return code;
}

// Device address of the scratch array for the current device (looked up once per device).
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(SEXPM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return err(SEXPM_ECUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return err(SEXPM_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return SEXPM_OK;
}

#define NA_CUDA(x)                                                                          \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess) return err(SEXPM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int run(const sexpm_csr_view* A, double eps_g, double e_r, int32_t max_iters, void* stream, int64_t* out_row_ptr,
        int32_t* out_col, double* out_val, int64_t out_capacity, int64_t* nnz_out, double* t_out, int32_t* iters_out,
        double* b_out) {
  if (!A || !out_row_ptr || !nnz_out) return err(SEXPM_EINVAL, "null argument");
  if (!A->on_device) return err(SEXPM_EINVAL, "the no-allocation filter takes device arrays only (on_device = 1)");
  if (A->n < 0 || A->nnz < 0) return err(SEXPM_EINVAL, "negative dimensions");
  if (A->n > kMaxRows)
    return err(SEXPM_EOVERFLOW, "matrix has " + std::to_string(A->n) + " rows; the no-allocation filter's scratch holds at most " +
                                    std::to_string(kMaxRows) + " (SEXPM_NOALLOC_MAX_ROWS)");
  if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return err(SEXPM_EINVAL, "null CSR array");
  if (out_capacity < 0 || (out_capacity > 0 && (!out_col || !out_val))) return err(SEXPM_EINVAL, "bad output arrays");
  if (!(eps_g >= 0.0) || !std::isfinite(eps_g) || !(e_r > 0.0) || !std::isfinite(e_r) || max_iters < 1)
    return err(SEXPM_EINVAL, "bad filter parameters");
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != SEXPM_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    // the cached scratch address is the current device's: the stream must run there too
    int dev = 0, sdev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    NA_CUDA(cudaStreamGetDevice(s, &sdev));
    if (sdev != dev)
      return err(SEXPM_EINVAL, "the stream belongs to device " + std::to_string(sdev) + ", the current device is " +
                                   std::to_string(dev));
  }
  const View V{A->n, A->nnz, A->row_ptr, A->col, A->val};
  int32_t* keep = reinterpret_cast<int32_t*>(base + kOffKeep);
  double* part = reinterpret_cast<double*>(base + kOffPart);
  int64_t* tile = reinterpret_cast<int64_t*>(base + kOffTile);
  int* flag = reinterpret_cast<int*>(base + kOffFlag);
  const int64_t n = A->n;
  if (n == 0) {
    NA_CUDA(cudaMemsetAsync(out_row_ptr, 0, sizeof(int64_t), s));
    NA_CUDA(cudaStreamSynchronize(s));
    *nnz_out = 0;
    if (t_out) *t_out = eps_g;
    if (iters_out) *iters_out = 1;
    if (b_out) *b_out = 0.0;
    sexpm::set_last_error("");
    return SEXPM_OK;
  }
  // the validation flag must start at zero; every other scratch word is overwritten before use
  NA_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  k_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, flag);
  NA_CUDA(cudaGetLastError());
  int hflag = 0;
  NA_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  if (hflag) return err(SEXPM_EINVAL, "invalid device CSR (row_ptr, column order/range or non-finite value)");
  // Algorithm 4.1: t = eps_g / m, b = ||{|v| <= t}||_F, m = b / t, until b <= eps_g (1 + e_r)
  double m = 1.0, b = std::numeric_limits<double>::infinity(), eps_f = eps_g;
  int it = 0;
  while (b > eps_g * (1.0 + e_r)) {
    if (it >= max_iters) return err(SEXPM_ENOCONV, "Algorithm 4.1 did not converge within " + std::to_string(max_iters) + " passes");
    eps_f = eps_g / m;
    k_pass<<<kBlocks, kThreads, 0, s>>>(V, eps_f, keep, part);
    k_total<<<1, 1024, 0, s>>>(part, kBlocks, part + kBlocks);
    NA_CUDA(cudaGetLastError());
    double sum = 0.0;
    NA_CUDA(cudaMemcpyAsync(&sum, part + kBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    b = std::sqrt(sum);
    m = b / eps_f;
    ++it;
  }
  // kept total first (tile sums and their scan live in the scratch array), so that nothing of
  // the caller's outputs is written when they are too small; then row pointers and compaction
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  k_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(keep, n, tile);
  k_tile_scan<<<1, 32, 0, s>>>(tile, tiles);
  NA_CUDA(cudaGetLastError());
  int64_t kept = 0;
  NA_CUDA(cudaMemcpyAsync(&kept, tile + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  if (kept > out_capacity)
    return err(SEXPM_EOVERFLOW, "kept " + std::to_string(kept) + " entries but the output holds " + std::to_string(out_capacity));
  k_rows<<<(unsigned)tiles, kScanThreads, 0, s>>>(keep, n, tile, out_row_ptr);
  NA_CUDA(cudaGetLastError());
  if (kept > 0) {
    k_keep<<<kBlocks, kThreads, 0, s>>>(V, eps_f, out_row_ptr, out_col, out_val);
    NA_CUDA(cudaGetLastError());
  }
  NA_CUDA(cudaStreamSynchronize(s));
  *nnz_out = kept;
  if (t_out) *t_out = eps_f;
  if (iters_out) *iters_out = it;
  if (b_out) *b_out = b;
  sexpm::set_last_error("");
  return SEXPM_OK;
}

}  // namespace
}  // namespace sexpm_noalloc

extern "C" int sexpm_filter_noalloc(const sexpm_csr_view* A, double eps_g, double e_r, int32_t max_iters, void* stream,
                                    int64_t* out_row_ptr, int32_t* out_col, double* out_val, int64_t out_capacity,
                                    int64_t* nnz_out, double* t, int32_t* iters, double* b) {
  return sexpm_noalloc::run(A, eps_g, e_r, max_iters, stream, out_row_ptr, out_col, out_val, out_capacity, nnz_out, t,
                            iters, b);
}
