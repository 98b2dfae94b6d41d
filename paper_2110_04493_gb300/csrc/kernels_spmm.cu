// Sparse times dense block of vectors, Y = A X (X: n x r, row-major), and the time stepping
// U_{k+1} = E U_k with a computed E = e^{tau H} (Eq. 2.2: the propagator of a linear system
// with a fixed step is applied once per step).
//
// One warp per row, persistent grid.  The lanes stream the row's entries 32 at a time
// (coalesced column and value loads); each lane multiplies its entry by the row X_k of the
// block, which it loads as 16-byte pairs, and keeps R_CHUNK running sums; the warp then adds
// its lanes' sums (butterfly) and writes the R_CHUNK outputs of the row.  Blocks wider than
// R_CHUNK vectors are done R_CHUNK columns at a time.  Bound by HBM bandwidth: 12 bytes of A
// per entry, the rows of X come mostly from L2 (banded matrices read nearby rows of X).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sexpm_internal.cuh"

namespace sexpm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int R_CHUNK = 8;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// Y[:, c0 .. c0 + RC) = A X[:, c0 .. c0 + RC) for RC <= R_CHUNK columns (RC compile-time).
template <int RC>
__global__ void __launch_bounds__(256) k_spmm(CsrD A, const double* __restrict__ X, int64_t ldx,
                                              double* __restrict__ Y, int64_t ldy, int64_t c0) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const bool vec = (RC % 2 == 0) && ((ldx & 1) == 0) && ((c0 & 1) == 0) &&
                   ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.n; i += nw) {
    double acc[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[c] = 0.0;
    const int64_t p1 = A.rp[i + 1];
    for (int64_t p = A.rp[i] + lane_id(); p < p1; p += 32) {
      const int64_t k = __ldg(A.ci + p);
      const double a = __ldg(A.v + p);
      const double* xr = X + k * ldx + c0;
      if (vec) {
#pragma unroll
        for (int c = 0; c < RC; c += 2) {
          const double2 x = __ldg(reinterpret_cast<const double2*>(xr + c));
          acc[c] = fma(a, x.x, acc[c]);
          acc[c + 1] = fma(a, x.y, acc[c + 1]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[c] = fma(a, __ldg(xr + c), acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < RC; ++c)
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(FULL, acc[c], o);
    if (lane_id() < RC) {
      double out = acc[0];
#pragma unroll
      for (int c = 1; c < RC; ++c)
        if (lane_id() == c) out = acc[c];
      Y[i * ldy + c0 + lane_id()] = out;
    }
  }
}

int sm_count_spmm() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    SX_CUDA(cudaGetDevice(&dev));
    SX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

template <int RC>
void launch(const CsrD& A, const double* X, int64_t r, double* Y, int64_t c0, cudaStream_t s) {
  const int64_t grid = std::min<int64_t>((A.n + 7) / 8, (int64_t)sm_count_spmm() * 16);
  k_spmm<RC><<<(unsigned)grid, 256, 0, s>>>(A, X, r, Y, r, c0);
  SX_CUDA(cudaGetLastError());
  count_launches(1);
}

}  // namespace

void spmm(const CsrD& A, const double* X, int64_t r, double* Y, cudaStream_t s) {
  if (A.n == 0 || r == 0) return;
  for (int64_t c0 = 0; c0 < r; c0 += R_CHUNK) {
    switch ((int)std::min<int64_t>(R_CHUNK, r - c0)) {
      case 1: launch<1>(A, X, r, Y, c0, s); break;
      case 2: launch<2>(A, X, r, Y, c0, s); break;
      case 3: launch<3>(A, X, r, Y, c0, s); break;
      case 4: launch<4>(A, X, r, Y, c0, s); break;
      case 5: launch<5>(A, X, r, Y, c0, s); break;
      case 6: launch<6>(A, X, r, Y, c0, s); break;
      case 7: launch<7>(A, X, r, Y, c0, s); break;
      default: launch<8>(A, X, r, Y, c0, s); break;
    }
  }
}

}  // namespace sexpm
