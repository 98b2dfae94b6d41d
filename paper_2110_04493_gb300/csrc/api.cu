// C ABI and host driver of Algorithm 4.2 (filtered incremental scaling and squaring).
//
// The driver runs on the host and sequences device kernels on one stream:
//   step 1  ||tau H||_F (device reduction) and (M, N) by Eq. (4.20) on the host;
//   step 2  a = 1/(N+1) for normal H, else 1/||H||_F;
//   step 3  H_0 = tau H 2^-N, the filtered Taylor terms S^_i of Eq. (4.11), T^_0 = sum S^_i;
//   step 4  N squarings T~_i = 2 T^_{i-1} + T^_{i-1}^2, each filtered by Algorithm 4.1;
//   step 5  e^{tau H} = I + T^_N.
// Algorithm 4.1 is a host loop over device reduction passes: each pass returns one
// scalar (the F-norm of the candidate dropped part) and the next eps_f is computed on
// the host exactly as the algorithm states.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sexpm_internal.cuh"

namespace sexpm {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  cudaGetLastError();  // clear a sticky launch error where possible
  if (e == cudaErrorMemoryAllocation) fail(SEXPM_ENOMEM, std::string("out of device memory in ") + what);
  fail(SEXPM_ECUDA, std::string(cudaGetErrorString(e)) + " in " + what);
}

// ---------------------------------------------------------------- pool
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
std::atomic<int64_t> g_live{0}, g_peak{0};

cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(SEXPM_ECUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    SX_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
    uint64_t thr = std::numeric_limits<uint64_t>::max();
    SX_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr));
  }
  return g_pools[dev];
}
}  // namespace

// Host-side failure injection for tests of the error paths: when SEXPM_FAIL_ALLOC_AT=k is set
// in the environment, the k-th pool allocation of every sexpm_compute fails as if the device
// were out of memory (no device call is made for it).
std::atomic<int64_t> g_fail_countdown{0};

void arm_alloc_failure() {
  const char* e = std::getenv("SEXPM_FAIL_ALLOC_AT");
  g_fail_countdown.store(e && *e ? std::max<int64_t>(0, std::strtoll(e, nullptr, 10)) : 0);
}

void* Pool::alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (g_fail_countdown.load() > 0 && g_fail_countdown.fetch_sub(1) == 1)
    fail(SEXPM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected by SEXPM_FAIL_ALLOC_AT)");
  cudaMemPool_t pool = pool_for_current_device();
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
  if (e == cudaErrorMemoryAllocation) {
    // the pool keeps freed blocks (its release threshold is unbounded); blocks of other sizes may
    // be what is missing: return them to the device and try once more
    cudaGetLastError();
    SX_CUDA(cudaDeviceSynchronize());
    SX_CUDA(cudaMemPoolTrimTo(pool, 0));
    e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? SEXPM_ENOMEM : SEXPM_ECUDA,
         "device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  const int64_t now = g_live.fetch_add((int64_t)bytes) + (int64_t)bytes;
  int64_t pk = g_peak.load();
  while (now > pk && !g_peak.compare_exchange_weak(pk, now)) {
  }
  return p;
}

void Pool::release(void* p, size_t bytes, cudaStream_t s) {
  cudaFreeAsync(p, s);
  g_live.fetch_sub((int64_t)bytes);
}

int current_device() {
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(SEXPM_ECUDA, "device ordinal out of range");
  return dev;
}

std::mutex& device_setup_mutex() {
  static std::mutex mu;
  return mu;
}

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k); }
int64_t launches() { return g_launches.load(); }

int64_t Pool::live() { return g_live.load(); }
int64_t Pool::peak() { return g_peak.load(); }
void Pool::reset_peak() { g_peak.store(g_live.load()); }

// ---------------------------------------------------------------- helpers
namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    SX_CUDA(cudaEventCreate(&a));
    SX_CUDA(cudaEventCreate(&b));
    SX_CUDA(cudaEventRecord(a, s));
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  double ms() {
    SX_CUDA(cudaEventRecord(b, s));
    SX_CUDA(cudaEventSynchronize(b));
    float m = 0.f;
    SX_CUDA(cudaEventElapsedTime(&m, a, b));
    return m;
  }
};

void validate_host_csr(const sexpm_csr_view& H) {
  if (H.n < 0 || H.nnz < 0 || H.n > INT32_MAX) fail(SEXPM_EINVAL, "bad dimensions");
  if (H.n > 0 && (!H.row_ptr || (H.nnz > 0 && (!H.col || !H.val)))) fail(SEXPM_EINVAL, "null CSR array");
  if (H.n == 0) return;
  if (H.row_ptr[0] != 0 || H.row_ptr[H.n] != H.nnz) fail(SEXPM_EINVAL, "row_ptr must start at 0 and end at nnz");
  for (int64_t i = 0; i < H.n; ++i) {
    const int64_t p0 = H.row_ptr[i], p1 = H.row_ptr[i + 1];
    if (p1 < p0 || p1 > H.nnz) fail(SEXPM_EINVAL, "row_ptr not monotone at row " + std::to_string(i));
    int32_t prev = -1;
    for (int64_t p = p0; p < p1; ++p) {
      const int32_t c = H.col[p];
      if (c <= prev || c >= H.n) fail(SEXPM_EINVAL, "columns unsorted, duplicated or out of range in row " + std::to_string(i));
      if (!std::isfinite(H.val[p])) fail(SEXPM_EINVAL, "non-finite value in row " + std::to_string(i));
      prev = c;
    }
  }
}

// Copy a borrowed view (host or device) into an owned device CSR.
void upload(const sexpm_csr_view& V, cudaStream_t s, CsrOwned& out, HostScalars& hs) {
  if (!V.on_device) validate_host_csr(V);
  out.n = V.n;
  out.nnz = V.nnz;
  out.rp.reset(V.n + 1, s);
  out.ci.reset(V.nnz, s);
  out.v.reset(V.nnz, s);
  const cudaMemcpyKind k = V.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (V.n >= 0 && V.row_ptr) SX_CUDA(cudaMemcpyAsync(out.rp.p, V.row_ptr, (V.n + 1) * sizeof(int64_t), k, s));
  if (V.nnz) {
    SX_CUDA(cudaMemcpyAsync(out.ci.p, V.col, V.nnz * sizeof(int32_t), k, s));
    SX_CUDA(cudaMemcpyAsync(out.v.p, V.val, V.nnz * sizeof(double), k, s));
  }
  if (V.on_device) {
    if (V.n < 0 || V.nnz < 0 || V.n > INT32_MAX) fail(SEXPM_EINVAL, "bad dimensions");
    if (!csr_valid(out.view(), s, hs)) fail(SEXPM_EINVAL, "invalid device CSR (row_ptr, column order/range or non-finite value)");
  }
}

struct FilterOut {
  double t = 0.0, b = 0.0;
  int iters = 0;
  double ms = 0.0;
  double bytes = 0.0;
};

// Algorithm 4.1 on the stored values of the row pieces P (together rows 0..n-1, in order), then
// A~ = A - b_n into `out`.  `extra` is the sum of squares of entries dropped before (by the exact
// streaming bound, below every threshold the algorithm visits): it joins every pass's sum.
// Each pass streams the values once and records kept counts per (tile, warp); the compaction
// after the last pass uses the counts of that pass.
FilterOut filter_alg41_pieces(const std::vector<Piece>& P, int64_t n, double extra, double eps_g, double e_r,
                              int max_iters, cudaStream_t s, CsrOwned& out, HostScalars& hs) {
  FilterOut r;
  Timer tf(s);
  std::vector<int64_t> tile_base(P.size() + 1, 0);
  int64_t nnz_all = 0;
  for (size_t p = 0; p < P.size(); ++p) {
    tile_base[p + 1] = tile_base[p] + counts_of(P[p].nnz);
    nnz_all += P[p].nnz;
  }
  const int64_t T = tile_base.back();
  DevBuf<int32_t> tcnt(T ? T : 1, s);
  double m = 1.0;
  double b = std::numeric_limits<double>::infinity();  // the first pass always runs
  double eps_f = eps_g;
  int it = 0;
  while (b > eps_g * (1.0 + e_r)) {
    if (it >= max_iters) fail(SEXPM_ENOCONV, "Algorithm 4.1 did not converge within " + std::to_string(max_iters) + " passes");
    eps_f = eps_g / m;
    b = std::sqrt(pass_pieces(P, tile_base, eps_f, tcnt.p, s, hs) + extra);
    m = b / eps_f;
    ++it;
  }
  out.n = n;
  out.rp.reset(n + 1, s);
  DevBuf<int64_t> toff(T + 1, s);
  out.nnz = scan_counts(tcnt.p, T, toff.p, s, hs);
  out.ci.reset(out.nnz, s);
  out.v.reset(out.nnz, s);
  if (n == 0) SX_CUDA(cudaMemsetAsync(out.rp.p, 0, sizeof(int64_t), s));
  else compact_pieces(P, tile_base, eps_f, toff.p, n, out, s);
  r.t = eps_f;
  r.b = b;
  r.iters = it;
  r.ms = tf.ms();
  r.bytes = it * 8.0 * nnz_all + 12.0 * nnz_all + 12.0 * out.nnz + 16.0 * ((double)n + 1.0);
  return r;
}

// Algorithm 4.1 on one whole matrix.
FilterOut filter_alg41(const CsrD& A, double eps_g, double e_r, int max_iters, cudaStream_t s, CsrOwned& out,
                       HostScalars& hs) {
  Piece p;
  p.r0 = 0;
  p.r1 = A.n;
  p.nnz = A.nnz;
  p.rp = A.rp;
  p.ci = A.ci;
  p.v = A.v;
  return filter_alg41_pieces(std::vector<Piece>{p}, A.n, 0.0, eps_g, e_r, max_iters, s, out, hs);
}

void copy_csr(const CsrD& A, cudaStream_t s, CsrOwned& out) {
  out.n = A.n;
  out.nnz = A.nnz;
  out.rp.reset(A.n + 1, s);
  out.ci.reset(A.nnz, s);
  out.v.reset(A.nnz, s);
  SX_CUDA(cudaMemcpyAsync(out.rp.p, A.rp, (A.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (A.nnz) {
    SX_CUDA(cudaMemcpyAsync(out.ci.p, A.ci, A.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    SX_CUDA(cudaMemcpyAsync(out.v.p, A.v, A.nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
}

// Row schedule for cache locality.  When H looks like a stencil on a grid numbered
// x + m y (+ m^2 z) -- most rows store the offsets +-1 and +-m -- the products hand rows to
// the thread blocks in strips of kStrip consecutive x: all y (and z) of one strip before the
// next.  Rows processed together then read the B rows of a band about kStrip + (stencil
// radius) wide instead of whole grid lines, which keeps the B operand resident in L2.
// Returns the detected stride m (0 if none) and fills sched.
constexpr int kStrip = 32;
int64_t grid_schedule(const CsrOwned& H, cudaStream_t s, DevBuf<int32_t>& sched) {
  const int64_t n = H.n;
  if (n < 4 * kStrip * kStrip) return 0;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(H.nnz);
  SX_CUDA(cudaMemcpyAsync(rp.data(), H.rp.p, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (H.nnz) SX_CUDA(cudaMemcpyAsync(ci.data(), H.ci.p, H.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SX_CUDA(cudaStreamSynchronize(s));
  // most frequent offset > 1 among the entries above the diagonal
  std::map<int64_t, int64_t> freq;
  const int64_t step = std::max<int64_t>(1, n / 20000);
  int64_t sampled = 0;
  for (int64_t i = 0; i < n; i += step, ++sampled)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t d = (int64_t)ci[p] - i;
      if (d > 1) ++freq[d];
    }
  int64_t m = 0, best = 0;
  for (const auto& kv : freq)
    if (kv.second > best) { best = kv.second; m = kv.first; }
  if (m < 2 * kStrip || best < sampled / 2) return 0;
  // most sampled rows must also hold +1 (a grid line), else this is not a grid numbering
  int64_t ones = 0;
  for (int64_t i = 0; i < n; i += step)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if ((int64_t)ci[p] == i + 1) { ++ones; break; }
  if (ones < sampled / 2) return 0;
  std::vector<int32_t> order;
  order.reserve(n);
  const int64_t lines = (n + m - 1) / m;
  for (int64_t x0 = 0; x0 < m; x0 += kStrip)
    for (int64_t y = 0; y < lines; ++y)
      for (int64_t x = x0; x < std::min<int64_t>(x0 + kStrip, m); ++x) {
        const int64_t i = x + m * y;
        if (i < n) order.push_back((int32_t)i);
      }
  sched.reset(n, s);
  SX_CUDA(cudaMemcpyAsync(sched.p, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  SX_CUDA(cudaStreamSynchronize(s));
  return m;
}

// Algorithm 4.2 step 2: exact symmetry, and normality (H = H^T or H = -H^T exactly, else
// ||H H^T - H^T H||_F <= 64 u ||H||_F^2), unless overridden.
// normal_scale: the bound 64 u ||H||_F^2 is multiplied by it (1/sqrt(2) for the real embedding of
// a complex matrix, whose commutator and squared norm are sqrt(2) and 2 times the complex ones).
void classify_matrix(const CsrOwned& H, int normal_override, cudaStream_t s, HostScalars& hs, bool& symmetric,
                     int& normal, double normal_scale = 1.0) {
  CsrOwned Ht;
  transpose(H.view(), s, Ht, hs);
  symmetric = csr_equal(H.view(), Ht.view(), 1.0, s, hs);
  if (normal_override >= 0) {
    normal = normal_override;
  } else if (symmetric || csr_equal(H.view(), Ht.view(), -1.0, s, hs)) {
    normal = 1;
  } else {
    CsrOwned P, Q, C;
    CsrD none;
    spgemm(H.view(), Ht.view(), none, 1.0, 0.0, s, P, nullptr, hs);
    spgemm(Ht.view(), H.view(), none, 1.0, 0.0, s, Q, nullptr, hs);
    add(P.view(), Q.view(), -1.0, s, C, hs);
    const double nc = std::sqrt(sum_squares(C.view(), s, hs));
    const double nh2 = sum_squares(H.view(), s, hs);
    normal = nc <= 64.0 * std::ldexp(1.0, -53) * nh2 * normal_scale ? 1 : 0;
  }
}

struct SegFilterOut {
  std::vector<double> t, b;
  std::vector<int> iters;
  double ms = 0.0;
};

// Algorithm 4.1 run independently for every instance of a block-diagonal matrix: instance b
// uses bound eps_g[b]; instances with fixed[b] >= 0 are not iterated and use t = fixed[b]
// (0 keeps every nonzero entry, +inf drops every entry).  One device pass serves all
// unconverged instances; then A~ = A - b_n into `out`.
SegFilterOut filter_seg(const CsrD& A, const std::vector<double>& eps_g, const std::vector<double>& fixed, double e_r,
                        int max_iters, const int32_t* inst, const int64_t* seg, int count, cudaStream_t s,
                        CsrOwned& out, HostScalars& hs) {
  SegFilterOut r;
  Timer tf(s);
  r.t.assign(count, 0.0);
  r.b.assign(count, 0.0);
  r.iters.assign(count, 0);
  std::vector<double> m(count, 1.0), sums(count, 0.0);
  std::vector<char> conv(count, 0);
  for (int k = 0; k < count; ++k) {
    if (fixed[k] >= 0.0) {
      conv[k] = 1;
      r.t[k] = fixed[k];
    } else {
      r.t[k] = eps_g[k];
      r.b[k] = std::numeric_limits<double>::infinity();
    }
  }
  DevBuf<int32_t> keep(A.n ? A.n : 1, s);
  DevBuf<double> part(A.n ? A.n : 1, s), tdev(count, s);
  while (true) {
    for (int k = 0; k < count; ++k)
      if (!conv[k]) r.t[k] = eps_g[k] / m[k];
    SX_CUDA(cudaMemcpyAsync(tdev.p, r.t.data(), count * sizeof(double), cudaMemcpyHostToDevice, s));
    filter_pass_seg(A, inst, tdev.p, keep.p, part.p, seg, count, sums.data(), s);
    bool all = true;
    for (int k = 0; k < count; ++k) {
      if (conv[k]) continue;
      r.b[k] = std::sqrt(sums[k]);
      m[k] = r.b[k] / r.t[k];
      ++r.iters[k];
      if (r.b[k] <= eps_g[k] * (1.0 + e_r)) {
        conv[k] = 1;
      } else {
        all = false;
        if (r.iters[k] >= max_iters)
          fail(SEXPM_ENOCONV, "Algorithm 4.1 did not converge within " + std::to_string(max_iters) +
                                  " passes (instance " + std::to_string(k) + ")");
      }
    }
    if (all) break;
  }
  out.n = A.n;
  out.rp.reset(A.n + 1, s);
  out.nnz = scan_counts(keep.p, A.n, out.rp.p, s, hs);
  out.ci.reset(out.nnz, s);
  out.v.reset(out.nnz, s);
  compact_seg(A, inst, tdev.p, out, s);
  r.ms = tf.ms();
  return r;
}

}  // namespace
}  // namespace sexpm

using namespace sexpm;

struct sexpm_plan {
  int device = 0;
  cudaStream_t s = nullptr;
  sexpm_options opt;
  double eps = 0.0;
  CsrOwned H;
  int normal = 1;
  bool symmetric = false;  // H == H^T exactly
  HostScalars hs;
  // batched plans (count > 0): H is block diagonal, instance b owns rows row0[b] .. row0[b+1]
  int32_t count = 0;
  std::vector<int64_t> row0;
  std::vector<int> normal_b;
  std::vector<char> symmetric_b;
  DevBuf<int64_t> seg;
  DevBuf<int32_t> inst;
  // row schedule of the sparse products (empty: natural order)
  DevBuf<int32_t> sched;
  int64_t grid_stride = 0;
  // complex plans: H holds the n top rows of the real embedding [X | -Y] (2n columns)
  bool cplx = false;
  // batched plans: the captured squaring step and its arena (made on the first compute)
  GraphSquaring* graph = nullptr;
  int32_t layout_ks = -1, layout_wide = -1;  // accumulation layout chosen by sexpm_tune_batched
  ~sexpm_plan() {
    if (graph) graph_squaring_free(graph);
  }
};

struct sexpm_result {
  cudaStream_t s = nullptr;
  CsrOwned E;                  // complex results: the pattern (E.v empty) and
  bool cplx = false;
  DevBuf<double> vz;           // the values, (re, im) pairs
  sexpm_stats_t st;
  std::vector<sexpm_step_stats> steps;
};

// ---------------------------------------------------------------- the method (Algorithm 4.2)

// What the reverse pass needs from a forward run: H_0, the kept Taylor terms S_1..S_M'
// (S_1 = H_0), and T^_k at the checkpoints k = 0, stride, 2 stride, ..., N, together with the
// scalars that let a squaring step be replayed bit for bit.
struct Record {
  int stride = 0;  // 0: ceil(sqrt(N))
  CsrOwned H0;
  std::vector<CsrOwned> S;
  std::map<int, CsrOwned> T;
  int M = 0, N = 0;
  double tau = 0.0, a = 0.0, r0 = 0.0;
};

// A forward run kept for its reverse pass (sexpm_forward_keep).  The plan is borrowed.
struct sexpm_tape {
  sexpm_plan_t* plan = nullptr;
  double tau = 0.0;
  Record rec;
  sexpm_stats_t st;
  std::vector<sexpm_step_stats> steps;
};

// Device bytes the library can still allocate: free device memory plus what its pool holds
// unused.
int64_t device_available_bytes() {
  size_t fr = 0, tot = 0;
  SX_CUDA(cudaMemGetInfo(&fr, &tot));
  uint64_t reserved = 0, used = 0;
  cudaMemPool_t pool = pool_for_current_device();
  SX_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  SX_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  return (int64_t)fr + (int64_t)(reserved > used ? reserved - used : 0);
}

// Bytes of the unfiltered product one chunk may hold, or 0 when the product is formed whole.
// Whole: the product T~ (12 B per entry) and, in the worst case, a filtered copy of the same
// size must fit, with T^_{k-1} released after the product.  Otherwise chunks of an eighth of
// what is free (at least 256 MB) leave room for the kept pieces and the result.
int64_t chunk_limit(const sexpm_options& o, int64_t raw_entries, int64_t in_bytes, bool releases_input) {
  const int64_t raw = 12 * raw_entries;
  if (o.chunk_bytes > 0) return raw > o.chunk_bytes ? o.chunk_bytes : 0;
  const int64_t avail = device_available_bytes();
  const int64_t margin = (int64_t)2 << 30;
  if (raw + margin <= avail && 2 * raw + margin <= avail + (releases_input ? in_bytes : 0)) return 0;
  return std::max<int64_t>(avail / 8, (int64_t)256 << 20);
}

// One filtered incremental squaring T^_k = filter(2 T^_{k-1} + T^_{k-1}^2) (Eq. 4.15 with the
// threshold of reading 8); deterministic, so a replay reproduces the forward exactly.  When
// drop_input is given (the owner of T), it is released as soon as the product has been formed
// (stream-ordered), so that T^_{k-1} is not held while the unfiltered T~_k is filtered.
//
// When T~_k does not fit in memory it is formed in chunks of consecutive rows.  Each chunk is
// reduced at once to its entries above L = eps_g' / (2 sqrt(nnz(T~_k))), where eps_g' <= eps_g
// is the bound from the rows formed so far (the norm ||I + T~_k||_F of reading 8 only grows as
// rows are added); every threshold Algorithm 4.1 visits is >= eps_g / sqrt(nnz), so the entries
// dropped here are dropped by every pass, and their sum of squares joins every pass's sum.  In
// the symmetric mode a pair (i, j), (j, i) is decided once, by the row that forms its upper
// entry; the lower entry takes that entry's value and decision.
void square_step(const sexpm_options& o, const CsrD& T, int k, double a, double r0, bool sym, cudaStream_t s,
                 HostScalars& hs, RowStats& rs, CsrOwned& Tn, sexpm_step_stats* rec, const int32_t* sched,
                 CsrOwned* drop_input = nullptr) {
  Timer ts(s);
  const int64_t n = T.n;
  const int64_t nnz_in = T.nnz;
  const double ri = std::ldexp(r0, k);
  double ms_sym = 0.0, ms_num = 0.0;
  ProductSym ps;
  {
    Timer t1(s);
    product_symbolic(T, T, T, sym, nullptr, sched, &rs, s, hs, ps);
    ms_sym = t1.ms();
  }
  const int64_t products = ps.products;
  const int64_t in_bytes = 12 * nnz_in + 8 * (n + 1);
  const int64_t limit = chunk_limit(o, ps.nnz, in_bytes, drop_input != nullptr);
  int64_t done = 0;
  int chunks = 1;
  int64_t rows_class[kProductClasses] = {};
  FilterOut fo;
  double normF = 1.0, eps_g = 0.0;
  int64_t nnz_raw = ps.nnz, nnz_stream = 0;
  double bytes_stream = 0.0;
  auto release_input = [&]() {
    if (drop_input) {
      drop_input->rp.free();
      drop_input->ci.free();
      drop_input->v.free();
    }
  };
  auto eps_from_stats = [&](int64_t r1, double& sq_acc, double& tr_acc, int64_t from) {
    // ||I + T~||_F^2 over the rows formed so far = sum sq + rows + 2 sum diag
    if (!o.square_scale) return a * ri;
    sq_acc += reduce_sum(rs.sq.p + from, r1 - from, s, hs);
    tr_acc += reduce_sum(rs.diag.p + from, r1 - from, s, hs);
    const double f2 = sq_acc + (double)r1 + 2.0 * tr_acc;
    normF = std::sqrt(f2 > 0.0 ? f2 : 0.0);
    return a * ri * normF;
  };
  if (limit == 0) {
    CsrOwned Tt;
    Tt.n = n;
    Tt.nnz = ps.nnz;
    Tt.rp = std::move(ps.rp);
    ps.rp_ext = Tt.rp.p;
    Tt.ci.reset(Tt.nnz, s);
    Tt.v.reset(Tt.nnz, s);
    {
      Timer t2(s);
      done = product_numeric(ps, T, T, T, 1.0, 2.0, 0, n, 0, Tt.ci.p, Tt.v.p, &rs, s, hs);
      if (sym) mirror_lower(Tt, s, hs);
      ms_num = t2.ms();
    }
    release_input();
    for (int c = 0; c < kProductClasses; ++c) rows_class[c] = ps.rows_numeric[c];
    double sq = 0.0, tr = 0.0;
    eps_g = eps_from_stats(n, sq, tr, 0);
    fo = filter_alg41(Tt.view(), eps_g, o.e_r, o.max_filter_iters, s, Tn, hs);
  } else {
    // row boundaries from the product's row pointers
    std::vector<int64_t> rph(n + 1);
    SX_CUDA(cudaMemcpyAsync(rph.data(), ps.row_ptr(), (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SX_CUDA(cudaStreamSynchronize(s));
    const int64_t per_chunk = std::max<int64_t>(1, limit / 12);
    struct Owned {
      DevBuf<int64_t> rp;
      DevBuf<int32_t> ci;
      DevBuf<double> v;
    };
    std::vector<Owned> owned;
    std::vector<Piece> pieces;
    DevBuf<Piece> dpieces;
    double sq_acc = 0.0, tr_acc = 0.0, dropped = 0.0;
    const double sqrt_nnz = std::sqrt((double)std::max<int64_t>(ps.nnz, 1));
    chunks = 0;
    double ms_drop = 0.0;
    for (int64_t c0 = 0; c0 < n;) {
      // the largest c1 with at most per_chunk entries in [c0, c1) (at least one row)
      int64_t c1 = std::upper_bound(rph.begin() + c0 + 1, rph.end(), rph[c0] + per_chunk) - rph.begin() - 1;
      if (c1 <= c0) c1 = c0 + 1;
      const int64_t base = rph[c0], cn = rph[c1] - base;
      DevBuf<int32_t> cci(cn, s);
      DevBuf<double> cv(cn, s);
      {
        Timer t2(s);
        done += product_numeric(ps, T, T, T, 1.0, 2.0, c0, c1, base, cci.p, cv.p, &rs, s, hs);
        ms_num += t2.ms();
      }
      Timer t3(s);
      const double eps_c = eps_from_stats(c1, sq_acc, tr_acc, c0);
      const double L = 0.5 * eps_c / sqrt_nnz;
      if (!pieces.empty()) {
        dpieces.reset(pieces.size(), s);
        SX_CUDA(cudaMemcpyAsync(dpieces.p, pieces.data(), pieces.size() * sizeof(Piece), cudaMemcpyHostToDevice, s));
      }
      DevBuf<int32_t> keep(c1 - c0, s);
      dropped += drop_rows(c0, c1, ps.row_ptr(), base, cci.p, cv.p, sym, L, dpieces.p, (int)pieces.size(), keep.p, s,
                           hs);
      Owned ow;
      ow.rp.reset(c1 - c0 + 1, s);
      const int64_t kept = scan_counts(keep.p, c1 - c0, ow.rp.p, s, hs);
      ow.ci.reset(kept, s);
      ow.v.reset(kept, s);
      compact_rows(c0, c1, ps.row_ptr(), base, cci.p, cv.p, sym, L, ow.rp.p, ow.ci.p, ow.v.p, s);
      Piece pc;
      pc.r0 = c0;
      pc.r1 = c1;
      pc.nnz = kept;
      pc.rp = ow.rp.p;
      pc.ci = ow.ci.p;
      pc.v = ow.v.p;
      pieces.push_back(pc);
      owned.push_back(std::move(ow));
      nnz_stream += kept;
      bytes_stream += 24.0 * (double)cn + 12.0 * (double)kept + 24.0 * (double)(c1 - c0);
      ms_drop += t3.ms();
      ++chunks;
      c0 = c1;
    }
    release_input();
    for (int c = 0; c < kProductClasses; ++c) rows_class[c] = ps.rows_numeric[c];
    ps = ProductSym();  // word patterns and row lists are no longer needed
    dpieces.free();
    eps_g = o.square_scale ? a * ri * normF : a * ri;  // normF now covers every row
    fo = filter_alg41_pieces(pieces, n, dropped, eps_g, o.e_r, o.max_filter_iters, s, Tn, hs);
    fo.ms += ms_drop;
    fo.bytes += bytes_stream;
  }
  if (rec) {
    std::memset(rec, 0, sizeof(*rec));
    rec->phase = 1;
    rec->i = k;
    rec->iters = fo.iters;
    rec->chunks = chunks;
    rec->eps_g = eps_g;
    rec->t = fo.t;
    rec->b = fo.b;
    rec->norm_F = o.square_scale ? normF : 0.0;
    rec->nnz_raw = nnz_raw;
    rec->nnz = Tn.nnz;
    rec->nnz_stream = nnz_stream;
    rec->products = products;
    for (int c = 0; c < kProductClasses; ++c) rec->rows_class[c] = rows_class[c];
    rec->products_done = done;
    rec->ms_symbolic = ms_sym;
    rec->ms_numeric = ms_num;
    rec->ms_filter = fo.ms;
    rec->flops = 2.0 * (double)done + 2.0 * (double)nnz_in;
    rec->bytes_filter = fo.bytes;
    rec->ms = ts.ms();
  }
}

// ||H^k||_F for k = 1..kmax from exact sparse powers H^k = H^{k-1} H.
void power_norms(const CsrD& H, int kmax, cudaStream_t s, HostScalars& hs, double* out) {
  CsrOwned P;
  copy_csr(H, s, P);
  out[0] = std::sqrt(sum_squares(P.view(), s, hs));
  CsrD none;
  for (int k = 2; k <= kmax; ++k) {
    CsrOwned Q;
    spgemm(P.view(), H, none, 1.0, 0.0, s, Q, nullptr, hs);
    P = std::move(Q);
    out[k - 1] = std::sqrt(sum_squares(P.view(), s, hs));
  }
}

void compute_impl(sexpm_plan_t* p, double tau, sexpm_result* res, Record* record, bool allow_sym) {
  if (!std::isfinite(tau)) fail(SEXPM_EINVAL, "tau must be finite");
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) fail(SEXPM_EINVAL, "current device differs from the plan's device");
  cudaStream_t s = p->s;
  HostScalars& hs = p->hs;
  const sexpm_options& o = p->opt;
  const int64_t n = p->H.n;
  res->s = s;
  std::memset(&res->st, 0, sizeof(res->st));
  sexpm_stats_t& st = res->st;
  st.n = n;
  Pool::reset_peak();
  const int64_t live0 = Pool::live();
  const int64_t launches0 = launches();
  Timer t_all(s);
  // step 1: tau H and its F-norm, (M, N)
  CsrD Hs = p->H.view();
  DevBuf<double> hv(p->H.nnz, s);
  scale_values(p->H.v.p, tau, p->H.nnz, hv.p, s);
  Hs.v = hv.p;
  const double normH = std::sqrt(sum_squares(Hs, s, hs));
  st.norm_H = normH;
  int32_t M = 0, N = 0;
  std::vector<double> pnorms;
  if (o.scaling == 1 && normH > 0.0) {
    // the refined norm of Sec. 4.2: ||(tau H)^k||_F from exact sparse powers
    pnorms.resize(o.refine_kmax);
    power_norms(Hs, o.refine_kmax, s, hs, pnorms.data());
    const int rc = sexpm_choose_MN_refined(normH, pnorms.data(), o.refine_kmax, p->eps, o.n_extra, &M, &N);
    if (rc != SEXPM_OK) fail(rc, "no feasible (M, N) for this tolerance on the refined norm (raise refine_kmax)");
  } else {
    const int rc = sexpm_choose_MN(normH, p->eps, o.n_extra, o.max_taylor, &M, &N);
    if (rc != SEXPM_OK) fail(rc, rc == SEXPM_ENOPARAM ? "no feasible (M, N) for this tolerance" : "invalid (M, N) input");
  }
  st.M = M;
  st.N = N;
  const bool normal = (p->normal != 0) || normH == 0.0;
  st.normal = normal ? 1 : 0;
  const bool sym = p->symmetric && allow_sym;
  st.symmetric = sym ? 1 : 0;
  if (record) {
    record->M = M;
    record->N = N;
    record->tau = tau;
    if (record->stride <= 0) record->stride = std::max(1, (int)std::ceil(std::sqrt((double)N)));
  }
  if (M == 0) {
    // ||tau H|| = 0: e^0 = I
    CsrOwned Z;
    Z.n = n;
    Z.nnz = 0;
    Z.rp.reset(n + 1, s);
    SX_CUDA(cudaMemsetAsync(Z.rp.p, 0, (n + 1) * sizeof(int64_t), s));
    add_identity(Z.view(), s, res->E, hs);
    st.nnz_out = res->E.nnz;
    st.ms_total = t_all.ms();
    st.peak_bytes = Pool::peak() - live0;
    st.launches = launches() - launches0;
    return;
  }
  // step 2: filter parameter a
  const double a = normal ? 1.0 / (1.0 + N) : 1.0 / normH;
  st.a = a;
  // step 3: Taylor phase on H_0 = tau H 2^-N
  Timer t_tay(s);
  DevBuf<double> h0v(p->H.nnz, s);
  scale_values(hv.p, std::ldexp(1.0, -N), p->H.nnz, h0v.p, s);
  CsrD H0 = Hs;
  H0.v = h0v.p;
  // ||H_0|| of Eq. (4.5) and of the Taylor threshold; the refined norm h_{M,N} in the refined scaling
  const double x0 = pnorms.empty() ? std::ldexp(normH, -N) : h_refined(pnorms.data(), o.refine_kmax, M, N);
  const double r0 = sexpm_rho(M, x0);
  const double eps_g0 = a * r0 / ((double)M * std::exp(2.0 * x0));
  st.r0 = r0;
  st.eps_g0 = eps_g0;
  if (record) {
    record->a = a;
    record->r0 = r0;
    copy_csr(H0, s, record->H0);
    record->S.emplace_back();
    copy_csr(H0, s, record->S.back());
  }
  CsrOwned T;       // running T^_0, later T^_i
  copy_csr(H0, s, T);
  CsrOwned S;       // current filtered term (S_1 = H_0 is not filtered)
  CsrD Sv = H0;
  CsrD none;
  for (int i = 2; i <= M; ++i) {
    Timer ts(s);
    CsrOwned St;
    SpgemmTimes tm;
    int64_t done = 0;
    const int64_t prod = spgemm(Sv, H0, none, (double)i, 0.0, s, St, nullptr, hs, &tm, false, &done, nullptr,
                                p->sched.p);
    CsrOwned Sn;
    FilterOut fo = filter_alg41(St.view(), eps_g0, o.e_r, o.max_filter_iters, s, Sn, hs);
    sexpm_step_stats rec;
    std::memset(&rec, 0, sizeof(rec));
    rec.phase = 0;
    rec.i = i;
    rec.iters = fo.iters;
    rec.eps_g = eps_g0;
    rec.t = fo.t;
    rec.b = fo.b;
    rec.nnz_raw = St.nnz;
    rec.nnz = Sn.nnz;
    rec.products = prod;
    rec.ms_symbolic = tm.ms_symbolic;
    rec.ms_numeric = tm.ms_numeric;
    rec.ms_filter = fo.ms;
    rec.products_done = done;
    rec.flops = 2.0 * (double)done + (double)St.nnz;
    rec.bytes_filter = fo.bytes;
    if (Sn.nnz == 0) {
      rec.ms = ts.ms();
      res->steps.push_back(rec);
      break;
    }
    if (record) {
      record->S.emplace_back();
      copy_csr(Sn.view(), s, record->S.back());
    }
    CsrOwned Tn;
    add(T.view(), Sn.view(), 1.0, s, Tn, hs);
    T = std::move(Tn);
    S = std::move(Sn);
    Sv = S.view();
    rec.ms = ts.ms();
    res->steps.push_back(rec);
  }
  S.rp.free(); S.ci.free(); S.v.free();
  if (sym) {
    // For symmetric H the exact T_0 is symmetric, but a filtered term S^_i no longer commutes
    // with H_0, so S^_{i-1} H_0 (and T^_0) can lose symmetry at the level of the dropped
    // entries.  T^_0 <- (T^_0 + T^_0^T)/2 restores it; from then on every T~_i = 2T + T T is
    // symmetric and the squarings form only the entries at columns >= row.
    CsrOwned Ts;
    symmetric_part(T.view(), s, Ts, hs);
    T = std::move(Ts);
  }
  if (record) copy_csr(T.view(), s, record->T[0]);
  st.ms_taylor = t_tay.ms();
  // step 4: N filtered squarings
  Timer t_sq(s);
  RowStats rs;
  for (int i = 1; i <= N; ++i) {
    CsrOwned Tn;
    sexpm_step_stats rec;
    square_step(o, T.view(), i, a, r0, sym, s, hs, rs, Tn, &rec, p->sched.p, &T);
    T = std::move(Tn);
    res->steps.push_back(rec);
    if (record && (i % record->stride == 0 || i == N)) copy_csr(T.view(), s, record->T[i]);
  }
  st.ms_squaring = t_sq.ms();
  // step 5: e^{tau H} = I + T^_N
  Timer t_fin(s);
  add_identity(T.view(), s, res->E, hs);
  st.ms_final = t_fin.ms();
  st.nnz_out = res->E.nnz;
  st.n_steps = (int32_t)res->steps.size();
  st.ms_total = t_all.ms();
  st.peak_bytes = Pool::peak() - live0;
  st.launches = launches() - launches0;
}

// Algorithm 4.1 on the top rows of a complex iterate (decisions by |z|), then A~ = A - b_n.
FilterOut filter_complex(const CsrD& A, int64_t n, double eps_g, double e_r, int max_iters, cudaStream_t s,
                         CsrOwned& out, HostScalars& hs) {
  FilterOut r;
  Timer tf(s);
  DevBuf<int32_t> keep(A.n ? A.n : 1, s);
  DevBuf<double> part(A.n ? A.n : 1, s);
  double m = 1.0;
  double b = std::numeric_limits<double>::infinity();  // the first pass always runs
  double eps_f = eps_g;
  int it = 0;
  while (b > eps_g * (1.0 + e_r)) {
    if (it >= max_iters) fail(SEXPM_ENOCONV, "Algorithm 4.1 did not converge within " + std::to_string(max_iters) + " passes");
    eps_f = eps_g / m;
    b = std::sqrt(pass_complex(A, n, eps_f, keep.p, part.p, s, hs));
    m = b / eps_f;
    ++it;
  }
  compact_complex(A, n, eps_f, keep.p, s, out, hs);
  r.t = eps_f;
  r.b = b;
  r.iters = it;
  r.ms = tf.ms();
  r.bytes = it * 12.0 * A.nnz + 12.0 * A.nnz + 12.0 * out.nnz;
  return r;
}

// Algorithm 4.2 for a complex plan, on the even rows of the real embedding: every product forms
// the n even rows of R(A) R(B) (B rebuilt whole by the mirror), Algorithm 4.1 decides by the
// modulus, and the result is read back as complex entries.  The symmetric mode and the
// row chunking of the real path are not used.
void compute_complex(sexpm_plan_t* p, double tau, sexpm_result* res) {
  if (!std::isfinite(tau)) fail(SEXPM_EINVAL, "tau must be finite");
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) fail(SEXPM_EINVAL, "current device differs from the plan's device");
  cudaStream_t s = p->s;
  HostScalars& hs = p->hs;
  const sexpm_options& o = p->opt;
  const int64_t n = p->H.n;
  res->s = s;
  res->cplx = true;
  std::memset(&res->st, 0, sizeof(res->st));
  sexpm_stats_t& st = res->st;
  st.n = n;
  Pool::reset_peak();
  const int64_t live0 = Pool::live();
  const int64_t launches0 = launches();
  Timer t_all(s);
  // step 1: tau H; ||tau H||_F^2 = sum of |z|^2 = sum of v^2 over the top rows
  CsrD Hs = p->H.view();
  DevBuf<double> hv(p->H.nnz, s);
  scale_values(p->H.v.p, tau, p->H.nnz, hv.p, s);
  Hs.v = hv.p;
  const double normH = std::sqrt(sum_squares(Hs, s, hs));
  st.norm_H = normH;
  int32_t M = 0, N = 0;
  const int rc = sexpm_choose_MN(normH, p->eps, o.n_extra, o.max_taylor, &M, &N);
  if (rc != SEXPM_OK) fail(rc, rc == SEXPM_ENOPARAM ? "no feasible (M, N) for this tolerance" : "invalid (M, N) input");
  st.M = M;
  st.N = N;
  const bool normal = (p->normal != 0) || normH == 0.0;
  st.normal = normal ? 1 : 0;
  st.symmetric = 0;
  CsrOwned T;  // top rows of the running T^
  if (M == 0) {
    T.n = n;
    T.rp.reset(n + 1, s);
    SX_CUDA(cudaMemsetAsync(T.rp.p, 0, (n + 1) * sizeof(int64_t), s));
  } else {
    const double a = normal ? 1.0 / (1.0 + N) : 1.0 / normH;
    st.a = a;
    // step 3: Taylor phase on H_0 = tau H 2^-N
    Timer t_tay(s);
    DevBuf<double> h0v(p->H.nnz, s);
    scale_values(hv.p, std::ldexp(1.0, -N), p->H.nnz, h0v.p, s);
    CsrD H0 = Hs;
    H0.v = h0v.p;
    CsrOwned H0full;
    block_mirror(H0, n, s, H0full);
    const double x0 = std::ldexp(normH, -N);
    const double r0 = sexpm_rho(M, x0);
    const double eps_g0 = a * r0 / ((double)M * std::exp(2.0 * x0));
    st.r0 = r0;
    st.eps_g0 = eps_g0;
    copy_csr(H0, s, T);
    CsrOwned S;
    CsrD Sv = H0;
    CsrD none;
    for (int i = 2; i <= M; ++i) {
      Timer ts(s);
      CsrOwned St;
      SpgemmTimes tm;
      int64_t done = 0;
      const int64_t prod = spgemm(Sv, H0full.view(), none, (double)i, 0.0, s, St, nullptr, hs, &tm, false, &done);
      CsrOwned Sn;
      FilterOut fo = filter_complex(St.view(), n, eps_g0, o.e_r, o.max_filter_iters, s, Sn, hs);
      sexpm_step_stats rec;
      std::memset(&rec, 0, sizeof(rec));
      rec.phase = 0;
      rec.i = i;
      rec.iters = fo.iters;
      rec.eps_g = eps_g0;
      rec.t = fo.t;
      rec.b = fo.b;
      rec.nnz_raw = St.nnz;
      rec.nnz = Sn.nnz;
      rec.products = prod;
      rec.products_done = done;
      rec.ms_symbolic = tm.ms_symbolic;
      rec.ms_numeric = tm.ms_numeric;
      rec.ms_filter = fo.ms;
      rec.flops = 2.0 * (double)done + (double)St.nnz;
      rec.bytes_filter = fo.bytes;
      if (Sn.nnz == 0) {
        rec.ms = ts.ms();
        res->steps.push_back(rec);
        break;
      }
      CsrOwned Tn;
      add(T.view(), Sn.view(), 1.0, s, Tn, hs);
      T = std::move(Tn);
      S = std::move(Sn);
      Sv = S.view();
      rec.ms = ts.ms();
      res->steps.push_back(rec);
    }
    st.ms_taylor = t_tay.ms();
    // step 4: N filtered squarings T~ = 2 T + T T on the top rows
    Timer t_sq(s);
    RowStats rs;
    for (int i = 1; i <= N; ++i) {
      Timer ts(s);
      CsrOwned Tfull, Tt;
      block_mirror(T.view(), n, s, Tfull);
      SpgemmTimes tm;
      int64_t done = 0;
      const int64_t prod = spgemm(T.view(), Tfull.view(), T.view(), 1.0, 2.0, s, Tt, &rs, hs, &tm, false, &done);
      Tfull.rp.free(); Tfull.ci.free(); Tfull.v.free();
      double normF = 1.0;
      if (o.square_scale) {
        // ||I + T~||_F^2 = sum |z|^2 + n + 2 sum Re z_ii over the even rows (Re z_ii at column 2i)
        const double sq = reduce_sum(rs.sq.p, n, s, hs), tr = trace_re(Tt.view(), s, hs);
        const double f2 = sq + (double)n + 2.0 * tr;
        normF = std::sqrt(f2 > 0.0 ? f2 : 0.0);
      }
      const double eps_g = a * std::ldexp(r0, i) * normF;
      const int64_t nnz_in = T.nnz;
      T.rp.free(); T.ci.free(); T.v.free();
      CsrOwned Tn;
      FilterOut fo = filter_complex(Tt.view(), n, eps_g, o.e_r, o.max_filter_iters, s, Tn, hs);
      sexpm_step_stats rec;
      std::memset(&rec, 0, sizeof(rec));
      rec.phase = 1;
      rec.i = i;
      rec.iters = fo.iters;
      rec.eps_g = eps_g;
      rec.t = fo.t;
      rec.b = fo.b;
      rec.norm_F = normF;
      rec.nnz_raw = Tt.nnz;
      rec.nnz = Tn.nnz;
      rec.products = prod;
      rec.products_done = done;
      rec.ms_symbolic = tm.ms_symbolic;
      rec.ms_numeric = tm.ms_numeric;
      rec.ms_filter = fo.ms;
      rec.flops = 2.0 * (double)done + 2.0 * (double)nnz_in;
      rec.bytes_filter = fo.bytes;
      rec.chunks = 1;
      T = std::move(Tn);
      rec.ms = ts.ms();
      res->steps.push_back(rec);
    }
    st.ms_squaring = t_sq.ms();
  }
  // step 5: e^{tau H} = I + T^_N, read back as complex entries
  Timer t_fin(s);
  CsrOwned E, I2;
  identity_pairs(n, s, I2);
  add(T.view(), I2.view(), 1.0, s, E, hs);
  T.rp.free(); T.ci.free(); T.v.free();
  extract_complex(E.view(), n, s, res->E, res->vz, hs);
  st.ms_final = t_fin.ms();
  st.nnz_out = res->E.nnz;
  st.n_steps = (int32_t)res->steps.size();
  st.ms_total = t_all.ms();
  st.peak_bytes = Pool::peak() - live0;
  st.launches = launches() - launches0;
}

// A device CSR with the pattern of P and the values v (non-owning).
CsrD with_values(const CsrD& P, const double* v) {
  CsrD d = P;
  d.v = v;
  return d;
}

// Reverse pass of the recorded forward run: dL/dH on the stored pattern of H into res->E for
// dL/dE = W.  Returns the device milliseconds it took.
double reverse_pass(sexpm_plan_t* p, const Record& rec, double tau, const sexpm_csr_view* W, sexpm_result* res) {
  cudaStream_t s = p->s;
  HostScalars& hs = p->hs;
  const sexpm_options& o = p->opt;
  Timer t_all(s);
  CsrOwned Wd;
  upload(*W, s, Wd, hs);
  const CsrD Hp = p->H.view();
  res->s = s;
  std::memset(&res->st, 0, sizeof(res->st));
  res->E.n = Hp.n;
  res->E.nnz = Hp.nnz;
  res->E.rp.reset(Hp.n + 1, s);
  res->E.ci.reset(Hp.nnz, s);
  res->E.v.reset(Hp.nnz, s);
  SX_CUDA(cudaMemcpyAsync(res->E.rp.p, Hp.rp, (Hp.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (Hp.nnz) SX_CUDA(cudaMemcpyAsync(res->E.ci.p, Hp.ci, Hp.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  CsrD none;
  if (rec.M == 0) {
    // ||tau H|| = 0: the method returns I; its first-order term is tau H, so dL/dH = tau W
    sddmm(Hp, Wd.view(), none, 0.0, 1.0, false, res->E.v.p, s, hs);
    scale_values(res->E.v.p, tau, Hp.nnz, res->E.v.p, s);
  } else {
    const int N = rec.N;
    // dL/dT_N = W on the pattern of T^_N
    CsrD TN = rec.T.at(N).view();
    DevBuf<double> y(TN.nnz, s);
    sddmm(TN, Wd.view(), none, 0.0, 1.0, false, y.p, s, hs);
    CsrD Ypat = TN;                 // pattern of the current adjoint Y
    CsrOwned Ykeep;                 // owns Y's pattern when it is not a checkpoint
    std::map<int, CsrOwned> seg;    // replayed iterates of the current checkpoint segment
    RowStats rs;
    for (int k = N; k >= 1; --k) {
      // T^_{k-1}: a checkpoint, or replayed from the checkpoint below it
      const int km1 = k - 1;
      if (!rec.T.count(km1) && !seg.count(km1)) {
        seg.clear();
        int c = km1;
        while (!rec.T.count(c)) --c;
        CsrD cur = rec.T.at(c).view();
        for (int j = c + 1; j <= km1; ++j) {
          square_step(o, cur, j, rec.a, rec.r0, false, s, hs, rs, seg[j], nullptr, p->sched.p);
          cur = seg[j].view();
        }
      }
      const CsrD Tp = rec.T.count(km1) ? rec.T.at(km1).view() : seg.at(km1).view();
      // dL/dT_{k-1} = mask_{k-1}(2 Y + Y T^T + T^T Y)
      const CsrD Y = with_values(Ypat, y.p);
      CsrOwned Tpt, Yt;
      transpose(Tp, s, Tpt, hs);
      transpose(Y, s, Yt, hs);
      DevBuf<double> g(Tp.nnz, s);
      sddmm(Tp, Y, Tp, 1.0, 2.0, false, g.p, s, hs);
      sddmm(Tp, Tpt.view(), Yt.view(), 1.0, 0.0, true, g.p, s, hs);
      y = std::move(g);
      // the new Y lives on the pattern of T^_{k-1}; keep that pattern alive
      if (rec.T.count(km1)) {
        Ypat = rec.T.at(km1).view();
        Ykeep = CsrOwned();
      } else {
        CsrOwned pat;
        copy_csr(Tp, s, pat);
        Ykeep = std::move(pat);
        Ypat = Ykeep.view();
      }
      if (rec.T.count(k) && k != N) { /* checkpoints stay until the end */ }
      seg.erase(k);
    }
    // Taylor phase: dL/dS_i = dL/dT_0 on the pattern of S_i, then i = M'..2
    const int Mp = (int)rec.S.size();
    std::vector<DevBuf<double>> gs(Mp);
    const CsrD GT0 = with_values(Ypat, y.p);
    for (int i = 0; i < Mp; ++i) {
      gs[i].reset(rec.S[i].nnz, s);
      sddmm(rec.S[i].view(), GT0, none, 0.0, 1.0, false, gs[i].p, s, hs);
    }
    DevBuf<double> gh(Hp.nnz, s);
    SX_CUDA(cudaMemsetAsync(gh.p, 0, Hp.nnz * sizeof(double), s));
    const CsrD H0 = rec.H0.view();
    for (int i = Mp; i >= 2; --i) {
      const CsrD Yi = with_values(rec.S[i - 1].view(), gs[i - 1].p);
      const CsrD Sp = rec.S[i - 2].view();
      sddmm(Sp, Yi, H0, 1.0 / i, 0.0, true, gs[i - 2].p, s, hs);          // += mask(Y H_0^T)/i
      CsrOwned Spt, Yit;
      transpose(Sp, s, Spt, hs);
      transpose(Yi, s, Yit, hs);
      sddmm(Hp, Spt.view(), Yit.view(), 1.0 / i, 0.0, true, gh.p, s, hs);  // += mask_H(S^T Y)/i
    }
    sddmm(Hp, with_values(rec.S[0].view(), gs[0].p), none, 0.0, 1.0, true, gh.p, s, hs);  // += dL/dS_1
    scale_values(gh.p, tau * std::ldexp(1.0, -N), Hp.nnz, res->E.v.p, s);
  }
  SX_CUDA(cudaStreamSynchronize(s));
  res->st.nnz_out = res->E.nnz;
  return t_all.ms();
}

#define SX_API_BEGIN try {
#define SX_API_END                                         \
  }                                                        \
  catch (const sexpm::Error& e) {                          \
    set_last_error(e.msg);                                 \
    return e.code;                                         \
  }                                                        \
  catch (const std::bad_alloc&) {                          \
    set_last_error("host allocation failed");              \
    return SEXPM_ENOMEM;                                   \
  }                                                        \
  catch (...) {                                            \
    set_last_error("unexpected exception");                \
    return SEXPM_ECUDA;                                    \
  }                                                        \
  set_last_error("");                                      \
  return SEXPM_OK;

extern "C" {

const char* sexpm_last_error(void) { return g_last_error.c_str(); }

int64_t sexpm_kernel_launches(void) { return launches(); }

int sexpm_release_memory(void) {
  SX_API_BEGIN
  SX_CUDA(cudaDeviceSynchronize());
  SX_CUDA(cudaMemPoolTrimTo(pool_for_current_device(), 0));
  SX_API_END
}

int sexpm_pool_stats(int64_t* live_bytes, int64_t* peak_bytes) {
  if (live_bytes) *live_bytes = Pool::live();
  if (peak_bytes) *peak_bytes = Pool::peak();
  return SEXPM_OK;
}

int sexpm_options_default(sexpm_options* opt) {
  if (!opt) return SEXPM_EINVAL;
  opt->e_r = 0.1;
  opt->square_scale = 1;
  opt->normal_override = -1;
  opt->max_filter_iters = 100;
  opt->n_extra = 50;
  opt->max_taylor = 1000;
  opt->symmetric = 1;
  opt->row_order = 1;
  opt->chunk_bytes = 0;
  opt->scaling = 0;
  opt->refine_kmax = 41;
  opt->batched_graph = 1;
  opt->batch_arena_bytes = 0;
  return SEXPM_OK;
}

static void check_options(const sexpm_options& o) {
  if (!(o.e_r > 0.0) || !std::isfinite(o.e_r)) fail(SEXPM_EINVAL, "e_r must be positive and finite");
  if (o.square_scale != 0 && o.square_scale != 1) fail(SEXPM_EINVAL, "square_scale must be 0 or 1");
  if (o.normal_override < -1 || o.normal_override > 1) fail(SEXPM_EINVAL, "normal_override must be -1, 0 or 1");
  if (o.max_filter_iters < 1 || o.n_extra < 0 || o.max_taylor < 1) fail(SEXPM_EINVAL, "bad iteration limits");
  if (o.symmetric != 0 && o.symmetric != 1) fail(SEXPM_EINVAL, "symmetric must be 0 or 1");
  if (o.row_order != 0 && o.row_order != 1) fail(SEXPM_EINVAL, "row_order must be 0 or 1");
  if (o.chunk_bytes < 0) fail(SEXPM_EINVAL, "chunk_bytes must be >= 0");
  if (o.scaling != 0 && o.scaling != 1) fail(SEXPM_EINVAL, "scaling must be 0 or 1");
  if (o.refine_kmax < 3) fail(SEXPM_EINVAL, "refine_kmax must be >= 3");
  if (o.batched_graph != 0 && o.batched_graph != 1) fail(SEXPM_EINVAL, "batched_graph must be 0 or 1");
  if (o.batch_arena_bytes < 0) fail(SEXPM_EINVAL, "batch_arena_bytes must be >= 0");
}

int sexpm_plan(const sexpm_csr_view* H, int64_t n, double eps, const sexpm_options* opt, void* stream,
               sexpm_plan_t** out) {
  SX_API_BEGIN
  if (!H || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  if (H->n != n) fail(SEXPM_EINVAL, "n does not match the matrix dimension");
  if (!(eps > 0.0) || !std::isfinite(eps)) fail(SEXPM_EINVAL, "eps must be positive and finite");
  sexpm_plan_t* p = new sexpm_plan_t();
  try {
    if (opt) p->opt = *opt; else sexpm_options_default(&p->opt);
    check_options(p->opt);
    SX_CUDA(cudaGetDevice(&p->device));
    p->s = static_cast<cudaStream_t>(stream);
    p->eps = eps;
    upload(*H, p->s, p->H, p->hs);
    classify_matrix(p->H, p->opt.normal_override, p->s, p->hs, p->symmetric, p->normal);
    if (p->opt.row_order) p->grid_stride = grid_schedule(p->H, p->s, p->sched);
    SX_CUDA(cudaStreamSynchronize(p->s));
  } catch (...) {
    delete p;
    throw;
  }
  *out = p;
  SX_API_END
}

int sexpm_compute(sexpm_plan_t* p, double tau, sexpm_result_t** out) {
  SX_API_BEGIN
  if (!p || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  if (p->count > 0) fail(SEXPM_EINVAL, "batched plan: use sexpm_compute_batched");
  sexpm_result* res = new sexpm_result();
  arm_alloc_failure();
  try {
    if (p->cplx) compute_complex(p, tau, res);
    else compute_impl(p, tau, res, nullptr, p->opt.symmetric != 0);
  } catch (...) {
    delete res;
    throw;
  }
  *out = res;
  SX_API_END
}

int sexpm_result_info(const sexpm_result_t* r, int64_t* n, int64_t* nnz) {
  if (!r) {
    set_last_error("null result");
    return SEXPM_EINVAL;
  }
  if (n) *n = r->E.n;
  if (nnz) *nnz = r->E.nnz;
  return SEXPM_OK;
}

int sexpm_result_copy(const sexpm_result_t* r, int64_t* row_ptr, int32_t* col, double* val, int32_t on_device) {
  SX_API_BEGIN
  if (!r) fail(SEXPM_EINVAL, "null result");
  if (r->cplx) fail(SEXPM_EINVAL, "complex result: use sexpm_result_copy_z");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (row_ptr) SX_CUDA(cudaMemcpyAsync(row_ptr, r->E.rp.p, (r->E.n + 1) * sizeof(int64_t), k, r->s));
  if (r->E.nnz) {
    if (col) SX_CUDA(cudaMemcpyAsync(col, r->E.ci.p, r->E.nnz * sizeof(int32_t), k, r->s));
    if (val) SX_CUDA(cudaMemcpyAsync(val, r->E.v.p, r->E.nnz * sizeof(double), k, r->s));
  }
  SX_CUDA(cudaStreamSynchronize(r->s));
  SX_API_END
}

int sexpm_result_copy_z(const sexpm_result_t* r, int64_t* row_ptr, int32_t* col, double* val, int32_t on_device) {
  SX_API_BEGIN
  if (!r) fail(SEXPM_EINVAL, "null result");
  if (!r->cplx) fail(SEXPM_EINVAL, "real result: use sexpm_result_copy");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (row_ptr) SX_CUDA(cudaMemcpyAsync(row_ptr, r->E.rp.p, (r->E.n + 1) * sizeof(int64_t), k, r->s));
  if (r->E.nnz) {
    if (col) SX_CUDA(cudaMemcpyAsync(col, r->E.ci.p, r->E.nnz * sizeof(int32_t), k, r->s));
    if (val) SX_CUDA(cudaMemcpyAsync(val, r->vz.p, 2 * r->E.nnz * sizeof(double), k, r->s));
  }
  SX_CUDA(cudaStreamSynchronize(r->s));
  SX_API_END
}

int sexpm_result_is_complex(const sexpm_result_t* r, int32_t* is_complex) {
  if (!r || !is_complex) {
    set_last_error("null argument");
    return SEXPM_EINVAL;
  }
  *is_complex = r->cplx ? 1 : 0;
  return SEXPM_OK;
}

int sexpm_plan_z(const sexpm_csr_view* H, int64_t n, double eps, const sexpm_options* opt, void* stream,
                 sexpm_plan_t** out) {
  SX_API_BEGIN
  if (!H || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  if (H->n != n) fail(SEXPM_EINVAL, "n does not match the matrix");
  if (!(eps > 0.0) || !std::isfinite(eps)) fail(SEXPM_EINVAL, "eps must be positive and finite");
  if (H->n < 0 || H->nnz < 0 || H->n > INT32_MAX / 2) fail(SEXPM_EINVAL, "bad dimensions (n <= 2^30 for complex H)");
  if (H->n > 0 && (!H->row_ptr || (H->nnz > 0 && (!H->col || !H->val)))) fail(SEXPM_EINVAL, "null CSR array");
  sexpm_plan_t* p = new sexpm_plan_t();
  try {
    if (opt) p->opt = *opt; else sexpm_options_default(&p->opt);
    check_options(p->opt);
    if (p->opt.scaling != 0) fail(SEXPM_EINVAL, "complex plans use the scaling of Eq. (4.20) (scaling = 0)");
    SX_CUDA(cudaGetDevice(&p->device));
    p->s = static_cast<cudaStream_t>(stream);
    p->eps = eps;
    p->cplx = true;
    cudaStream_t s = p->s;
    const int64_t nn = H->n, nz = H->nnz;
    if (!H->on_device && nn > 0) {
      if (H->row_ptr[0] != 0 || H->row_ptr[nn] != nz) fail(SEXPM_EINVAL, "row_ptr must start at 0 and end at nnz");
      for (int64_t i = 0; i < nn; ++i) {
        const int64_t p0 = H->row_ptr[i], p1 = H->row_ptr[i + 1];
        if (p1 < p0 || p1 > nz) fail(SEXPM_EINVAL, "row_ptr not monotone at row " + std::to_string(i));
        int32_t prev = -1;
        for (int64_t q = p0; q < p1; ++q) {
          const int32_t c = H->col[q];
          if (c <= prev || c >= nn) fail(SEXPM_EINVAL, "columns unsorted, duplicated or out of range in row " + std::to_string(i));
          if (!std::isfinite(H->val[2 * q]) || !std::isfinite(H->val[2 * q + 1]))
            fail(SEXPM_EINVAL, "non-finite value in row " + std::to_string(i));
          prev = c;
        }
      }
    }
    DevBuf<int64_t> rp(nn + 1, s);
    DevBuf<int32_t> ci(nz, s);
    DevBuf<double> vz(2 * nz, s);
    const cudaMemcpyKind k = H->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nn > 0) SX_CUDA(cudaMemcpyAsync(rp.p, H->row_ptr, (nn + 1) * sizeof(int64_t), k, s));
    else SX_CUDA(cudaMemsetAsync(rp.p, 0, sizeof(int64_t), s));
    if (nz) {
      SX_CUDA(cudaMemcpyAsync(ci.p, H->col, nz * sizeof(int32_t), k, s));
      SX_CUDA(cudaMemcpyAsync(vz.p, H->val, 2 * nz * sizeof(double), k, s));
    }
    if (H->on_device && nn > 0 && !valid_complex(nn, nz, rp.p, ci.p, vz.p, s, p->hs))
      fail(SEXPM_EINVAL, "invalid device CSR (row_ptr, column order/range or non-finite value)");
    embed_top(nn, nz, rp.p, ci.p, vz.p, s, p->H);
    // Hermitian H <=> its embedding is symmetric; skew-Hermitian <=> skew-symmetric; otherwise
    // the commutator test with the complex norms
    CsrOwned full;
    block_mirror(p->H.view(), nn, s, full);
    bool herm = false;
    classify_matrix(full, p->opt.normal_override, s, p->hs, herm, p->normal, 1.0 / std::sqrt(2.0));
    p->symmetric = false;
    SX_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    delete p;
    throw;
  }
  *out = p;
  SX_API_END
}

int sexpm_stats(const sexpm_result_t* r, sexpm_stats_t* stats, sexpm_step_stats* steps, int32_t max_steps) {
  if (!r || !stats) {
    set_last_error("null argument");
    return SEXPM_EINVAL;
  }
  *stats = r->st;
  stats->n_steps = (int32_t)r->steps.size();
  if (steps)
    for (int32_t k = 0; k < max_steps && k < (int32_t)r->steps.size(); ++k) steps[k] = r->steps[k];
  return SEXPM_OK;
}

void sexpm_result_free(sexpm_result_t* r) { delete r; }

void sexpm_plan_destroy(sexpm_plan_t* p) { delete p; }

int sexpm_spgemm(const sexpm_csr_view* A, const sexpm_csr_view* B, const sexpm_csr_view* D, double div, double beta,
                 void* stream, sexpm_result_t** out, int64_t* products) {
  SX_API_BEGIN
  if (!A || !B || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  if (A->n != B->n || (D && D->n != A->n)) fail(SEXPM_EINVAL, "dimension mismatch");
  if (!(div != 0.0) || !std::isfinite(div) || !std::isfinite(beta)) fail(SEXPM_EINVAL, "div must be finite and nonzero, beta finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a, b, d;
  upload(*A, s, a, hs);
  upload(*B, s, b, hs);
  CsrD dv;
  if (D) {
    upload(*D, s, d, hs);
    dv = d.view();
  }
  sexpm_result* res = new sexpm_result();
  try {
    res->s = s;
    std::memset(&res->st, 0, sizeof(res->st));
    sexpm_step_stats rec;
    std::memset(&rec, 0, sizeof(rec));
    int64_t done = 0;
    const int64_t prod = spgemm(a.view(), b.view(), dv, div, beta, s, res->E, nullptr, hs, nullptr, false, &done,
                                nullptr, nullptr, rec.rows_class);
    SX_CUDA(cudaStreamSynchronize(s));
    res->st.n = res->E.n;
    res->st.nnz_out = res->E.nnz;
    rec.chunks = 1;
    rec.nnz_raw = rec.nnz = res->E.nnz;
    rec.products = prod;
    rec.products_done = done;
    res->steps.push_back(rec);
    res->st.n_steps = 1;
    if (products) *products = prod;
  } catch (...) {
    delete res;
    throw;
  }
  *out = res;
  SX_API_END
}

int sexpm_filter(const sexpm_csr_view* A, double eps_g, double e_r, int32_t max_iters, void* stream,
                 sexpm_result_t** out, double* t, int32_t* iters, double* b) {
  SX_API_BEGIN
  if (!A || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  if (!(eps_g >= 0.0) || !std::isfinite(eps_g) || !(e_r > 0.0) || !std::isfinite(e_r) || max_iters < 1)
    fail(SEXPM_EINVAL, "bad filter parameters");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*A, s, a, hs);
  sexpm_result* res = new sexpm_result();
  try {
    res->s = s;
    std::memset(&res->st, 0, sizeof(res->st));
    FilterOut fo = filter_alg41(a.view(), eps_g, e_r, max_iters, s, res->E, hs);
    SX_CUDA(cudaStreamSynchronize(s));
    res->st.n = res->E.n;
    res->st.nnz_out = res->E.nnz;
    if (t) *t = fo.t;
    if (iters) *iters = fo.iters;
    if (b) *b = fo.b;
  } catch (...) {
    delete res;
    throw;
  }
  *out = res;
  SX_API_END
}

int sexpm_result_spmm(const sexpm_result_t* E, const double* X, int64_t r, double* Y, void* stream) {
  SX_API_BEGIN
  if (!E || (E->E.n && r > 0 && (!X || !Y))) fail(SEXPM_EINVAL, "null argument");
  if (r < 0) fail(SEXPM_EINVAL, "r must be >= 0");
  if (E->cplx) fail(SEXPM_EINVAL, "e^H R takes a real result");
  if (X == Y && E->E.n && r) fail(SEXPM_EINVAL, "X and Y must not overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spmm(E->E.view(), X, r, Y, s);
  SX_CUDA(cudaStreamSynchronize(s));
  SX_API_END
}

int sexpm_propagate(const sexpm_result_t* E, const double* U0, int64_t r, int32_t steps, double* U, void* stream) {
  SX_API_BEGIN
  if (!E || (E->E.n && r > 0 && (!U0 || !U))) fail(SEXPM_EINVAL, "null argument");
  if (r < 0 || steps < 0) fail(SEXPM_EINVAL, "r and steps must be >= 0");
  if (E->cplx) fail(SEXPM_EINVAL, "time stepping takes a real result");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = E->E.n;
  const size_t bytes = (size_t)n * (size_t)r * sizeof(double);
  if (n && r) {
    // two work arrays, alternated; the last product is copied to U (which may alias U0)
    DevBuf<double> w0((size_t)n * (size_t)r, s), w1(steps > 1 ? (size_t)n * (size_t)r : 0, s);
    const double* src = U0;
    for (int k = 0; k < steps; ++k) {
      double* dst = (k % 2 == 0) ? w0.p : w1.p;
      spmm(E->E.view(), src, r, dst, s);
      src = dst;
    }
    if (src != U) SX_CUDA(cudaMemcpyAsync(U, src, bytes, cudaMemcpyDeviceToDevice, s));
  }
  SX_CUDA(cudaStreamSynchronize(s));
  SX_API_END
}

int sexpm_spmm(const sexpm_csr_view* A, const double* X, int64_t r, double* Y, void* stream) {
  SX_API_BEGIN
  if (!A || (A->n && r > 0 && (!X || !Y))) fail(SEXPM_EINVAL, "null argument");
  if (r < 0) fail(SEXPM_EINVAL, "r must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*A, s, a, hs);
  spmm(a.view(), X, r, Y, s);
  SX_CUDA(cudaStreamSynchronize(s));
  SX_API_END
}

int sexpm_power_norms(const sexpm_csr_view* H, int32_t kmax, void* stream, double* out) {
  SX_API_BEGIN
  if (!H || !out || kmax < 1) fail(SEXPM_EINVAL, "null argument or kmax < 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*H, s, a, hs);
  power_norms(a.view(), kmax, s, hs, out);
  SX_API_END
}

int sexpm_transpose(const sexpm_csr_view* A, void* stream, sexpm_result_t** out) {
  SX_API_BEGIN
  if (!A || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*A, s, a, hs);
  sexpm_result* res = new sexpm_result();
  try {
    res->s = s;
    std::memset(&res->st, 0, sizeof(res->st));
    transpose(a.view(), s, res->E, hs);
    SX_CUDA(cudaStreamSynchronize(s));
    res->st.n = res->E.n;
    res->st.nnz_out = res->E.nnz;
  } catch (...) {
    delete res;
    throw;
  }
  *out = res;
  SX_API_END
}

int sexpm_filter_pass(const sexpm_csr_view* A, double t, void* stream, double* sum_dropped, int64_t* kept) {
  SX_API_BEGIN
  if (!A || !sum_dropped) fail(SEXPM_EINVAL, "null argument");
  if (!(t >= 0.0)) fail(SEXPM_EINVAL, "t must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*A, s, a, hs);
  Piece p;
  p.r1 = a.n;
  p.nnz = a.nnz;
  p.rp = a.rp.p;
  p.ci = a.ci.p;
  p.v = a.v.p;
  std::vector<Piece> P{p};
  std::vector<int64_t> base{0, counts_of(a.nnz)};
  DevBuf<int32_t> tc(base[1] ? base[1] : 1, s);
  *sum_dropped = pass_pieces(P, base, t, tc.p, s, hs);
  if (kept) {
    DevBuf<int64_t> off(base[1] + 1, s);
    *kept = scan_counts(tc.p, base[1], off.p, s, hs);
  }
  SX_API_END
}

int sexpm_filter_apply(const sexpm_csr_view* A, double t, void* stream, sexpm_result_t** out) {
  SX_API_BEGIN
  if (!A || !out) fail(SEXPM_EINVAL, "null argument");
  *out = nullptr;
  if (!(t >= 0.0)) fail(SEXPM_EINVAL, "t must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*A, s, a, hs);
  sexpm_result* res = new sexpm_result();
  try {
    res->s = s;
    std::memset(&res->st, 0, sizeof(res->st));
    Piece p;
    p.r1 = a.n;
    p.nnz = a.nnz;
    p.rp = a.rp.p;
    p.ci = a.ci.p;
    p.v = a.v.p;
    std::vector<Piece> P{p};
    std::vector<int64_t> base{0, counts_of(a.nnz)};
    DevBuf<int32_t> tc(base[1] ? base[1] : 1, s);
    pass_pieces(P, base, t, tc.p, s, hs);
    res->E.n = a.n;
    res->E.rp.reset(a.n + 1, s);
    DevBuf<int64_t> off(base[1] + 1, s);
    res->E.nnz = scan_counts(tc.p, base[1], off.p, s, hs);
    res->E.ci.reset(res->E.nnz, s);
    res->E.v.reset(res->E.nnz, s);
    if (a.n == 0) SX_CUDA(cudaMemsetAsync(res->E.rp.p, 0, sizeof(int64_t), s));
    else compact_pieces(P, base, t, off.p, a.n, res->E, s);
    SX_CUDA(cudaStreamSynchronize(s));
    res->st.n = res->E.n;
    res->st.nnz_out = res->E.nnz;
  } catch (...) {
    delete res;
    throw;
  }
  *out = res;
  SX_API_END
}

int sexpm_norm2_I_plus_rows(const sexpm_csr_view* A, int64_t r0, int64_t r1, void* stream, double* out) {
  SX_API_BEGIN
  if (!A || !out) fail(SEXPM_EINVAL, "null argument");
  if (r0 < 0 || r1 < r0 || r1 > A->n) fail(SEXPM_EINVAL, "row range outside the matrix");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostScalars hs;
  CsrOwned a;
  upload(*A, s, a, hs);
  *out = norm2_I_plus_rows(a.view(), r0, r1, s, hs);
  SX_API_END
}

int sexpm_plan_batched(const sexpm_csr_view* Hs, int32_t count, double eps, const sexpm_options* opt, void* stream,
                       sexpm_plan_t** out) {
  SX_API_BEGIN
  if (!Hs || !out || count < 1) fail(SEXPM_EINVAL, "need count >= 1 matrices");
  *out = nullptr;
  if (!(eps > 0.0) || !std::isfinite(eps)) fail(SEXPM_EINVAL, "eps must be positive and finite");
  sexpm_plan_t* p = new sexpm_plan_t();
  try {
    if (opt) p->opt = *opt; else sexpm_options_default(&p->opt);
    check_options(p->opt);
    if (p->opt.scaling != 0) fail(SEXPM_EINVAL, "the batched form uses the scaling of Eq. (4.20) (scaling = 0)");
    SX_CUDA(cudaGetDevice(&p->device));
    p->s = static_cast<cudaStream_t>(stream);
    p->eps = eps;
    p->count = count;
    cudaStream_t s = p->s;
    p->row0.assign(count + 1, 0);
    std::vector<int64_t> nz0(count + 1, 0);
    for (int b = 0; b < count; ++b) {
      if (Hs[b].n < 0 || Hs[b].nnz < 0) fail(SEXPM_EINVAL, "bad dimensions of instance " + std::to_string(b));
      p->row0[b + 1] = p->row0[b] + Hs[b].n;
      nz0[b + 1] = nz0[b] + Hs[b].nnz;
    }
    if (p->row0[count] > INT32_MAX) fail(SEXPM_EOVERFLOW, "the batch has more than 2^31 rows");
    const int64_t n = p->row0[count], nnz = nz0[count];
    p->H.n = n;
    p->H.nnz = nnz;
    p->H.rp.reset(n + 1, s);
    p->H.ci.reset(nnz, s);
    p->H.v.reset(nnz, s);
    p->normal_b.assign(count, 1);
    p->symmetric_b.assign(count, 1);
    for (int b = 0; b < count; ++b) {
      CsrOwned Hb;
      upload(Hs[b], s, Hb, p->hs);
      bool sym = false;
      int nor = 1;
      classify_matrix(Hb, p->opt.normal_override, s, p->hs, sym, nor);
      p->symmetric_b[b] = sym ? 1 : 0;
      p->normal_b[b] = nor;
      block_put(Hb.view(), p->row0[b], nz0[b], p->H.rp.p, p->H.ci.p, p->H.v.p, s);
      SX_CUDA(cudaStreamSynchronize(s));
    }
    SX_CUDA(cudaMemcpyAsync(p->H.rp.p + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    p->seg.reset(count + 1, s);
    SX_CUDA(cudaMemcpyAsync(p->seg.p, p->row0.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    p->inst.reset(n ? n : 1, s);
    instance_of_row(p->seg.p, count, n, p->inst.p, s);
    p->symmetric = true;
    for (int b = 0; b < count; ++b) p->symmetric = p->symmetric && p->symmetric_b[b];
    SX_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    delete p;
    throw;
  }
  *out = p;
  SX_API_END
}

int sexpm_compute_batched(sexpm_plan_t* p, const double* taus, sexpm_result_t** outs) {
  SX_API_BEGIN
  if (!p || !taus || !outs) fail(SEXPM_EINVAL, "null argument");
  if (p->count == 0) {
    const int rc = sexpm_compute(p, taus[0], outs);
    if (rc != SEXPM_OK) return rc;
    set_last_error("");
    return SEXPM_OK;
  }
  const int count = p->count;
  for (int b = 0; b < count; ++b) {
    outs[b] = nullptr;
    if (!std::isfinite(taus[b])) fail(SEXPM_EINVAL, "tau of instance " + std::to_string(b) + " is not finite");
  }
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) fail(SEXPM_EINVAL, "current device differs from the plan's device");
  cudaStream_t s = p->s;
  HostScalars& hs = p->hs;
  const sexpm_options& o = p->opt;
  const int64_t n = p->H.n;
  const int32_t* inst = p->inst.p;
  const int64_t* seg = p->seg.p;
  Pool::reset_peak();
  const int64_t live0 = Pool::live();
  const int64_t launches0 = launches();
  Timer t_all(s);
  std::vector<sexpm_step_stats> steps;
  // step 1: tau_b H_b, ||tau_b H_b||_F, (M_b, N_b)
  DevBuf<double> dtmp(count, s);
  SX_CUDA(cudaMemcpyAsync(dtmp.p, taus, count * sizeof(double), cudaMemcpyHostToDevice, s));
  DevBuf<double> hv(p->H.nnz, s);
  CsrD Hs = p->H.view();
  scale_rows(Hs, inst, dtmp.p, hv.p, s);
  Hs.v = hv.p;
  std::vector<double> sums(count, 0.0), normH(count), a(count), r0(count), eps_g0(count), x0(count);
  std::vector<int32_t> M(count), N(count);
  {
    DevBuf<int32_t> keep(n ? n : 1, s);
    DevBuf<double> part(n ? n : 1, s);
    std::vector<double> inf(count, std::numeric_limits<double>::infinity());
    SX_CUDA(cudaMemcpyAsync(dtmp.p, inf.data(), count * sizeof(double), cudaMemcpyHostToDevice, s));
    filter_pass_seg(Hs, inst, dtmp.p, keep.p, part.p, seg, count, sums.data(), s);
  }
  int32_t Mmax = 0, Nmax = 0;
  for (int b = 0; b < count; ++b) {
    normH[b] = std::sqrt(sums[b]);
    const int rc = sexpm_choose_MN(normH[b], p->eps, o.n_extra, o.max_taylor, &M[b], &N[b]);
    if (rc != SEXPM_OK) fail(rc, "no feasible (M, N) for instance " + std::to_string(b));
    const bool nor = p->normal_b[b] != 0 || normH[b] == 0.0;
    a[b] = nor ? 1.0 / (1.0 + N[b]) : 1.0 / normH[b];
    x0[b] = std::ldexp(normH[b], -N[b]);
    r0[b] = M[b] > 0 ? sexpm_rho(M[b], x0[b]) : 0.0;
    eps_g0[b] = M[b] > 0 ? a[b] * r0[b] / ((double)M[b] * std::exp(2.0 * x0[b])) : 0.0;
    Mmax = std::max(Mmax, M[b]);
    Nmax = std::max(Nmax, N[b]);
  }
  const bool sym = p->symmetric && o.symmetric;
  // step 3: Taylor phase for all instances at once
  Timer t_tay(s);
  std::vector<double> fac(count);
  for (int b = 0; b < count; ++b) fac[b] = std::ldexp(1.0, -N[b]);
  SX_CUDA(cudaMemcpyAsync(dtmp.p, fac.data(), count * sizeof(double), cudaMemcpyHostToDevice, s));
  DevBuf<double> h0v(p->H.nnz, s);
  scale_rows(Hs, inst, dtmp.p, h0v.p, s);
  CsrD H0 = Hs;
  H0.v = h0v.p;
  CsrOwned T;
  copy_csr(H0, s, T);
  CsrOwned S;
  CsrD Sv = H0;
  CsrD none;
  std::vector<char> done_b(count, 0);
  for (int b = 0; b < count; ++b) done_b[b] = M[b] <= 1;
  std::vector<int64_t> bnd(count + 1);
  const double inf = std::numeric_limits<double>::infinity();
  // the captured steps' description of the batch (Taylor terms and squarings)
  GraphSquaringIn gi;
  gi.count = count;
  gi.n = n;
  gi.inst = inst;
  gi.seg = seg;
  gi.N = N;
  gi.M = M;
  gi.a = a;
  gi.r0 = r0;
  gi.eps_g0 = eps_g0;
  gi.nb.resize(count);
  for (int b = 0; b < count; ++b) {
    const int64_t nb = p->row0[b + 1] - p->row0[b];
    gi.nb[b] = (double)nb;
    gi.n_max = std::max(gi.n_max, nb);
    gi.dense += nb * nb;
  }
  gi.arena_bytes = o.batch_arena_bytes;
  gi.sym = sym;
  gi.square_scale = o.square_scale != 0;
  gi.e_r = o.e_r;
  gi.max_iters = o.max_filter_iters;
  // the Taylor terms as captured graphs (one per term); host-driven launches when they are off
  // or the arena does not fit in device memory
  bool taylor_done = false;
  if (o.batched_graph != 0 && Mmax >= 2 && Mmax <= 128) {
    if (!p->graph) p->graph = graph_squaring_new();
    graph_squaring_set_layout(p->graph, p->layout_ks, p->layout_wide);
    GraphSquaringOut tout;
    try {
      graph_taylor(p->graph, H0, gi, tout, s);
      CsrOwned Tg;
      copy_csr(tout.T, s, Tg);
      T = std::move(Tg);
      for (const auto& st : tout.steps) steps.push_back(st);
      taylor_done = true;
    } catch (const Error& e) {
      if (e.code != SEXPM_ENOMEM) throw;
      graph_squaring_release(p->graph, false);
    }
  }
  for (int i = 2; i <= Mmax && !taylor_done; ++i) {
    Timer ts(s);
    CsrOwned St;
    SpgemmTimes tm;
    int64_t done = 0;
    const int64_t prod = spgemm(Sv, H0, none, (double)i, 0.0, s, St, nullptr, hs, &tm, false, &done);
    std::vector<double> eg(count), fixed(count, -1.0);
    for (int b = 0; b < count; ++b) {
      eg[b] = eps_g0[b];
      if (done_b[b] || i > M[b]) fixed[b] = inf;
    }
    CsrOwned Sn;
    SegFilterOut fo = filter_seg(St.view(), eg, fixed, o.e_r, o.max_filter_iters, inst, seg, count, s, Sn, hs);
    gather_row_ptr(Sn.rp.p, seg, count, bnd.data(), s);
    for (int b = 0; b < count; ++b)
      if (bnd[b + 1] == bnd[b]) done_b[b] = 1;
    sexpm_step_stats rec;
    std::memset(&rec, 0, sizeof(rec));
    rec.phase = 0;
    rec.i = i;
    for (int b = 0; b < count; ++b) {
      rec.iters = std::max(rec.iters, fo.iters[b]);
      if (fixed[b] < 0.0) rec.t = std::max(rec.t, fo.t[b]);
    }
    rec.nnz_raw = St.nnz;
    rec.nnz = Sn.nnz;
    rec.products = prod;
    rec.products_done = done;
    rec.ms_symbolic = tm.ms_symbolic;
    rec.ms_numeric = tm.ms_numeric;
    rec.ms_filter = fo.ms;
    rec.flops = 2.0 * (double)done + (double)St.nnz;
    if (Sn.nnz == 0) {
      rec.ms = ts.ms();
      steps.push_back(rec);
      break;
    }
    CsrOwned Tn;
    add(T.view(), Sn.view(), 1.0, s, Tn, hs);
    T = std::move(Tn);
    S = std::move(Sn);
    Sv = S.view();
    rec.ms = ts.ms();
    steps.push_back(rec);
  }
  S.rp.free(); S.ci.free(); S.v.free();
  if (sym) {
    CsrOwned Ts;
    symmetric_part(T.view(), s, Ts, hs);
    T = std::move(Ts);
  }
  const double ms_taylor = t_tay.ms();
  // step 4: squarings; instance b is frozen (copied through) once its N_b squarings are done
  Timer t_sq(s);
  // the captured step first (all N_max squarings unless device memory runs out; the
  // host-driven launches below then do the rest from the last completed step)
  const bool use_graph = o.batched_graph != 0 && Nmax > 0 && Nmax <= 128;
  GraphSquaringOut gout;
  int g_start = 1;
  if (use_graph) {
    if (!p->graph) p->graph = graph_squaring_new();
    graph_squaring_set_layout(p->graph, p->layout_ks, p->layout_wide);
    graph_squarings(p->graph, T.view(), gi, gout, s);
    for (const auto& st : gout.steps) steps.push_back(st);
    g_start = gout.steps_done + 1;
    if (gout.steps_done < Nmax) {
      if (gout.steps_done > 0) {
        CsrOwned Tg;
        copy_csr(gout.T, s, Tg);
        T = std::move(Tg);
      }
      graph_squaring_release(p->graph, false);
      graph_squaring_note_host_steps(p->graph, Nmax - gout.steps_done);
    }
  }
  const bool graph_result = use_graph && gout.steps_done == Nmax;
  RowStats rs;
  DevBuf<uint8_t> frozen_inst(count, s), frozen_row(n ? n : 1, s);
  std::vector<uint8_t> fz(count);
  std::vector<double> sq(count), tr(count);
  for (int g = graph_result ? Nmax + 1 : g_start; g <= Nmax; ++g) {
    Timer ts(s);
    for (int b = 0; b < count; ++b) fz[b] = N[b] < g ? 1 : 0;
    SX_CUDA(cudaMemcpyAsync(frozen_inst.p, fz.data(), count, cudaMemcpyHostToDevice, s));
    row_flags(inst, frozen_inst.p, n, frozen_row.p, s);
    CsrOwned Tt;
    SpgemmTimes tm;
    int64_t done = 0;
    const int64_t prod = spgemm(T.view(), T.view(), T.view(), 1.0, 2.0, s, Tt, &rs, hs, &tm, sym, &done, frozen_row.p);
    std::vector<double> eg(count, 0.0), fixed(count, -1.0);
    if (o.square_scale) {
      seg_sums(rs.sq.p, seg, count, sq.data(), s);
      seg_sums(rs.diag.p, seg, count, tr.data(), s);
    }
    for (int b = 0; b < count; ++b) {
      if (fz[b]) {
        fixed[b] = 0.0;  // keep every stored nonzero: the instance is finished
        continue;
      }
      double normF = 1.0;
      if (o.square_scale) {
        const double f2 = sq[b] + (double)(p->row0[b + 1] - p->row0[b]) + 2.0 * tr[b];
        normF = std::sqrt(f2 > 0.0 ? f2 : 0.0);
      }
      eg[b] = a[b] * std::ldexp(r0[b], g) * normF;
    }
    const double flops = 2.0 * (double)done + 2.0 * (double)T.nnz;
    T.rp.free(); T.ci.free(); T.v.free();
    CsrOwned Tn;
    SegFilterOut fo = filter_seg(Tt.view(), eg, fixed, o.e_r, o.max_filter_iters, inst, seg, count, s, Tn, hs);
    sexpm_step_stats rec;
    std::memset(&rec, 0, sizeof(rec));
    rec.phase = 1;
    rec.i = g;
    for (int b = 0; b < count; ++b) {
      rec.iters = std::max(rec.iters, fo.iters[b]);
      if (fixed[b] < 0.0) {
        rec.t = std::max(rec.t, fo.t[b]);
        rec.eps_g = std::max(rec.eps_g, eg[b]);
      }
    }
    rec.nnz_raw = Tt.nnz;
    rec.nnz = Tn.nnz;
    rec.products = prod;
    rec.products_done = done;
    rec.ms_symbolic = tm.ms_symbolic;
    rec.ms_numeric = tm.ms_numeric;
    rec.ms_filter = fo.ms;
    rec.flops = flops;
    Tt.rp.free(); Tt.ci.free(); Tt.v.free();
    T = std::move(Tn);
    rec.ms = ts.ms();
    steps.push_back(rec);
  }
  const double ms_squaring = t_sq.ms();
  // step 5: e^{tau_b H_b} = I + T^_{N_b}, then one result per instance
  Timer t_fin(s);
  CsrOwned E;
  if (graph_result) {
    T.rp.free(); T.ci.free(); T.v.free();  // the Taylor phase's T^_0
    // T^_N is in the arena.  An arena above a quarter of the device's memory makes room for the
    // result: its other buffers go first, then T^ (the next compute allocates the sizes of this
    // one at once and captures the step again); a smaller one stays, with its graph, for the
    // next compute.
    size_t fr = 0, tot = 0;
    SX_CUDA(cudaMemGetInfo(&fr, &tot));
    const bool big = gout.arena_bytes > (int64_t)(tot / 4);
    if (big) graph_squaring_release(p->graph, true);
    add_identity(gout.T, s, E, hs);
    if (big) graph_squaring_release(p->graph, false);
  } else {
    add_identity(T.view(), s, E, hs);
    T.rp.free(); T.ci.free(); T.v.free();
  }
  gather_row_ptr(E.rp.p, seg, count, bnd.data(), s);
  std::vector<sexpm_result*> res(count, nullptr);
  try {
    for (int b = 0; b < count; ++b) {
      res[b] = new sexpm_result();
      res[b]->s = s;
      block_get(E.view(), p->row0[b], p->row0[b + 1] - p->row0[b], bnd[b + 1] - bnd[b], res[b]->E, s);
    }
    SX_CUDA(cudaStreamSynchronize(s));
    const double ms_final = t_fin.ms();
    const double ms_total = t_all.ms();
    for (int b = 0; b < count; ++b) {
      sexpm_stats_t& st = res[b]->st;
      std::memset(&st, 0, sizeof(st));
      st.n = p->row0[b + 1] - p->row0[b];
      st.norm_H = normH[b];
      st.M = M[b];
      st.N = N[b];
      st.normal = (p->normal_b[b] != 0 || normH[b] == 0.0) ? 1 : 0;
      st.symmetric = sym ? 1 : 0;
      st.a = M[b] ? a[b] : 0.0;
      st.r0 = r0[b];
      st.eps_g0 = eps_g0[b];
      st.nnz_out = res[b]->E.nnz;
      st.ms_total = ms_total;
      st.ms_taylor = ms_taylor;
      st.ms_squaring = ms_squaring;
      st.ms_final = ms_final;
      st.peak_bytes = Pool::peak() - live0;
      st.launches = launches() - launches0;
      res[b]->steps = steps;
      st.n_steps = (int32_t)steps.size();
    }
  } catch (...) {
    for (auto* r : res) delete r;
    throw;
  }
  for (int b = 0; b < count; ++b) outs[b] = res[b];
  SX_API_END
}

int sexpm_batched_graph_info(const sexpm_plan_t* p, int64_t* arena_bytes, int32_t* captures, int32_t* reruns,
                             int32_t* host_steps, int64_t* kernels_per_step, int64_t* kernels_per_pass) {
  SX_API_BEGIN
  if (!p) fail(SEXPM_EINVAL, "null plan");
  graph_squaring_info(p->graph, arena_bytes, captures, reruns, host_steps, kernels_per_step, kernels_per_pass);
  SX_API_END
}

int sexpm_tune_batched(sexpm_plan_t* p, const double* taus, int32_t ncand, const int32_t* ks_bytes,
                       const int32_t* wide, double* ms_out, int32_t* best) {
  SX_API_BEGIN
  if (!p || !taus) fail(SEXPM_EINVAL, "null argument");
  if (p->count == 0) fail(SEXPM_EINVAL, "the tuner takes a batched plan");
  if (p->opt.batched_graph == 0) fail(SEXPM_EINVAL, "the tuner sets the layout of the captured step (batched_graph = 1)");
  if (ncand < 0 || (ncand > 0 && (!ks_bytes || !wide))) fail(SEXPM_EINVAL, "bad candidate list");
  static const int32_t kKs[4] = {225280, 112640, 0, 225280};
  static const int32_t kWide[4] = {1, 1, 1, 0};
  const int nc = ncand ? ncand : 4;
  const int32_t* ks = ncand ? ks_bytes : kKs;
  const int32_t* wd = ncand ? wide : kWide;
  for (int c = 0; c < nc; ++c)
    if (ks[c] < 0 || ks[c] > (1 << 20) || (wd[c] != 0 && wd[c] != 1)) fail(SEXPM_EINVAL, "bad candidate");
  const int32_t ks0 = p->layout_ks, w0 = p->layout_wide;
  std::vector<sexpm_result_t*> outs(p->count, nullptr);
  double best_ms = std::numeric_limits<double>::infinity();
  int bi = 0;
  for (int c = 0; c < nc; ++c) {
    p->layout_ks = ks[c];
    p->layout_wide = wd[c];
    const int rc = sexpm_compute_batched(p, taus, outs.data());
    if (rc != SEXPM_OK) {
      p->layout_ks = ks0;
      p->layout_wide = w0;
      return rc;
    }
    const double ms = outs[0]->st.ms_squaring;
    for (auto*& r : outs) {
      sexpm_result_free(r);
      r = nullptr;
    }
    if (ms_out) ms_out[c] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      bi = c;
    }
  }
  p->layout_ks = ks[bi];
  p->layout_wide = wd[bi];
  if (best) *best = bi;
  SX_API_END
}

int sexpm_forward_keep(sexpm_plan_t* p, double tau, int32_t ckpt_stride, sexpm_result_t** expm_out,
                       sexpm_tape_t** tape) {
  SX_API_BEGIN
  if (!p || !tape) fail(SEXPM_EINVAL, "null argument");
  *tape = nullptr;
  if (expm_out) *expm_out = nullptr;
  if (p->count > 0) fail(SEXPM_EINVAL, "the adjoint takes a plain (non-batched) plan");
  if (p->cplx) fail(SEXPM_EINVAL, "the adjoint takes a real plan");
  if (ckpt_stride < 0) fail(SEXPM_EINVAL, "ckpt_stride must be >= 0");
  sexpm_tape_t* t = new sexpm_tape_t();
  sexpm_result* fwd = new sexpm_result();
  try {
    t->plan = p;
    t->tau = tau;
    t->rec.stride = ckpt_stride;
    // forward with every product formed (the reverse pass differentiates exactly this map)
    compute_impl(p, tau, fwd, &t->rec, false);
    t->st = fwd->st;
    t->steps = fwd->steps;
  } catch (...) {
    delete t;
    delete fwd;
    throw;
  }
  *tape = t;
  if (expm_out) *expm_out = fwd; else delete fwd;
  SX_API_END
}

int sexpm_adjoint_tape(sexpm_tape_t* t, const sexpm_csr_view* W, sexpm_result_t** dH) {
  SX_API_BEGIN
  if (!t || !W || !dH) fail(SEXPM_EINVAL, "null argument");
  *dH = nullptr;
  if (W->n != t->plan->H.n) fail(SEXPM_EINVAL, "W must have the dimension of H");
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (dev != t->plan->device) fail(SEXPM_EINVAL, "current device differs from the plan's device");
  sexpm_result* res = new sexpm_result();
  try {
    res->st = t->st;
    res->steps = t->steps;
    res->st.ms_total = t->st.ms_total + reverse_pass(t->plan, t->rec, t->tau, W, res);
    res->st.nnz_out = res->E.nnz;
  } catch (...) {
    delete res;
    throw;
  }
  *dH = res;
  SX_API_END
}

void sexpm_tape_free(sexpm_tape_t* t) { delete t; }

int sexpm_adjoint(sexpm_plan_t* p, double tau, const sexpm_csr_view* W, int32_t ckpt_stride, sexpm_result_t** dH,
                  sexpm_result_t** expm_out) {
  if (!p || !W || !dH) {
    set_last_error("null argument");
    return SEXPM_EINVAL;
  }
  *dH = nullptr;
  if (expm_out) *expm_out = nullptr;
  if (W->n != p->H.n) {
    set_last_error("W must have the dimension of H");
    return SEXPM_EINVAL;
  }
  sexpm_tape_t* tape = nullptr;
  int rc = sexpm_forward_keep(p, tau, ckpt_stride, expm_out, &tape);
  if (rc != SEXPM_OK) return rc;
  rc = sexpm_adjoint_tape(tape, W, dH);
  sexpm_tape_free(tape);
  if (rc != SEXPM_OK && expm_out && *expm_out) {
    sexpm_result_free(*expm_out);
    *expm_out = nullptr;
  }
  return rc;
}

}  // extern "C"
