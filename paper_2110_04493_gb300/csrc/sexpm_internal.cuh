// Internal declarations shared by the translation units of libsexpm.
// Device CSR layout: int64 row pointers, int32 sorted column indices, float64 values.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sexpm.h"

namespace sexpm {

// Non-owning device CSR view used by the kernels.
struct CsrD {
  int64_t n = 0;
  int64_t nnz = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* v = nullptr;
};

// Error carried from deep inside the host driver up to the C ABI.
struct Error {
  int code;
  std::string msg;
};

void set_last_error(const std::string& msg);
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define SX_CUDA(x) ::sexpm::check_cuda((x), #x)

// ---------------------------------------------------------------- device memory
// Stream-ordered allocations from a library-owned pool.  Tracks live and peak bytes.
struct Pool {
  static void* alloc(size_t bytes, cudaStream_t s);
  static void release(void* p, size_t bytes, cudaStream_t s);
  static int64_t live();
  static int64_t peak();
  static void reset_peak();
};

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t count = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(size_t n, cudaStream_t st) { reset(n, st); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), count(o.count), s(o.s) { o.p = nullptr; o.count = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      free();
      p = o.p; count = o.count; s = o.s;
      o.p = nullptr; o.count = 0;
    }
    return *this;
  }
  ~DevBuf() { free(); }
  void reset(size_t n, cudaStream_t st) {
    free();
    s = st;
    count = n;
    p = n ? static_cast<T*>(Pool::alloc(n * sizeof(T), st)) : nullptr;
  }
  void free() {
    if (p) Pool::release(p, count * sizeof(T), s);
    p = nullptr;
    count = 0;
  }
};

// An owned device CSR matrix.
struct CsrOwned {
  int64_t n = 0;
  int64_t nnz = 0;
  DevBuf<int64_t> rp;
  DevBuf<int32_t> ci;
  DevBuf<double> v;
  CsrD view() const {
    CsrD d;
    d.n = n; d.nnz = nnz; d.rp = rp.p; d.ci = ci.p; d.v = v.p;
    return d;
  }
};

// Per-row statistics written by the numeric product kernel.
struct RowStats {
  DevBuf<double> sq;    // sum of v^2 over the row
  DevBuf<double> diag;  // value stored at (i, i), 0 if absent
};

// Small pinned host buffer used to read back scalars.
struct HostScalars {
  double* d = nullptr;
  int64_t* i = nullptr;
  HostScalars();
  ~HostScalars();
};

// Number of kernels this library has enqueued (all launchers add to it).
// Runs set() once per CUDA device for this flag set (the current device; devices 0..63), for
// per-device settings such as a kernel's shared-memory limit (cudaFuncSetAttribute applies to
// the current device only).  Thread-safe; a device counts as done only once set() returned.
int current_device();
std::mutex& device_setup_mutex();
template <typename F>
void once_per_device(bool (&done)[64], F set) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(device_setup_mutex());
  if (done[dev]) return;
  set();
  done[dev] = true;
}
void count_launches(int64_t k);
int64_t launches();

// Device times of the phases of one sparse product (filled when requested).
struct SpgemmTimes {
  double ms_symbolic = 0.0;  // analysis, classification and the symbolic pass
  double ms_numeric = 0.0;   // the numeric pass (products, fused scaling and beta D)
};

// Word pattern of a CSR matrix: row r touches the 32-column words wi[rp[r] .. rp[r+1]) with the
// column bits wb[...] inside each word.
struct WPat {
  const int64_t* rp = nullptr;
  const int32_t* wi = nullptr;
  const uint32_t* wb = nullptr;
};

// Symbolic phase of a sparse product C = (A B)/div + beta D, kept so that the numeric phase can
// run on row ranges: word patterns of B (and D), per-row column span, per-row entry counts, the
// row pointers of the unfiltered C, and the per-class row lists and counters.
constexpr int kProductClasses = 6;
struct ProductSym {
  int64_t n = 0, products = 0, nnz = 0;
  bool upper = false, hasD = false, sameD = false;
  int ks_bytes = 0;
  const uint8_t* frozen = nullptr;
  const int32_t* sched = nullptr;
  DevBuf<int64_t> wB_rp, wD_rp;
  DevBuf<int32_t> wB_wi, wD_wi;
  DevBuf<uint32_t> wB_wb, wD_wb;
  DevBuf<int32_t> base, words, cnt, cnt_up, lists;
  DevBuf<int64_t> rp;              // n + 1 row pointers of the unfiltered C
  const int64_t* rp_ext = nullptr; // set when rp has been handed to an owner of C
  DevBuf<unsigned long long> ctr, row_ctr;
  int64_t rows_symbolic[kProductClasses] = {};  // rows per size class (symbolic pass)
  int64_t rows_numeric[kProductClasses] = {};   // rows per size class, summed over numeric calls
  const int64_t* row_ptr() const { return rp_ext ? rp_ext : rp.p; }
  WPat wpat_B() const {
    WPat w;
    w.rp = wB_rp.p; w.wi = wB_wi.p; w.wb = wB_wb.p;
    return w;
  }
  WPat wpat_D() const {
    if (!hasD) return WPat();
    if (sameD) return wpat_B();
    WPat w;
    w.rp = wD_rp.p; w.wi = wD_wi.p; w.wb = wD_wb.p;
    return w;
  }
};

// ---------------------------------------------------------------- kernels (launchers)
// All launchers enqueue on stream s and do not synchronise unless stated.

// Symbolic phase of C = (A B)/div + beta D (D.n == 0: absent): word patterns, row analysis,
// size classes, per-row counts (and upper-part counts when upper) and the row pointers ps.rp;
// allocates stats (n rows) when given and zeroes the statistics of empty rows.  Synchronises s.
void product_symbolic(const CsrD& A, const CsrD& B, const CsrD& D, bool upper, const uint8_t* frozen,
                      const int32_t* sched, RowStats* stats, cudaStream_t s, HostScalars& hs, ProductSym& ps);
// Numeric phase for the rows [r0, r1): row i is written to ci_out/v_out at ps.row_ptr()[i] - out_base
// (upper mode: the values below the diagonal are left for a mirror step).  Fills the statistics of
// those rows.  Returns the products formed.  Synchronises s.
int64_t product_numeric(ProductSym& ps, const CsrD& A, const CsrD& B, const CsrD& D, double div, double beta,
                        int64_t r0, int64_t r1, int64_t out_base, int32_t* ci_out, double* v_out, RowStats* stats,
                        cudaStream_t s, HostScalars& hs);
// Fills the values below the diagonal of a symmetric product from their mirror entries.
void mirror_lower(const CsrOwned& C, cudaStream_t s, HostScalars& hs);

// C = (A B) / div + beta D.  D may have n == 0 (absent).  Allocates C; fills row
// statistics (sum of squares, diagonal) when stats != nullptr.  Synchronises s
// to size C.  Returns the number of scalar products.
// upper: A, B and D are symmetric (so is C); only the products at columns >= row are
// formed and the entries below the diagonal are copied from their mirror entries.
// done (optional) receives the number of products actually formed.
// frozen (optional, one byte per row): rows with frozen[i] != 0 form no products and are a plain
// copy of D_i (used by the batched method for instances that have finished their squarings).
// sched (optional, n row ids): the order in which rows are handed to the thread blocks (a
// permutation chosen for cache locality; results do not depend on it).
// rows_class (optional, kProductClasses entries) receives the rows of the numeric pass per size class.
int64_t spgemm(const CsrD& A, const CsrD& B, const CsrD& D, double div, double beta, cudaStream_t s,
               CsrOwned& C, RowStats* stats, HostScalars& hs, SpgemmTimes* times = nullptr, bool upper = false,
               int64_t* done = nullptr, const uint8_t* frozen = nullptr, const int32_t* sched = nullptr,
               int64_t* rows_class = nullptr);

// sum_i x[i] over n doubles, deterministic order.  Synchronises and returns the sum.
double reduce_sum(const double* x, int64_t n, cudaStream_t s, HostScalars& hs);
// sum over the stored values of A of v^2.
double sum_squares(const CsrD& A, cudaStream_t s, HostScalars& hs);

// Exclusive scan of int32 counts into int64 row pointers (n+1 entries).  Returns the total
// (synchronises s).
int64_t scan_counts(const int32_t* cnt, int64_t n, int64_t* rp, cudaStream_t s, HostScalars& hs);

// C = A + beta B (union pattern).
void add(const CsrD& A, const CsrD& B, double beta, cudaStream_t s, CsrOwned& C, HostScalars& hs);

// C = I + A (diagonal inserted where absent).
void add_identity(const CsrD& A, cudaStream_t s, CsrOwned& C, HostScalars& hs);

// y[k] = alpha x[k] (values only).
void scale_values(const double* x, double alpha, int64_t n, double* y, cudaStream_t s);

// S = (A + A^T)/2 (pattern of A plus the mirrors of entries whose mirror is absent).
void symmetric_part(const CsrD& A, cudaStream_t s, CsrOwned& S, HostScalars& hs);

// A^T into T (columns sorted within rows).
void transpose(const CsrD& A, cudaStream_t s, CsrOwned& T, HostScalars& hs);

// Pattern and values of A and B equal (sign = +1) or B = -A (sign = -1)?  Synchronises s.
bool csr_equal(const CsrD& A, const CsrD& B, double sign, cudaStream_t s, HostScalars& hs);

// Validation on device: sorted unique in-range columns, finite values, monotone row_ptr.
bool csr_valid(const CsrD& A, cudaStream_t s, HostScalars& hs);

// ---------------------------------------------------------------- Algorithm 4.1 over row pieces
// A block of rows [r0, r1) of a sparse matrix with local row pointers (rp[0] = 0, r1 - r0 + 1
// entries, rp[r1 - r0] = nnz).  A whole matrix is one piece (r0 = 0, r1 = n).
struct Piece {
  int64_t r0 = 0, r1 = 0, nnz = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* v = nullptr;
};

// Tiles of the flat filter kernels covering nnz entries, and their kept counts (one per warp
// of a tile).
int64_t tiles_of(int64_t nnz);
int64_t counts_of(int64_t nnz);
// One Algorithm 4.1 pass over all pieces: returns sum_{|v| <= t} v^2 and writes the kept
// counts (|v| > t) of every tile and warp (piece p's counts start at tile_cnt + tile_base[p],
// tile_base in units of counts_of).  Synchronises s.
double pass_pieces(const std::vector<Piece>& P, const std::vector<int64_t>& tile_base, double t, int32_t* tile_cnt,
                   cudaStream_t s, HostScalars& hs);
// Compaction of the entries |v| > t of all pieces into out (rows 0..n-1; out.rp/ci/v allocated);
// tile_off = exclusive scan of the counts of the last pass (total at tile_off[total counts]).
void compact_pieces(const std::vector<Piece>& P, const std::vector<int64_t>& tile_base, double t,
                    const int64_t* tile_off, int64_t n, CsrOwned& out, cudaStream_t s);
// Exact streaming step of a row chunk [r0, r1) of an unfiltered product (row i at
// rp[i] - base of ci/v): per-row kept counts at the lower bound L (keep, r1 - r0 entries) and the
// returned sum of squares of the dropped entries; in the symmetric mode lower entries take their
// mirror's value and decision (same chunk, or the earlier device pieces).  Synchronises s.
double drop_rows(int64_t r0, int64_t r1, const int64_t* rp, int64_t base, const int32_t* ci, double* v, bool sym,
                 double L, const Piece* pieces, int npieces, int32_t* keep, cudaStream_t s, HostScalars& hs);
// sum over the rows r0 <= i < r1 of sum_j (delta_ij + a_ij)^2.  Synchronises s.
double norm2_I_plus_rows(const CsrD& A, int64_t r0, int64_t r1, cudaStream_t s, HostScalars& hs);
// Copies the entries drop_rows kept into a piece (out_rp: scanned keep, r1 - r0 + 1 entries).
void compact_rows(int64_t r0, int64_t r1, const int64_t* rp, int64_t base, const int32_t* ci, const double* v, bool sym,
                  double L, const int64_t* out_rp, int32_t* out_ci, double* out_v, cudaStream_t s);

// h_{M1,Np} of Sec. 4.2 from pnorms[k-1] = ||H^k|| (k <= kmax); -1 when kmax < 2 M1 + 1.
double h_refined(const double* pnorms, int32_t kmax, int32_t M1, int32_t Np);

// Y = A X (X, Y device, n x r row-major, no overlap).
void spmm(const CsrD& A, const double* X, int64_t r, double* Y, cudaStream_t s);

// ---------------------------------------------------------------- batched (block-diagonal) helpers
// inst[i]: instance of row i; seg[b] .. seg[b+1]: rows of instance b (device arrays).

// sums_host[b] = sum over instance b's rows of x (device x; synchronises s).
void seg_sums(const double* x, const int64_t* seg, int count, double* out_host, cudaStream_t s);
// Algorithm 4.1 pass with thresholds t_inst[b] (device): keep[i] and per-instance sums.
void filter_pass_seg(const CsrD& A, const int32_t* inst, const double* t_inst, int32_t* keep, double* row_part,
                     const int64_t* seg, int count, double* sums_host, cudaStream_t s);
void compact_seg(const CsrD& A, const int32_t* inst, const double* t_inst, CsrOwned& C, cudaStream_t s);
void scale_rows(const CsrD& A, const int32_t* inst, const double* factor, double* out_v, cudaStream_t s);
void instance_of_row(const int64_t* seg, int count, int64_t n, int32_t* inst, cudaStream_t s);
void row_flags(const int32_t* inst, const uint8_t* inst_flag, int64_t n, uint8_t* row_flag, cudaStream_t s);
void block_put(const CsrD& X, int64_t row0, int64_t nnz0, int64_t* rp, int32_t* ci, double* v, cudaStream_t s);
void block_get(const CsrD& E, int64_t row0, int64_t nb, int64_t nnz_b, CsrOwned& out, cudaStream_t s);
void gather_row_ptr(const int64_t* rp, const int64_t* seg, int count, int64_t* out_host, cudaStream_t s);

// Device-only forms for a step whose sizes are decided on the device (the captured batched
// squaring step): no host read-back, grids independent of the data.
int64_t scan_tiles(int64_t n);  // int64 scratch values scan_counts_dev needs
// Exclusive scan into rp (n + 1 entries; the total stays on the device at rp[n]).
void scan_counts_dev(const int32_t* cnt, int64_t n, int64_t* rp, int64_t* ts, cudaStream_t s);
// out[b] = sum over instance b's rows of x (device out).
void seg_sums_dev(const double* x, const int64_t* seg, int count, double* out, cudaStream_t s);
// One Algorithm 4.1 pass with thresholds t_inst[b]: keep[i], row_part[i]; skipped while *status != 0.
void filter_pass_seg_dev(const CsrD& A, const int32_t* inst, const double* t_inst, int32_t* keep, double* row_part,
                         const int32_t* status, cudaStream_t s);
// A~ = A - b_n into rp_out/ci_out/v_out; skipped while *status != 0.
void compact_seg_dev(const CsrD& A, const int32_t* inst, const double* t_inst, const int64_t* rp_out, int32_t* ci_out,
                     double* v_out, const int32_t* status, cudaStream_t s);

// C = A + beta B into rp_out/ci_out/v_out (capacity cap): when the sum does not fit, status
// gets `bit` and nothing is written; nothing runs while the status is set.
void add_dev(const CsrD& A, const CsrD& B, double beta, int32_t* cnt, int64_t* rp_out, int64_t* ts, int32_t* ci_out,
             double* v_out, int64_t cap, int32_t* status, unsigned long long* need, int32_t bit, cudaStream_t s);

// Status bits of a device-sized step.
constexpr int32_t kStProduct = 1;   // the unfiltered product exceeded its capacity
constexpr int32_t kStFiltered = 2;  // the filtered product exceeded its capacity
constexpr int32_t kStMirror = 4;    // symmetric mode: an entry without its mirror partner
constexpr int32_t kStNoConv = 8;    // Algorithm 4.1 reached its iteration cap
constexpr int32_t kStBound = 16;    // a row exceeded the scratch bound of its size class
constexpr int32_t kStWords = 32;    // the word pattern of B exceeded its capacity
constexpr int32_t kStSum = 64;      // a sum (T^_0 + S^_i) exceeded its capacity

// Buffers of C = (A B)/div + beta D formed with sizes decided on the device: every buffer is
// allocated beforehand (capacities in entries), B and D share one pattern (D is B or absent).
struct DevProduct {
  int64_t n = 0;
  int64_t* wrp = nullptr;           // word pattern of B: n + 1 row pointers,
  int32_t* wi = nullptr;            // word indices and
  uint32_t* wb = nullptr;           // masks (wcap words)
  int64_t wcap = 0;
  int32_t *base = nullptr, *words = nullptr, *cnt = nullptr, *cnt_up = nullptr;  // per row
  int32_t* lists = nullptr;         // kProductClasses x n row lists
  int64_t* flops = nullptr;         // per row
  unsigned long long* ctr = nullptr;      // 2 (2 kProductClasses + 4) counters: symbolic half, numeric half
  unsigned long long* row_ctr = nullptr;  // 2 kProductClasses
  int64_t* scan_ts = nullptr;       // scan_tiles(n)
  uint32_t* gs_sym = nullptr;       // global-class scratch of the symbolic pass (gs_sym_grid blocks)
  int64_t gs_sym_stride = 0, gs_sym_grid = 0;   // (uint32 words per block)
  unsigned char* gs_num = nullptr;  // global-class scratch of the numeric pass
  int64_t gs_num_stride = 0, gs_num_grid = 0;   // (bytes per block)
  int64_t* rp_out = nullptr;        // n + 1
  int32_t* ci_out = nullptr;
  double* v_out = nullptr;
  int64_t cap_out = 0;
  double *row_sq = nullptr, *row_diag = nullptr;  // per-row statistics of the product
  int32_t* status = nullptr;        // kSt* bits (sticky)
  unsigned long long* need = nullptr;    // largest unfiltered size requested
  unsigned long long* need_w = nullptr;  // largest word pattern requested
  int ks_bytes = 0;
  bool wide = true;
  int64_t grid_sym[kProductClasses] = {}, grid_num[kProductClasses] = {};  // set by dev_product_prepare
  bool prepared = false;
};
// Scratch sizes of the global-memory class for rows of instances with at most n_max rows.
void dev_product_scratch(int64_t n_max, int ks_bytes, bool wide, int64_t& sym_stride, int64_t& sym_grid,
                         int64_t& num_stride, int64_t& num_grid);
// Launch shapes of dev_product (occupancy queries and shared-memory limits, done before any
// capture).
void dev_product_prepare(DevProduct& P);
// Enqueues the whole product (word pattern, analysis, classes, symbolic, scan, capacity checks,
// numeric, mirror) on s without reading anything back: when a size exceeds its capacity the
// numeric pass forms nothing and status gets the matching bit.
void dev_product(const CsrD& A, const CsrD& B, bool hasD, double div, double beta, bool upper, const uint8_t* frozen,
                 const DevProduct& P, cudaStream_t s);
// Index of the products counter (symbolic half) and of the formed-products counter (numeric
// half) in DevProduct::ctr.
int dev_product_products_index();
int dev_product_formed_index();
// Accumulation layout defaults of the numeric pass (k-split byte budget, wide blocks for the
// global-memory class), from the environment when set.
int default_ks_bytes();
bool default_wide_blocks();

// ---------------------------------------------------------------- captured batched squarings
// The squaring phase of a batched plan replayed as one captured CUDA graph per step (sizes
// decided on the device, Algorithm 4.1 in a conditional WHILE node, a fixed-capacity arena that
// is grown when a product does not fit, the run resuming at that step).
struct GraphSquaring;
struct GraphSquaringIn {
  int count = 0;
  int64_t n = 0;          // rows of the batch
  int64_t n_max = 0;      // rows of its largest instance
  int64_t dense = 0;      // sum of n_b^2 (no product is larger)
  int64_t arena_bytes = 0;  // first arena budget (0: small, grown by the run)
  const int32_t* inst = nullptr;  // device: instance of each row
  const int64_t* seg = nullptr;   // device: first row of each instance (count + 1)
  std::vector<int32_t> N;         // squarings per instance
  std::vector<double> a, r0, nb;  // a_b, r_0,b and n_b per instance
  bool sym = false, square_scale = true;
  double e_r = 0.1;
  int max_iters = 100;
  // Taylor phase (graph_taylor): degree M_b and threshold eps_g^(0) per instance
  std::vector<int32_t> M;
  std::vector<double> eps_g0;
};
struct GraphSquaringOut {
  CsrD T;                 // T^ after steps_done squarings (block diagonal), in the arena
  int steps_done = 0;     // squarings completed by the graph (all of them unless the arena ran out)
  std::vector<sexpm_step_stats> steps;
  int reruns = 0;
  int64_t launches = 0;
  int64_t arena_bytes = 0;
};
GraphSquaring* graph_squaring_new();
void graph_squaring_free(GraphSquaring* G);
// Frees the arena's T~ and word pattern, and T^ unless keep_T (the graph is captured again on
// the next run, which allocates the sizes of this one at once).
void graph_squaring_release(GraphSquaring* G, bool keep_T);
// Arena bytes, graph captures, resumed steps after an arena overflow, squaring steps left to the
// host-driven launches (device memory ran out), kernels per step outside the Algorithm 4.1 loop
// and kernels per pass of that loop.
void graph_squaring_info(const GraphSquaring* G, int64_t* arena_bytes, int32_t* captures, int32_t* reruns,
                         int32_t* host_steps, int64_t* kernels_per_step, int64_t* kernels_per_pass);
void graph_squaring_note_host_steps(GraphSquaring* G, int steps);
// Accumulation layout of the numeric pass (ks_bytes < 0 / wide < 0: the defaults).
void graph_squaring_set_layout(GraphSquaring* G, int ks_bytes, int wide);
// Runs the squarings from T^_0 (T0, device, block diagonal).  Orders itself after s and s after it.
void graph_squarings(GraphSquaring* G, const CsrD& T0, const GraphSquaringIn& in, GraphSquaringOut& out,
                     cudaStream_t s);
// The Taylor phase (Algorithm 4.2 step 3 for every instance) as one captured graph per term:
// from H_0 (device, block diagonal), T^_0 = H_0 + sum_i S^_i into out.T (in the arena, valid
// until the next run); out.steps are the terms' records (phase 0).  Orders itself after s and s
// after it.  Requires max M_b <= 128.
void graph_taylor(GraphSquaring* G, const CsrD& H0, const GraphSquaringIn& in, GraphSquaringOut& out,
                  cudaStream_t s);

// ---------------------------------------------------------------- complex H
// Z = X + iY through the real embedding R(Z) = X (x) I_2 + Y (x) J; the method keeps its n even
// rows (row i: the pairs (2j: Re z_ij, 2j + 1: -Im z_ij), 2n columns).  Complex values are
// (re, im) pairs of doubles.  ("top rows" below are these even rows.)
// Input check: sorted unique columns in [0, n), finite values, monotone row pointers.  Syncs s.
bool valid_complex(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* vz, cudaStream_t s,
                   HostScalars& hs);
// Top rows of R(Z) from a complex CSR (device arrays).
void embed_top(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* vz, cudaStream_t s,
               CsrOwned& top);
// All 2n rows of R(Z) from its even rows (rows 2i and 2i + 1).
void block_mirror(const CsrD& top, int64_t n, cudaStream_t s, CsrOwned& full);
// Algorithm 4.1 pass deciding by |z| (pairs of columns 2j, 2j + 1 of a row): returns the sum of
// squares of the dropped entries (= sum of |z|^2), per-row kept counts in keep.  Syncs s.
double pass_complex(const CsrD& top, int64_t n, double t, int32_t* keep, double* part, cudaStream_t s,
                    HostScalars& hs);
// The entries with |z| > t (keep: the counts of the pass at t).
void compact_complex(const CsrD& top, int64_t n, double t, const int32_t* keep, cudaStream_t s, CsrOwned& out,
                     HostScalars& hs);
// The identity in the even-row layout (row i: (2i: 1, 2i + 1: 0)).
void identity_pairs(int64_t n, cudaStream_t s, CsrOwned& I);
// sum_i Re z_ii of the even rows (the value at column 2i of row i).  Syncs s.
double trace_re(const CsrD& top, cudaStream_t s, HostScalars& hs);
// The complex matrix of top rows: pattern (rp, ci) and values vz (2 nnz doubles).
void extract_complex(const CsrD& top, int64_t n, cudaStream_t s, CsrOwned& pattern, DevBuf<double>& vz,
                     HostScalars& hs);

// ---------------------------------------------------------------- adjoint helpers
// out[p] = (accumulate ? out[p] : 0) + alpha sum_l A_il B_jl + beta A_ij for every stored (i, j)
// of P (out has P.nnz entries in P's order).
void sddmm(const CsrD& P, const CsrD& A, const CsrD& B, double alpha, double beta, bool accumulate, double* out,
           cudaStream_t s, HostScalars& hs);
// Sorts the columns (with their values) of every row in place.
void sort_rows(int64_t n, const int64_t* rp, int32_t* ci, double* v, cudaStream_t s);

}  // namespace sexpm
