// The batched method (Algorithm 4.2 steps 3 and 4 for every instance of a block-diagonal batch)
// as CUDA graphs: one squaring step -- T~_i = 2 T^_{i-1} + T^_{i-1}^2 for all instances, each
// instance's Algorithm 4.1 with its own bound eps_g^(i) = a_b 2^i r_0,b ||I + T~_i||_F, and the
// compaction -- is captured once and replayed N_max times with no host involvement between the
// steps; each Taylor term (S~_i = S^_{i-1} H_0 / i, Algorithm 4.1 with eps_g^(0), T^_0 += S^_i) is
// one captured graph of its own (the divisor i is a kernel argument), the same machinery.
//
//  * Sizes are decided on the device.  Every buffer lives in a device arena allocated
//    beforehand with fixed capacities (T^, the unfiltered T~, the word pattern of T^ and the
//    per-row work arrays).  The scans leave nnz(T~_i), nnz(T^_i) and the word count on the
//    device, and check kernels compare them with the capacities; a size that does not fit sets
//    a sticky status bit, the numeric pass forms nothing and every later kernel of the run
//    returns at once.  The host reads the status once, after the last step, grows the arena to
//    the size the device recorded and resumes at the step that did not fit (T^ of the step before
//    is still in the arena: a step that stops writes nothing back).
//  * The filtered T^_i is compacted into T^'s own arrays: T^_{i-1} is not read after the product.
//  * Launch shapes do not depend on the data: the row kernels are persistent over the size
//    classes' row lists (one launch per class, covering the rows of every instance in that
//    class, list lengths read on the device), with each class's full shared-memory budget.
//  * Algorithm 4.1 iterates inside the graph: a conditional WHILE node runs the pass (every
//    row, its instance's threshold), the per-instance sums and an update kernel that applies
//    the Algorithm 4.1 recurrence to every unconverged instance and sets the loop condition.
//    The update stops the loop at the iteration cap, so the loop always ends.
//  * Per step, records (products, sizes, thresholds, passes) are written on the device and read
//    after the run; events between the graph launches time each step.
// The arithmetic is the host-driven batched path's, kernel for kernel (same kernels, same
// reduction orders, same formula for the bounds), so the two give bit-identical results.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "sexpm_internal.cuh"

namespace sexpm {

// Device-side state of a run.
struct GState {
  int32_t g;        // squaring steps begun
  int32_t status;   // kSt* bits (sticky)
  int32_t loop;     // Algorithm 4.1 passes of the current step
  int32_t fail_g;   // first step that set the status (0: none)
  unsigned long long need_raw;  // largest unfiltered product requested (entries)
  unsigned long long need_out;  // largest filtered product requested (entries)
  unsigned long long need_w;    // largest word pattern requested (words)
  unsigned long long need_sum;  // largest T^_0 + S^_i requested (entries)
};

// One record per squaring step, written on the device.
struct GStepRec {
  unsigned long long products, formed, nnz_raw, nnz;
  double t_max, eps_max, b_max;
  int32_t iters_max, loops;
};

namespace {

// SEXPM_ARENA_LOG=1 in the environment: one line on stderr per arena growth.
bool arena_log() {
  const char* e = std::getenv("SEXPM_ARENA_LOG");
  return e && *e == '1';
}

constexpr int kRecCap = 128;  // step records kept (N_max is far below: N_0 + n_extra)

// g += 1; an instance with N_b < g has finished its squarings and is carried unchanged.
__global__ void k_g_begin(GState* st, int count, const int32_t* N, uint8_t* frozen) {
  __shared__ int g;
  if (threadIdx.x == 0) {
    g = st->g + 1;
    st->g = g;
    st->loop = 0;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < count; b += blockDim.x) frozen[b] = N[b] < g ? 1 : 0;
}

// Bound of every instance for this step (Sec. 4.2, relative reading): eps_g = a_b 2^g r_0,b
// ||I + T~||_F with ||I + T~||_F^2 = sum v^2 + n_b + 2 trace (square_scale = 1), or a_b 2^g r_0,b.
// The first pass uses t = eps_g; a finished instance keeps every nonzero (t = 0) and is not
// iterated.
__global__ void k_g_alg41_init(const GState* st, int count, const uint8_t* frozen, const double* a, const double* r0,
                               const double* nb, const double* sq, const double* tr, int square_scale, double* eps,
                               double* t, double* m, double* bval, int32_t* iters, int32_t* conv) {
  const int g = st->g;
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    iters[b] = 0;
    bval[b] = 0.0;
    if (frozen[b]) {
      conv[b] = 1;
      t[b] = 0.0;
      eps[b] = 0.0;
      continue;
    }
    double normF = 1.0;
    if (square_scale) {
      const double f2 = sq[b] + nb[b] + 2.0 * tr[b];
      normF = sqrt(f2 > 0.0 ? f2 : 0.0);
    }
    const double e = a[b] * ldexp(r0[b], g) * normF;
    eps[b] = e;
    m[b] = 1.0;
    t[b] = e;
    conv[b] = 0;
  }
}

// After a pass: for every unconverged instance b_n = sqrt(sum), m = b_n / t; converged when
// b_n <= eps_g (1 + e_r), else t = eps_g / m for the next pass (Algorithm 4.1).  Sets the WHILE
// node's condition: another pass while an instance is unconverged, the status is clear and the
// iteration cap is not reached.  One block.
__global__ void k_g_alg41_update(GState* st, int count, double e_r, int max_iters, const double* eps, double* t,
                                 double* m, const double* bsum, double* bval, int32_t* iters, int32_t* conv,
                                 cudaGraphConditionalHandle h) {
  volatile GState* vs = st;
  const bool ok = vs->status == 0;
  int again = 0;
  if (ok) {
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
      if (conv[b]) continue;
      const double bv = sqrt(bsum[b]);
      bval[b] = bv;
      m[b] = bv / t[b];
      iters[b] += 1;
      if (bv <= eps[b] * (1.0 + e_r)) {
        conv[b] = 1;
      } else if (iters[b] >= max_iters) {
        conv[b] = 1;
        atomicOr(&st->status, kStNoConv);
      } else {
        t[b] = eps[b] / m[b];
        again = 1;
      }
    }
  }
  again = __syncthreads_or(again);
  if (threadIdx.x == 0) {
    const int loop = vs->loop + 1;
    vs->loop = loop;
    const bool go = again && vs->status == 0 && loop < max_iters;
    cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// status |= kStFiltered when the filtered product does not fit; skipped once the status is set
// (the kept counts were not computed then).
__global__ void k_g_cap_check_out(GState* st, const int64_t* rp_n, int64_t cap) {
  if (st->status) return;
  const long long total = *rp_n;
  atomicMax(&st->need_out, (unsigned long long)total);
  if (total > cap) atomicOr(&st->status, kStFiltered);
}

// The filtered result was compacted into T^'s arrays: its row pointers become T^'s, when the
// step succeeded.
__global__ void k_g_row_ptrs(const GState* st, int64_t n, const int64_t* rpF, int64_t* rpT) {
  if (st->status) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) rpT[i] = rpF[i];
}

__device__ __forceinline__ double block_max_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x & 31) < nw ? red[threadIdx.x & 31] : 0.0;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Step record: sizes, products and the largest threshold, bound, b_n and pass count over the
// instances that squared in this step; the first step that set the status.  One block.
__global__ void k_g_record(GState* st, GStepRec* rec, int count, const unsigned long long* ctr, int products_idx,
                           int formed_idx, const int64_t* rpR_n, const int64_t* rpF_n, const uint8_t* frozen,
                           const double* eps, const double* t, const double* bval, const int32_t* iters) {
  __shared__ double red[32];
  double tm = 0.0, em = 0.0, bm = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    if (frozen[b]) continue;
    tm = fmax(tm, t[b]);
    em = fmax(em, eps[b]);
    bm = fmax(bm, bval[b]);
    im = fmax(im, (double)iters[b]);
  }
  tm = block_max_d(tm, red);
  em = block_max_d(em, red);
  bm = block_max_d(bm, red);
  im = block_max_d(im, red);
  const int g = st->g;
  if (threadIdx.x == 0 && st->status && st->fail_g == 0) st->fail_g = g;
  if (threadIdx.x == 0 && g >= 1 && g <= kRecCap) {
    GStepRec r;
    r.products = ctr[products_idx];
    r.formed = ctr[formed_idx];
    r.nnz_raw = (unsigned long long)*rpR_n;
    r.nnz = (unsigned long long)*rpF_n;
    r.t_max = tm;
    r.eps_max = em;
    r.b_max = bm;
    r.iters_max = (int32_t)im;
    r.loops = st->loop;
    rec[g - 1] = r;
  }
}

// Taylor term i: an instance whose series has ended (an empty S^ term) or whose degree M_b is
// below i forms nothing this step.
__global__ void k_t_begin(GState* st, int i, int count, const int32_t* M, const uint8_t* done, uint8_t* frozen) {
  if (threadIdx.x == 0) {
    st->g = i;
    st->loop = 0;
  }
  for (int b = threadIdx.x; b < count; b += blockDim.x) frozen[b] = (done[b] || i > M[b]) ? 1 : 0;
}

// Taylor bound of every instance (eps_g^(0), Eq. 4.14); an instance that forms nothing drops
// everything (t = +inf) and is not iterated.
__global__ void k_t_alg41_init(int count, const uint8_t* frozen, const double* eps0, double* eps, double* t,
                               double* m, double* bval, int32_t* iters, int32_t* conv) {
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    iters[b] = 0;
    bval[b] = 0.0;
    if (frozen[b]) {
      conv[b] = 1;
      t[b] = __longlong_as_double(0x7ff0000000000000ll);
      eps[b] = 0.0;
    } else {
      eps[b] = eps0[b];
      m[b] = 1.0;
      t[b] = eps0[b];
      conv[b] = 0;
    }
  }
}

// After the term: an instance whose S^_i has no entry ends its series.
__global__ void k_t_done(const GState* st, int count, const int64_t* seg, const int64_t* rpS, uint8_t* done) {
  if (st->status) return;
  for (int b = threadIdx.x; b < count; b += blockDim.x)
    if (rpS[seg[b + 1]] == rpS[seg[b]]) done[b] = 1;
}

// T^_0 <- the sum T^_0 + S^_i (row pointers and entries), when the step succeeded.
__global__ void k_t_copy(const GState* st, int64_t n, const int64_t* rpN, const int32_t* ciN, const double* vN,
                         int64_t* rpT, int32_t* ciT, double* vT) {
  if (st->status) return;
  const int64_t nnz = rpN[n];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = t0; i <= n; i += stride) rpT[i] = rpN[i];
  for (int64_t q = t0; q < nnz; q += stride) {
    ciT[q] = ciN[q];
    vT[q] = vN[q];
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

struct GraphSquaring {
  int device = -1;
  // what the arena and the captured graph were made for
  int count = 0;
  int64_t n = 0, n_max = 0;
  bool sym = false, square_scale = true;
  double e_r = 0.0;
  int max_iters = 0;
  const int32_t* inst = nullptr;
  const int64_t* seg = nullptr;
  int ks_bytes = -1;  // accumulation layout of the numeric pass (-1: the library default)
  int wide = -1;
  int64_t capT = 0, capR = 0, capW = 0;        // capacities allocated now
  int64_t hintT = 0, hintR = 0, hintW = 0;     // capacities of the last run, for the next one
  // streams, events, graph
  cudaStream_t gs = nullptr, gs2 = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaEvent_t> ev_step;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t k_outer = 0, k_body = 0;  // kernels per step outside / inside the Algorithm 4.1 loop
  int captures = 0, reruns = 0, host_steps = 0;
  // Taylor phase: H_0, S^ (capS; the filtered term is compacted into it), T^_0 and the sum
  // T^_0 + S^_i (capT0 each); one graph per term (index i)
  int64_t capS = 0, capT0 = 0, capH = 0;
  DevBuf<int64_t> rpH, rpS, rpSN, rpT0, rpTN;
  DevBuf<int32_t> ciH, ciS, ciSN, ciT0, ciTN, Mb;
  DevBuf<double> vH, vS, vSN, vT0, vTN, eps0;
  int t_captures = 0, t_reruns = 0;
  int64_t t_outer = 0, t_body = 0;  // kernels per Taylor term outside / inside its Algorithm 4.1 loop
  DevBuf<uint8_t> done;
  DevBuf<GStepRec> recT;
  std::vector<cudaGraph_t> tgraph;
  std::vector<cudaGraphExec_t> texec;
  int t_captured_for = 0;  // the M_max the Taylor graphs were captured for (0: none)
  bool parked = false;  // T^'s entries are in T~'s buffers (while T^ is reallocated)
  // arena
  DevBuf<int64_t> rpT, rpR, rpF, wrp, flops, scan_ts;
  DevBuf<int32_t> ciT, ciR, wi, base, words, cnt, cnt_up, lists, keep;
  DevBuf<uint32_t> wb, gs_sym;
  DevBuf<unsigned char> gs_num;
  DevBuf<uint8_t> frozen_row, frozen_inst;
  DevBuf<double> vT, vR, row_sq, row_diag, part;
  DevBuf<unsigned long long> ctr, row_ctr;
  DevBuf<GState> st;
  DevBuf<GStepRec> rec;
  DevBuf<int32_t> Nb, iters, conv;
  DevBuf<double> a, r0, nb, sq, tr, eps, t, m, bsum, bval;
  int64_t sym_stride = 0, sym_grid = 0, num_stride = 0, num_grid = 0;

  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    for (auto& e : texec)
      if (e) cudaGraphExecDestroy(e);
    for (auto& g : tgraph)
      if (g) cudaGraphDestroy(g);
    texec.clear();
    tgraph.clear();
    t_captured_for = 0;
  }
  // Frees T~ and the word pattern (and T^ unless keep_T); their sizes stay as hints.
  void release_matrices(bool keep_T) {
    drop_graph();
    if (capR) hintR = capR;
    if (capW) hintW = capW;
    ciR.free(); vR.free(); wi.free(); wb.free();
    capR = capW = 0;
    parked = false;
    if (!keep_T) {
      if (capT) hintT = capT;
      ciT.free(); vT.free();
      capT = 0;
    }
    ciS.free(); vS.free(); ciSN.free(); vSN.free(); ciT0.free(); vT0.free(); ciTN.free(); vTN.free();
    capS = capT0 = 0;
  }
  ~GraphSquaring() {
    if (gs) cudaStreamSynchronize(gs);
    drop_graph();
    for (cudaEvent_t e : ev_step) cudaEventDestroy(e);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (gs2) cudaStreamDestroy(gs2);
    if (gs) cudaStreamDestroy(gs);
  }
  int64_t arena_bytes() const {
    return (int64_t)(12 * (capT + capR) + 8 * capW + 8 * 4 * (n + 1) + 4 * 12 * n + 8 * 4 * n + gs_num.count +
                     4 * gs_sym.count);
  }
};

GraphSquaring* graph_squaring_new() { return new GraphSquaring(); }
void graph_squaring_free(GraphSquaring* G) { delete G; }
void graph_squaring_release(GraphSquaring* G, bool keep_T) {
  if (G) {
    if (G->gs) SX_CUDA(cudaStreamSynchronize(G->gs));
    G->release_matrices(keep_T);
  }
}
void graph_squaring_info(const GraphSquaring* G, int64_t* arena_bytes, int32_t* captures, int32_t* reruns,
                         int32_t* host_steps, int64_t* kernels_per_step, int64_t* kernels_per_pass) {
  if (arena_bytes) *arena_bytes = G ? G->arena_bytes() : 0;
  if (captures) *captures = G ? G->captures : 0;
  if (reruns) *reruns = G ? G->reruns : 0;
  if (host_steps) *host_steps = G ? G->host_steps : 0;
  if (kernels_per_step) *kernels_per_step = G ? G->k_outer : 0;
  if (kernels_per_pass) *kernels_per_pass = G ? G->k_body : 0;
}
void graph_squaring_note_host_steps(GraphSquaring* G, int steps) {
  if (G) G->host_steps += steps;
}
void graph_squaring_set_layout(GraphSquaring* G, int ks_bytes, int wide) {
  if (G->ks_bytes != ks_bytes || G->wide != wide) G->drop_graph();
  G->ks_bytes = ks_bytes;
  G->wide = wide;
}

namespace {

// The per-row and per-instance buffers (sizes fixed by the plan).
void setup_rows(GraphSquaring& G, const GraphSquaringIn& in, cudaStream_t s) {
  const bool same = G.count == in.count && G.n == in.n && G.n_max == in.n_max && G.sym == in.sym &&
                    G.square_scale == in.square_scale && G.e_r == in.e_r && G.max_iters == in.max_iters &&
                    G.inst == in.inst && G.seg == in.seg;
  if (same && G.gs) return;
  G.drop_graph();
  if (!G.gs) {
    SX_CUDA(cudaGetDevice(&G.device));
    SX_CUDA(cudaStreamCreateWithFlags(&G.gs, cudaStreamNonBlocking));
    SX_CUDA(cudaStreamCreateWithFlags(&G.gs2, cudaStreamNonBlocking));
    SX_CUDA(cudaEventCreateWithFlags(&G.ev_in, cudaEventDisableTiming));
    SX_CUDA(cudaEventCreateWithFlags(&G.ev_out, cudaEventDisableTiming));
  }
  G.count = in.count;
  G.n = in.n;
  G.n_max = in.n_max;
  G.sym = in.sym;
  G.square_scale = in.square_scale;
  G.e_r = in.e_r;
  G.max_iters = in.max_iters;
  G.inst = in.inst;
  G.seg = in.seg;
  const int64_t n = in.n, c = in.count;
  G.rpT.reset(n + 1, s); G.rpR.reset(n + 1, s); G.rpF.reset(n + 1, s); G.wrp.reset(n + 1, s);
  G.flops.reset(n, s); G.scan_ts.reset(scan_tiles(n), s);
  G.base.reset(n, s); G.words.reset(n, s); G.cnt.reset(n, s); G.cnt_up.reset(n, s);
  G.lists.reset((size_t)n * kProductClasses, s); G.keep.reset(n, s);
  G.frozen_row.reset(n, s); G.frozen_inst.reset(c, s);
  G.row_sq.reset(n, s); G.row_diag.reset(n, s); G.part.reset(n, s);
  G.ctr.reset(2 * (2 * kProductClasses + 4), s); G.row_ctr.reset(2 * kProductClasses, s);
  G.st.reset(1, s);
  G.rec.reset(kRecCap, s);
  G.Nb.reset(c, s); G.iters.reset(c, s); G.conv.reset(c, s);
  G.a.reset(c, s); G.r0.reset(c, s); G.nb.reset(c, s); G.sq.reset(c, s); G.tr.reset(c, s);
  G.eps.reset(c, s); G.t.reset(c, s); G.m.reset(c, s); G.bsum.reset(c, s); G.bval.reset(c, s);
  // zeroed once so that no kernel ever reads an unwritten value
  SX_CUDA(cudaMemsetAsync(G.part.p, 0, n * sizeof(double), s));
  SX_CUDA(cudaMemsetAsync(G.keep.p, 0, n * sizeof(int32_t), s));
  SX_CUDA(cudaMemsetAsync(G.cnt.p, 0, n * sizeof(int32_t), s));
  SX_CUDA(cudaMemsetAsync(G.bsum.p, 0, c * sizeof(double), s));
  SX_CUDA(cudaMemsetAsync(G.sq.p, 0, c * sizeof(double), s));
  SX_CUDA(cudaMemsetAsync(G.tr.p, 0, c * sizeof(double), s));
}

// The arena of the matrices: T^ (capT entries; the filtered result is compacted into it), T~
// (capR entries), the word pattern of T^ (capW words) and the global-class scratch.  When T^
// grows its first keep_T entries are kept (a resumed run continues from them).  The buffers
// are replaced in the order T~, words, T^; T^ is parked in T~'s buffers while it is replaced.
// The global-memory class's scratch of the products (for the current layout).
void setup_scratch(GraphSquaring& G, cudaStream_t s) {
  const int ks = G.ks_bytes >= 0 ? G.ks_bytes : default_ks_bytes();
  const bool wide = G.wide >= 0 ? G.wide != 0 : default_wide_blocks();
  int64_t ss, sg, ns, ng;
  dev_product_scratch(G.n_max, ks, wide, ss, sg, ns, ng);
  const bool same = ss == G.sym_stride && sg == G.sym_grid && ns == G.num_stride && ng == G.num_grid;
  if (same && G.gs_num.p && G.gs_sym.p) return;
  G.drop_graph();
  G.sym_stride = ss; G.sym_grid = sg; G.num_stride = ns; G.num_grid = ng;
  G.gs_sym.reset((size_t)(ss * sg), s);
  G.gs_num.reset((size_t)(ns * ng), s);
}

void setup_arena(GraphSquaring& G, int64_t capT, int64_t capR, int64_t capW, int64_t keep_T, cudaStream_t s) {
  setup_scratch(G, s);
  if (capT == G.capT && capR == G.capR && capW == G.capW && G.ciT.p) return;
  G.drop_graph();
  if (capR != G.capR || !G.ciR.p) {
    G.ciR.free(); G.vR.free();
    G.capR = 0;
    G.ciR.reset(capR, s); G.vR.reset(capR, s);
    G.capR = capR;
  }
  if (capW != G.capW || !G.wi.p) {
    G.wi.free(); G.wb.free();
    G.capW = 0;
    G.wi.reset(capW, s); G.wb.reset(capW, s);
    G.capW = capW;
  }
  if (capT != G.capT || !G.ciT.p) {
    if (keep_T > 0 && G.ciT.p && G.capR >= keep_T) {
      // T~'s buffers hold nothing a resumed run needs: T^ waits there while it is reallocated,
      // so the old and the new T^ are never held together
      SX_CUDA(cudaMemcpyAsync(G.ciR.p, G.ciT.p, keep_T * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      SX_CUDA(cudaMemcpyAsync(G.vR.p, G.vT.p, keep_T * sizeof(double), cudaMemcpyDeviceToDevice, s));
      G.ciT.free(); G.vT.free();
      G.capT = 0;
      G.parked = true;
      G.ciT.reset(capT, s); G.vT.reset(capT, s);
      SX_CUDA(cudaMemcpyAsync(G.ciT.p, G.ciR.p, keep_T * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      SX_CUDA(cudaMemcpyAsync(G.vT.p, G.vR.p, keep_T * sizeof(double), cudaMemcpyDeviceToDevice, s));
      G.parked = false;
    } else {
      DevBuf<int32_t> ci(capT, s);
      DevBuf<double> v(capT, s);
      if (keep_T > 0) {
        SX_CUDA(cudaMemcpyAsync(ci.p, G.ciT.p, keep_T * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        SX_CUDA(cudaMemcpyAsync(v.p, G.vT.p, keep_T * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
      G.ciT = std::move(ci);
      G.vT = std::move(v);
    }
    G.capT = capT;
  }
}

DevProduct product_bufs(GraphSquaring& G) {
  DevProduct P;
  P.n = G.n;
  P.wrp = G.wrp.p; P.wi = G.wi.p; P.wb = G.wb.p; P.wcap = G.capW;
  P.base = G.base.p; P.words = G.words.p; P.cnt = G.cnt.p; P.cnt_up = G.cnt_up.p;
  P.lists = G.lists.p; P.flops = G.flops.p;
  P.ctr = G.ctr.p; P.row_ctr = G.row_ctr.p; P.scan_ts = G.scan_ts.p;
  P.gs_sym = G.gs_sym.p; P.gs_sym_stride = G.sym_stride; P.gs_sym_grid = G.sym_grid;
  P.gs_num = G.gs_num.p; P.gs_num_stride = G.num_stride; P.gs_num_grid = G.num_grid;
  P.rp_out = G.rpR.p; P.ci_out = G.ciR.p; P.v_out = G.vR.p; P.cap_out = G.capR;
  P.row_sq = G.row_sq.p; P.row_diag = G.row_diag.p;
  P.status = &G.st.p->status;
  P.need = &G.st.p->need_raw;
  P.need_w = &G.st.p->need_w;
  P.ks_bytes = G.ks_bytes >= 0 ? G.ks_bytes : default_ks_bytes();
  P.wide = G.wide >= 0 ? G.wide != 0 : default_wide_blocks();
  return P;
}

// Captures one squaring step into G.graph (kernels and memsets only; nothing is allocated or
// read back while capturing).
void capture(GraphSquaring& G) {
  G.drop_graph();
  DevProduct P = product_bufs(G);
  dev_product_prepare(P);
  const int64_t n = G.n;
  const int c = G.count;
  CsrD T, R;
  T.n = R.n = n;
  T.rp = G.rpT.p; T.ci = G.ciT.p; T.v = G.vT.p;
  R.rp = G.rpR.p; R.ci = G.ciR.p; R.v = G.vR.p;
  GState* st = G.st.p;
  const int32_t* status = &st->status;
  cudaStream_t gs = G.gs, gs2 = G.gs2;
  int dev_sms = 0;
  SX_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, G.device));
  const int64_t L0 = launches();
  bool body_open = false;
  SX_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
  try {
    k_g_begin<<<1, 256, 0, gs>>>(st, c, G.Nb.p, G.frozen_inst.p);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
    row_flags(G.inst, G.frozen_inst.p, n, G.frozen_row.p, gs);
    dev_product(T, T, true, 1.0, 2.0, G.sym, G.frozen_row.p, P, gs);
    if (G.square_scale) {
      seg_sums_dev(G.row_sq.p, G.seg, c, G.sq.p, gs);
      seg_sums_dev(G.row_diag.p, G.seg, c, G.tr.p, gs);
    }
    k_g_alg41_init<<<1, 256, 0, gs>>>(st, c, G.frozen_inst.p, G.a.p, G.r0.p, G.nb.p, G.sq.p, G.tr.p,
                                     G.square_scale ? 1 : 0, G.eps.p, G.t.p, G.m.p, G.bval.p, G.iters.p, G.conv.p);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
    const int64_t L1 = launches();
    // Algorithm 4.1 as a WHILE node whose body is one pass over every row
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    SX_CUDA(cudaStreamGetCaptureInfo(gs, &cs, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h;
    SX_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cn;
    SX_CUDA(cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &np));
    SX_CUDA(cudaStreamUpdateCaptureDependencies(gs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
    SX_CUDA(cudaStreamBeginCaptureToGraph(gs2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    body_open = true;
    filter_pass_seg_dev(R, G.inst, G.t.p, G.keep.p, G.part.p, status, gs2);
    seg_sums_dev(G.part.p, G.seg, c, G.bsum.p, gs2);
    k_g_alg41_update<<<1, 256, 0, gs2>>>(st, c, G.e_r, G.max_iters, G.eps.p, G.t.p, G.m.p, G.bsum.p, G.bval.p,
                                        G.iters.p, G.conv.p, h);
    SX_CUDA(cudaGetLastError());
    count_launches(1);
    cudaGraph_t body = nullptr;
    body_open = false;
    SX_CUDA(cudaStreamEndCapture(gs2, &body));
    const int64_t L2 = launches();
    // the kept entries, compacted into T^'s arrays, and the step's record
    scan_counts_dev(G.keep.p, n, G.rpF.p, G.scan_ts.p, gs);
    k_g_cap_check_out<<<1, 1, 0, gs>>>(st, G.rpF.p + n, G.capT);
    SX_CUDA(cudaGetLastError());
    compact_seg_dev(R, G.inst, G.t.p, G.rpF.p, G.ciT.p, G.vT.p, status, gs);
    k_g_record<<<1, 256, 0, gs>>>(st, G.rec.p, c, G.ctr.p, dev_product_products_index(), dev_product_formed_index(),
                                  G.rpR.p + n, G.rpF.p + n, G.frozen_inst.p, G.eps.p, G.t.p, G.bval.p, G.iters.p);
    k_g_row_ptrs<<<(unsigned)(dev_sms * 2), 256, 0, gs>>>(st, n, G.rpF.p, G.rpT.p);
    SX_CUDA(cudaGetLastError());
    count_launches(3);
    const int64_t L3 = launches();
    SX_CUDA(cudaStreamEndCapture(gs, &G.graph));
    G.k_outer = (L1 - L0) + (L3 - L2);
    G.k_body = L2 - L1;
    count_launches(-(L3 - L0));  // captured, not launched
  } catch (...) {
    cudaGraph_t tmp = nullptr;
    if (body_open && cudaStreamEndCapture(gs2, &tmp) == cudaSuccess && tmp) cudaGraphDestroy(tmp);
    tmp = nullptr;
    if (cudaStreamEndCapture(gs, &tmp) == cudaSuccess && tmp) cudaGraphDestroy(tmp);
    cudaGetLastError();
    G.graph = nullptr;
    throw;
  }
  SX_CUDA(cudaGraphInstantiate(&G.exec, G.graph, 0));
  ++G.captures;
}

}  // namespace

void graph_squarings(GraphSquaring* Gp, const CsrD& T0, const GraphSquaringIn& in, GraphSquaringOut& out,
                     cudaStream_t s) {
  GraphSquaring& G = *Gp;
  const int count = in.count;
  int Nmax = 0;
  for (int b = 0; b < count; ++b) Nmax = std::max(Nmax, in.N[b]);
  if (Nmax > kRecCap) fail(SEXPM_EINVAL, "the captured squaring step keeps at most 128 step records");
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (G.device >= 0 && dev != G.device) fail(SEXPM_EINVAL, "current device differs from the captured graph's device");
  setup_rows(G, in, s);
  out.steps.clear();
  out.reruns = 0;
  out.steps_done = 0;
  out.T = T0;
  // capacities: those of the last run; else from the caller's budget (T^ 1/4, T~ 3/4 of the
  // entries, words 1/4 of T^'s), else small (a few times T^_0) and grown by the run; never above
  // the instances' dense size
  const int64_t dense = std::max<int64_t>(in.dense, 1);
  int64_t capT = G.capT ? G.capT : G.hintT, capR = G.capR ? G.capR : G.hintR, capW = G.capW ? G.capW : G.hintW;
  if (capT == 0 || capR == 0 || capW == 0) {
    if (in.arena_bytes > 0) {
      capT = std::max<int64_t>(in.arena_bytes / (12 * 4 + 2), 1);
      capR = 3 * capT;
    } else {
      capT = std::max<int64_t>(4 * T0.nnz, 1 << 20);
      capR = 4 * capT;
    }
    capW = std::max<int64_t>(capT / 4, 1);
  }
  capT = std::min(std::max(capT, T0.nnz), dense);
  capR = std::min(capR, dense);
  capW = std::min(capW, dense);
  std::vector<GStepRec> rec(Nmax);
  std::vector<double> ms_step(Nmax + 1, 0.0);
  GState hst;
  int g_from = 1;        // first step of this attempt
  int64_t keep_T = 0;    // entries of T^_{g_from - 1} to keep when the arena grows
  for (int attempt = 0;; ++attempt) {
    try {
      setup_arena(G, capT, capR, capW, keep_T, s);
    } catch (const Error& e) {
      if (e.code != SEXPM_ENOMEM) throw;
      // device memory ran out: the steps done so far stand, the caller runs the rest
      if (arena_log()) std::fprintf(stderr, "sexpm arena: out of device memory at step %d (%s)\n", g_from, e.msg.c_str());
      cudaGetLastError();
      out.steps_done = g_from - 1;
      if (g_from > 1) {
        out.T.n = G.n;
        out.T.nnz = keep_T;
        out.T.rp = G.rpT.p;
        out.T.ci = G.parked ? G.ciR.p : G.ciT.p;  // (T^ may be parked in T~'s buffers)
        out.T.v = G.parked ? G.vR.p : G.vT.p;
      }
      break;
    }
    if (!G.exec) capture(G);
    if ((int)G.ev_step.size() < Nmax + 1) {
      for (int k = (int)G.ev_step.size(); k <= Nmax; ++k) {
        cudaEvent_t e;
        SX_CUDA(cudaEventCreate(&e));
        G.ev_step.push_back(e);
      }
    }
    SX_CUDA(cudaEventRecord(G.ev_in, s));
    SX_CUDA(cudaStreamWaitEvent(G.gs, G.ev_in, 0));
    if (attempt == 0) {
      // inputs of the run
      SX_CUDA(cudaMemcpyAsync(G.rpT.p, T0.rp, (G.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, G.gs));
      if (T0.nnz) {
        SX_CUDA(cudaMemcpyAsync(G.ciT.p, T0.ci, T0.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, G.gs));
        SX_CUDA(cudaMemcpyAsync(G.vT.p, T0.v, T0.nnz * sizeof(double), cudaMemcpyDeviceToDevice, G.gs));
      }
      SX_CUDA(cudaMemcpyAsync(G.Nb.p, in.N.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, G.gs));
      SX_CUDA(cudaMemcpyAsync(G.a.p, in.a.data(), count * sizeof(double), cudaMemcpyHostToDevice, G.gs));
      SX_CUDA(cudaMemcpyAsync(G.r0.p, in.r0.data(), count * sizeof(double), cudaMemcpyHostToDevice, G.gs));
      SX_CUDA(cudaMemcpyAsync(G.nb.p, in.nb.data(), count * sizeof(double), cudaMemcpyHostToDevice, G.gs));
    }
    // the state of a run whose first g_from - 1 steps are done
    std::memset(&hst, 0, sizeof(hst));
    hst.g = g_from - 1;
    SX_CUDA(cudaMemcpyAsync(G.st.p, &hst, sizeof(GState), cudaMemcpyHostToDevice, G.gs));
    SX_CUDA(cudaEventRecord(G.ev_step[g_from - 1], G.gs));
    for (int g = g_from; g <= Nmax; ++g) {
      SX_CUDA(cudaGraphLaunch(G.exec, G.gs));
      SX_CUDA(cudaEventRecord(G.ev_step[g], G.gs));
    }
    SX_CUDA(cudaMemcpyAsync(&hst, G.st.p, sizeof(GState), cudaMemcpyDeviceToHost, G.gs));
    SX_CUDA(cudaMemcpyAsync(rec.data(), G.rec.p, Nmax * sizeof(GStepRec), cudaMemcpyDeviceToHost, G.gs));
    SX_CUDA(cudaStreamSynchronize(G.gs));
    const int done_to = hst.status ? hst.fail_g - 1 : Nmax;  // last step completed by this attempt
    for (int g = g_from; g <= done_to; ++g) {
      float ms = 0.f;
      SX_CUDA(cudaEventElapsedTime(&ms, G.ev_step[g - 1], G.ev_step[g]));
      ms_step[g] = ms;
    }
    if (hst.status == 0) {
      out.steps_done = Nmax;
      out.T.n = G.n;
      out.T.nnz = Nmax ? (int64_t)rec[Nmax - 1].nnz : T0.nnz;
      out.T.rp = G.rpT.p;
      out.T.ci = G.ciT.p;
      out.T.v = G.vT.p;
      break;
    }
    if (hst.status & kStNoConv)
      fail(SEXPM_ENOCONV, "Algorithm 4.1 did not converge within " + std::to_string(in.max_iters) + " passes");
    if (hst.status & kStMirror) fail(SEXPM_ECUDA, "symmetric product: an entry without its mirror partner");
    if (hst.status & kStBound) fail(SEXPM_ECUDA, "a product row exceeded the scratch bound of its size class");
    if (hst.fail_g < g_from || hst.fail_g > Nmax) fail(SEXPM_ECUDA, "captured squaring step: bad failure record");
    // grow to the size the failing step asked for (+1/16; the small word pattern +1/2), with
    // room for the steps after it
    const int64_t needR = (int64_t)hst.need_raw, needT = (int64_t)hst.need_out, needW = (int64_t)hst.need_w;
    const int64_t nR = (hst.status & kStProduct) ? std::min(dense, needR + needR / 16) : capR;
    const int64_t nW = (hst.status & kStWords) ? std::min(dense, needW + needW / 2) : capW;
    int64_t nT = (hst.status & kStFiltered) ? std::min(dense, needT + needT / 16) : capT;
    const int f = hst.fail_g;
    keep_T = f == 1 ? T0.nnz : (int64_t)rec[f - 2].nnz;
    if ((hst.status & kStProduct) && f >= 2 && rec[f - 2].nnz_raw > 0) {
      // a larger T~ keeps a share of its entries that grows from step to step (the instances
      // densify): T^ gets room for half-way between the last step's share and all of T~, so a
      // step whose product has just been formed is seldom stopped by its filtered size
      const double share = (double)rec[f - 2].nnz / (double)rec[f - 2].nnz_raw;
      const double room = std::min(1.0, 1.05 * (share + 0.5 * (1.0 - share)));
      nT = std::max(nT, std::min(dense, (int64_t)(room * (double)nR)));
    }
    if (((hst.status & kStProduct) && nR < needR) || ((hst.status & kStFiltered) && nT < needT) ||
        ((hst.status & kStWords) && nW < needW) || attempt >= 6 * Nmax + 8)
      fail(SEXPM_EOVERFLOW, "the batched squarings do not fit the device arena");
    if (arena_log()) {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      std::fprintf(stderr,
                   "sexpm arena: step %d status %d needs T~ %lld T^ %lld words %lld; capacities T~ %lld -> %lld, "
                   "T^ %lld -> %lld, words %lld -> %lld; device free %.1f GB\n",
                   f, hst.status, (long long)needR, (long long)needT, (long long)needW, (long long)capR, (long long)nR,
                   (long long)capT, (long long)std::max(nT, keep_T), (long long)capW, (long long)nW, fr / 1e9);
    }
    g_from = f;
    capR = nR;
    capW = nW;
    capT = std::max(nT, keep_T);
    ++G.reruns;
    ++out.reruns;
  }
  SX_CUDA(cudaEventRecord(G.ev_out, G.gs));
  SX_CUDA(cudaStreamWaitEvent(s, G.ev_out, 0));
  // per-step records of the steps done
  int64_t kernels = 0;
  int64_t nnz_prev = T0.nnz;
  for (int g = 1; g <= out.steps_done; ++g) {
    const GStepRec& r = rec[g - 1];
    sexpm_step_stats st;
    std::memset(&st, 0, sizeof(st));
    st.phase = 1;
    st.i = g;
    st.iters = r.iters_max;
    st.t = r.t_max;
    st.eps_g = r.eps_max;
    st.b = r.b_max;
    st.nnz_raw = (int64_t)r.nnz_raw;
    st.nnz = (int64_t)r.nnz;
    st.products = (int64_t)r.products;
    st.products_done = (int64_t)r.formed;
    st.flops = 2.0 * (double)r.formed + 2.0 * (double)nnz_prev;
    st.chunks = 1;
    st.ms = ms_step[g];
    out.steps.push_back(st);
    nnz_prev = (int64_t)r.nnz;
    kernels += G.k_outer + G.k_body * r.loops;
  }
  count_launches(kernels);
  out.launches = kernels;
  out.arena_bytes = G.arena_bytes();
}


// ---------------------------------------------------------------- the Taylor phase

namespace {

// Buffers of the Taylor phase: H_0 (capH), S^ and the new term (capS each), T^_0 and the sum
// (capT0 each); T~ and the word pattern are the squarings' (capR, capW).  S^ and T^_0 keep their
// first keepS / keepT0 entries when they grow.
void setup_taylor(GraphSquaring& G, int64_t capH, int64_t capS, int64_t capT0, int64_t capR, int64_t capW,
                  int64_t keepS, int64_t keepT0, cudaStream_t s) {
  const int64_t n = G.n;
  setup_scratch(G, s);
  if (G.rpS.count != (size_t)(n + 1)) {
    G.drop_graph();
    G.rpH.reset(n + 1, s); G.rpS.reset(n + 1, s); G.rpSN.reset(n + 1, s);
    G.rpT0.reset(n + 1, s); G.rpTN.reset(n + 1, s);
  }
  if (G.Mb.count != (size_t)G.count) {
    G.drop_graph();
    G.Mb.reset(G.count, s); G.eps0.reset(G.count, s); G.done.reset(G.count, s);
  }
  if (!G.recT.p) G.recT.reset(kRecCap, s);
  if (capR != G.capR || !G.ciR.p) {
    G.drop_graph();
    G.ciR.free(); G.vR.free();
    G.capR = 0;
    G.ciR.reset(capR, s); G.vR.reset(capR, s);
    G.capR = capR;
  }
  if (capW != G.capW || !G.wi.p) {
    G.drop_graph();
    G.wi.free(); G.wb.free();
    G.capW = 0;
    G.wi.reset(capW, s); G.wb.reset(capW, s);
    G.capW = capW;
  }
  if (capH != G.capH || !G.ciH.p) {
    G.drop_graph();
    G.ciH.reset(capH, s); G.vH.reset(capH, s);
    G.capH = capH;
  }
  auto grow = [&](DevBuf<int32_t>& ci, DevBuf<double>& v, int64_t cap, int64_t keep) {
    DevBuf<int32_t> c2(cap, s);
    DevBuf<double> v2(cap, s);
    if (keep > 0) {
      SX_CUDA(cudaMemcpyAsync(c2.p, ci.p, keep * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      SX_CUDA(cudaMemcpyAsync(v2.p, v.p, keep * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    ci = std::move(c2);
    v = std::move(v2);
  };
  if (capS != G.capS || !G.ciS.p) {
    G.drop_graph();
    grow(G.ciS, G.vS, capS, G.ciS.p ? keepS : 0);
    G.ciSN.reset(capS, s); G.vSN.reset(capS, s);
    G.capS = capS;
  }
  if (capT0 != G.capT0 || !G.ciT0.p) {
    G.drop_graph();
    grow(G.ciT0, G.vT0, capT0, G.ciT0.p ? keepT0 : 0);
    G.ciTN.reset(capT0, s); G.vTN.reset(capT0, s);
    G.capT0 = capT0;
  }
}

// Captures Taylor term i into G.tgraph[i] / G.texec[i].
void capture_taylor(GraphSquaring& G, int i) {
  DevProduct P = product_bufs(G);
  dev_product_prepare(P);
  const int64_t n = G.n;
  const int c = G.count;
  CsrD S, H, R, SN, T0;
  S.n = H.n = R.n = SN.n = T0.n = n;
  S.rp = G.rpS.p; S.ci = G.ciS.p; S.v = G.vS.p;
  H.rp = G.rpH.p; H.ci = G.ciH.p; H.v = G.vH.p;
  R.rp = G.rpR.p; R.ci = G.ciR.p; R.v = G.vR.p;
  SN.rp = G.rpSN.p; SN.ci = G.ciSN.p; SN.v = G.vSN.p;
  T0.rp = G.rpT0.p; T0.ci = G.ciT0.p; T0.v = G.vT0.p;
  GState* st = G.st.p;
  int32_t* status = &st->status;
  cudaStream_t gs = G.gs, gs2 = G.gs2;
  int dev_sms = 0;
  SX_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, G.device));
  const int64_t L0 = launches();
  bool body_open = false;
  cudaGraph_t graph = nullptr;
  SX_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
  try {
    k_t_begin<<<1, 256, 0, gs>>>(st, i, c, G.Mb.p, G.done.p, G.frozen_inst.p);
    check_cuda(cudaGetLastError(), "taylor: after k_t_begin");
    row_flags(G.inst, G.frozen_inst.p, n, G.frozen_row.p, gs);
    // S~_i = S^_{i-1} H_0 / i
    dev_product(S, H, false, (double)i, 0.0, false, G.frozen_row.p, P, gs);
    k_t_alg41_init<<<1, 256, 0, gs>>>(c, G.frozen_inst.p, G.eps0.p, G.eps.p, G.t.p, G.m.p, G.bval.p, G.iters.p,
                                     G.conv.p);
    check_cuda(cudaGetLastError(), "taylor: after k_t_alg41_init");
    count_launches(2);
    const int64_t L1 = launches();
    // Algorithm 4.1 per instance (WHILE node)
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    SX_CUDA(cudaStreamGetCaptureInfo(gs, &cs, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h;
    SX_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cn;
    SX_CUDA(cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &np));
    SX_CUDA(cudaStreamUpdateCaptureDependencies(gs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
    SX_CUDA(cudaStreamBeginCaptureToGraph(gs2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    body_open = true;
    filter_pass_seg_dev(R, G.inst, G.t.p, G.keep.p, G.part.p, status, gs2);
    seg_sums_dev(G.part.p, G.seg, c, G.bsum.p, gs2);
    k_g_alg41_update<<<1, 256, 0, gs2>>>(st, c, G.e_r, G.max_iters, G.eps.p, G.t.p, G.m.p, G.bsum.p, G.bval.p,
                                        G.iters.p, G.conv.p, h);
    check_cuda(cudaGetLastError(), "taylor: after k_g_alg41_update");
    count_launches(1);
    cudaGraph_t body = nullptr;
    body_open = false;
    SX_CUDA(cudaStreamEndCapture(gs2, &body));
    const int64_t L2 = launches();
    // S^_i (new term) and T^_0 + S^_i, each within its capacity; then, when the step succeeded,
    // the instances whose series ended, S^ <- S^_i and T^_0 <- the sum
    scan_counts_dev(G.keep.p, n, G.rpSN.p, G.scan_ts.p, gs);
    k_g_cap_check_out<<<1, 1, 0, gs>>>(st, G.rpSN.p + n, G.capS);
    compact_seg_dev(R, G.inst, G.t.p, G.rpSN.p, G.ciSN.p, G.vSN.p, status, gs);
    add_dev(T0, SN, 1.0, G.cnt.p, G.rpTN.p, G.scan_ts.p, G.ciTN.p, G.vTN.p, G.capT0, status, &st->need_sum, kStSum,
            gs);
    k_t_done<<<1, 256, 0, gs>>>(st, c, G.seg, G.rpSN.p, G.done.p);
    k_t_copy<<<(unsigned)(dev_sms * 4), 256, 0, gs>>>(st, n, G.rpSN.p, G.ciSN.p, G.vSN.p, G.rpS.p, G.ciS.p, G.vS.p);
    k_t_copy<<<(unsigned)(dev_sms * 4), 256, 0, gs>>>(st, n, G.rpTN.p, G.ciTN.p, G.vTN.p, G.rpT0.p, G.ciT0.p,
                                                     G.vT0.p);
    k_g_record<<<1, 256, 0, gs>>>(st, G.recT.p, c, G.ctr.p, dev_product_products_index(), dev_product_formed_index(),
                                  G.rpR.p + n, G.rpSN.p + n, G.frozen_inst.p, G.eps.p, G.t.p, G.bval.p, G.iters.p);
    check_cuda(cudaGetLastError(), "taylor: after k_g_record");
    count_launches(6);
    const int64_t L3 = launches();
    G.t_outer = (L1 - L0) + (L3 - L2);
    G.t_body = L2 - L1;
    SX_CUDA(cudaStreamEndCapture(gs, &graph));
  } catch (...) {
    cudaGraph_t tmp = nullptr;
    if (body_open && cudaStreamEndCapture(gs2, &tmp) == cudaSuccess && tmp) cudaGraphDestroy(tmp);
    tmp = nullptr;
    if (cudaStreamEndCapture(gs, &tmp) == cudaSuccess && tmp) cudaGraphDestroy(tmp);
    cudaGetLastError();
    throw;
  }
  count_launches(-(launches() - L0));  // captured, not launched
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    SX_CUDA(e);
  }
  G.tgraph[i] = graph;
  G.texec[i] = ex;
  ++G.t_captures;
}

}  // namespace

void graph_taylor(GraphSquaring* Gp, const CsrD& H0, const GraphSquaringIn& in, GraphSquaringOut& out,
                  cudaStream_t s) {
  GraphSquaring& G = *Gp;
  const int count = in.count;
  int Mmax = 0;
  for (int b = 0; b < count; ++b) Mmax = std::max(Mmax, in.M[b]);
  if (Mmax > kRecCap) fail(SEXPM_EINVAL, "the captured Taylor terms keep at most 128 records");
  int dev = 0;
  SX_CUDA(cudaGetDevice(&dev));
  if (G.device >= 0 && dev != G.device) fail(SEXPM_EINVAL, "current device differs from the captured graph's device");
  setup_rows(G, in, s);
  out.steps.clear();
  out.reruns = 0;
  out.steps_done = 0;
  const int64_t n = G.n;
  const int64_t dense = std::max<int64_t>(in.dense, 1);
  // capacities: those held, else from the caller's budget, else a few times H_0 (grown by the
  // run); S^ and T^_0 start as H_0, so they hold at least its entries
  const int64_t budget = in.arena_bytes > 0 ? std::max<int64_t>(in.arena_bytes / 64, 1) : 0;
  int64_t capS = G.capS ? G.capS : (budget ? budget : std::min(dense, std::max<int64_t>(8 * H0.nnz, 1 << 20)));
  capS = std::max(capS, H0.nnz);
  int64_t capT0 = std::max(G.capT0 ? G.capT0 : capS, H0.nnz);
  int64_t capR = G.capR ? G.capR : (G.hintR ? G.hintR : (budget ? budget : std::min(dense, 4 * capS)));
  int64_t capW = G.capW ? G.capW : (G.hintW ? G.hintW : std::max<int64_t>(capS / 4, 1));
  capW = std::max(capW, H0.nnz);  // the word pattern of H_0 (at most one word per entry)
  capR = std::max<int64_t>(std::min(capR, dense), 1);
  std::vector<GStepRec> rec(Mmax + 1);
  std::vector<double> ms_step(Mmax + 1, 0.0);
  int g_from = 2;
  int64_t keepS = 0, keepT0 = 0;
  GState hst;
  for (int attempt = 0;; ++attempt) {
    setup_taylor(G, H0.nnz, capS, capT0, capR, capW, keepS, keepT0, s);
    if (G.t_captured_for != Mmax || (int)G.texec.size() < Mmax + 1) {
      for (auto& e : G.texec)
        if (e) cudaGraphExecDestroy(e);
      for (auto& g : G.tgraph)
        if (g) cudaGraphDestroy(g);
      G.texec.assign(Mmax + 1, nullptr);
      G.tgraph.assign(Mmax + 1, nullptr);
      for (int i = 2; i <= Mmax; ++i) capture_taylor(G, i);
      G.t_captured_for = Mmax;
    }
    if ((int)G.ev_step.size() < Mmax + 1) {
      for (int k = (int)G.ev_step.size(); k <= Mmax; ++k) {
        cudaEvent_t e;
        SX_CUDA(cudaEventCreate(&e));
        G.ev_step.push_back(e);
      }
    }
    SX_CUDA(cudaEventRecord(G.ev_in, s));
    SX_CUDA(cudaStreamWaitEvent(G.gs, G.ev_in, 0));
    if (attempt == 0) {
      // inputs: H_0, S^_1 = H_0, T^_0 = H_0; an instance of degree M_b <= 1 has no further term
      std::vector<uint8_t> done0(count);
      for (int b = 0; b < count; ++b) done0[b] = in.M[b] <= 1 ? 1 : 0;
      for (int64_t* rp : {G.rpH.p, G.rpS.p, G.rpT0.p})
        SX_CUDA(cudaMemcpyAsync(rp, H0.rp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, G.gs));
      if (H0.nnz) {
        for (int32_t* ci : {G.ciH.p, G.ciS.p, G.ciT0.p})
          SX_CUDA(cudaMemcpyAsync(ci, H0.ci, H0.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, G.gs));
        for (double* v : {G.vH.p, G.vS.p, G.vT0.p})
          SX_CUDA(cudaMemcpyAsync(v, H0.v, H0.nnz * sizeof(double), cudaMemcpyDeviceToDevice, G.gs));
      }
      SX_CUDA(cudaMemcpyAsync(G.Mb.p, in.M.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, G.gs));
      SX_CUDA(cudaMemcpyAsync(G.eps0.p, in.eps_g0.data(), count * sizeof(double), cudaMemcpyHostToDevice, G.gs));
      SX_CUDA(cudaMemcpyAsync(G.done.p, done0.data(), count, cudaMemcpyHostToDevice, G.gs));
    }
    std::memset(&hst, 0, sizeof(hst));
    SX_CUDA(cudaMemcpyAsync(G.st.p, &hst, sizeof(GState), cudaMemcpyHostToDevice, G.gs));
    SX_CUDA(cudaEventRecord(G.ev_step[g_from - 1], G.gs));
    for (int i = g_from; i <= Mmax; ++i) {
      SX_CUDA(cudaGraphLaunch(G.texec[i], G.gs));
      SX_CUDA(cudaEventRecord(G.ev_step[i], G.gs));
    }
    int64_t nS = 0, nT0 = 0;
    SX_CUDA(cudaMemcpyAsync(&hst, G.st.p, sizeof(GState), cudaMemcpyDeviceToHost, G.gs));
    SX_CUDA(cudaMemcpyAsync(rec.data(), G.recT.p, (Mmax + 1) * sizeof(GStepRec), cudaMemcpyDeviceToHost, G.gs));
    SX_CUDA(cudaMemcpyAsync(&nS, G.rpS.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, G.gs));
    SX_CUDA(cudaMemcpyAsync(&nT0, G.rpT0.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, G.gs));
    SX_CUDA(cudaStreamSynchronize(G.gs));
    const int done_to = hst.status ? hst.fail_g - 1 : Mmax;
    for (int i = g_from; i <= done_to; ++i) {
      float ms = 0.f;
      SX_CUDA(cudaEventElapsedTime(&ms, G.ev_step[i - 1], G.ev_step[i]));
      ms_step[i] = ms;
    }
    if (hst.status == 0) {
      out.T.n = n;
      out.T.nnz = nT0;
      out.T.rp = G.rpT0.p;
      out.T.ci = G.ciT0.p;
      out.T.v = G.vT0.p;
      break;
    }
    if (hst.status & kStNoConv)
      fail(SEXPM_ENOCONV, "Algorithm 4.1 did not converge within " + std::to_string(in.max_iters) + " passes");
    if (hst.status & (kStMirror | kStBound)) fail(SEXPM_ECUDA, "captured Taylor term: internal bound exceeded");
    if (hst.fail_g < g_from || hst.fail_g > Mmax) fail(SEXPM_ECUDA, "captured Taylor term: bad failure record");
    const int64_t needR = (int64_t)hst.need_raw, needS = (int64_t)hst.need_out, needW = (int64_t)hst.need_w,
                  needT = (int64_t)hst.need_sum;
    const int64_t nR = (hst.status & kStProduct) ? std::min(dense, needR + needR / 4) : capR;
    const int64_t nS2 = (hst.status & kStFiltered) ? std::min(dense, needS + needS / 4) : capS;
    const int64_t nW = (hst.status & kStWords) ? std::min(dense, needW + needW / 2) : capW;
    const int64_t nT = (hst.status & kStSum) ? std::min(dense, needT + needT / 4) : capT0;
    if (((hst.status & kStProduct) && nR < needR) || ((hst.status & kStFiltered) && nS2 < needS) ||
        ((hst.status & kStWords) && nW < needW) || ((hst.status & kStSum) && nT < needT) || attempt >= 6 * Mmax + 8)
      fail(SEXPM_EOVERFLOW, "the batched Taylor terms do not fit the device arena");
    g_from = hst.fail_g;
    keepS = nS;
    keepT0 = nT0;
    capR = nR;
    capS = std::max(nS2, nS);
    capW = nW;
    capT0 = std::max(nT, nT0);
    ++G.t_reruns;
    ++out.reruns;
  }
  SX_CUDA(cudaEventRecord(G.ev_out, G.gs));
  SX_CUDA(cudaStreamWaitEvent(s, G.ev_out, 0));
  // the terms' records, up to the first term that was empty for every instance (the series ended)
  int64_t kernels = 0;
  for (int i = 2; i <= Mmax; ++i) {
    const GStepRec& r = rec[i - 1];
    sexpm_step_stats st;
    std::memset(&st, 0, sizeof(st));
    st.phase = 0;
    st.i = i;
    st.iters = r.iters_max;
    st.t = r.t_max;
    st.eps_g = r.eps_max;
    st.b = r.b_max;
    st.nnz_raw = (int64_t)r.nnz_raw;
    st.nnz = (int64_t)r.nnz;
    st.products = (int64_t)r.products;
    st.products_done = (int64_t)r.formed;
    st.flops = 2.0 * (double)r.formed + (double)r.nnz_raw;
    st.ms = ms_step[i];
    out.steps.push_back(st);
    kernels += G.t_outer + G.t_body * r.loops;
    if (r.nnz == 0) break;
  }
  count_launches(kernels);
  out.launches = kernels;
  out.steps_done = Mmax;
}

}  // namespace sexpm
