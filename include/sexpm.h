/*
 * sexpm.h - C ABI of the GB300 library for the filtered incremental
 * scaling-and-squaring method for a large sparse matrix exponential
 * (Wu, Zhang, Zhu, Hu, arXiv 2110.04493).
 *
 * Problem statement (Algorithm 4.2): given a sparse real H (n x n) and an
 * error tolerance eps_tol, return an approximation of e^{tau H} as a sparse
 * matrix together with the choices the method made: the scaling N and the
 * Taylor degree M (Eq. 4.20), the filter parameter a, the error bound r_0
 * (Eq. 4.5) and the filter thresholds of every Taylor term and squaring step
 * (Algorithm 4.1).
 *
 * Conventions shared by every call:
 *   - Matrices are square CSR: int64 row pointers (n+1 entries, row_ptr[0]=0,
 *     non-decreasing), int32 column indices sorted strictly increasing within
 *     each row, float64 values.  All arithmetic is IEEE float64 on the GPU.
 *   - Input views are borrowed: the library copies what it needs before the
 *     call returns and never frees caller memory.
 *   - Result handles (sexpm_result_t) own device memory allocated by the
 *     library from its own stream-ordered pool; release them with
 *     sexpm_result_free().
 *   - Every call returns an int status (SEXPM_OK = 0 or a negative code);
 *     no C++ exception crosses this boundary.  sexpm_last_error() returns a
 *     thread-local message describing the last failure on the calling thread.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Calls synchronise that stream before they
 *     return, because the method reads scalar reductions back to the host
 *     between kernels (Algorithm 4.1 is a host-driven iteration).
 *   - Results are reproducible run to run: every sum has an order fixed by
 *     the input and the launch shapes.
 *
 * Environment (tuning only; results change at most by rounding):
 *   SEXPM_KSPLIT_BYTES  per-SM shared-memory budget (bytes) under which a sparse
 *                       product row gives its warps private accumulators and
 *                       splits the k's of A_i among them (default 225280; 0 =
 *                       every warp owns a column range).  Read at every product.
 * Environment (testing the error paths):
 *   SEXPM_FAIL_ALLOC_AT=k  the k-th device allocation of each sexpm_compute fails
 *                       on the host as if the device were out of memory
 *                       (SEXPM_ENOMEM; everything allocated so far is released
 *                       and the plan stays usable).  Read at every sexpm_compute.
 */
#ifndef SEXPM_H_
#define SEXPM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define SEXPM_OK 0
#define SEXPM_EINVAL (-1)    /* bad CSR, n mismatch, NaN/Inf, eps <= 0, non-finite tau */
#define SEXPM_ENOMEM (-2)    /* device or host allocation failed */
#define SEXPM_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define SEXPM_ENOCONV (-4)   /* Algorithm 4.1 hit its iteration cap */
#define SEXPM_ENOPARAM (-5)  /* no feasible (M, N) in [N0, N0 + n_extra] */
#define SEXPM_ETIMEOUT (-6)  /* a bounded device wait gave up (reserved: no call of this version
                                waits on the device with a bound) */
#define SEXPM_EOVERFLOW (-7) /* a size exceeded an index type or a fixed capacity */

/* ------------------------------------------------------------------ types */

/* Borrowed square CSR matrix.  on_device = 1: the three arrays are device
 * pointers of the current device; 0: host pointers. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  int32_t on_device;
} sexpm_csr_view;

/* Options.  Fill with sexpm_options_default() and override fields. */
typedef struct {
  double e_r;               /* Algorithm 4.1 tolerance e_r (> 0); default 0.1 */
  int32_t square_scale;     /* 1: ||B_i|| <= a r_i ||I + T~_i||_F (Sec. 4.2, default);
                               0: ||B_i|| <= a r_i (the value printed in Algorithm 4.2) */
  int32_t normal_override;  /* -1: test normality; 0: treat H as non-normal; 1: as normal */
  int32_t max_filter_iters; /* Algorithm 4.1 iteration cap; default 100 */
  int32_t n_extra;          /* N_max = N_0 + n_extra in Eq. (4.20); default 50 */
  int32_t max_taylor;       /* cap on M (SEXPM_ENOPARAM above it); default 1000 */
  int32_t symmetric;        /* 1 (default): when H == H^T exactly, T^_0 is symmetrised
                               ((T^_0 + T^_0^T)/2; its asymmetry is at the level of the Taylor
                               filter) and every squaring T~_i = 2T + T T, symmetric by
                               construction, forms only the entries at columns >= row and
                               mirrors the rest (halves the FP64 work); 0: form every entry */
  int32_t row_order;        /* 1 (default): when H is a stencil on a grid numbered x + m y (+ m^2 z),
                               the sparse products visit the rows in strips of 32 consecutive x for
                               cache locality (the results do not depend on the order); 0: natural
                               row order */
  int64_t chunk_bytes;      /* squaring steps whose unfiltered product T~_i would not fit in free
                               device memory are formed in row chunks and filtered exactly as the
                               whole (Algorithm 4.1 streamed: every threshold it visits is at least
                               eps_g / sqrt(nnz(T~_i)), so a chunk keeps only its entries above that
                               bound and the sum of squares of the rest).  0 (default): chunk only
                               when needed, chunks sized from free memory; > 0: chunks of at most
                               this many bytes of T~_i whenever T~_i is larger. */
  int32_t scaling;          /* 0 (default): (M, N) by Eq. (4.20) on ||tau H||_F; 1: the refined norm of
                               Sec. 4.2, h_{M,N} = max_{M+1<=k<=2M+1} ||(tau H 2^-N)^k||_F^(1/k) from
                               exact sparse powers of tau H (up to k = refine_kmax), in the choice
                               of (M, N) (sexpm_choose_MN_refined), in r_0 = rho(M, h_{M,N}) and in
                               eps_g^(0) = a r_0 / (M e^{2 h_{M,N}}) */
  int32_t refine_kmax;      /* highest power of tau H the refined norm uses (odd, >= 3; default 41) */
  int32_t batched_graph;    /* batched plans: 1 (default): every Taylor term and every squaring step
                               runs as one captured CUDA graph -- sizes decided on the device,
                               Algorithm 4.1 iterated
                               by a conditional WHILE node, a fixed-capacity device arena held by the
                               plan, grown when a product does not fit (the run resumes at that step);
                               if device memory runs out the remaining steps run as host-driven
                               launches; an arena above a quarter of the device memory is freed at
                               the end of each compute (the next one allocates its sizes at once);
                               0: host-driven launches.  Both give bit-identical results. */
  int64_t batch_arena_bytes; /* first arena size for batched_graph = 1 (0, default: a few times H_0
                               and T^_0, grown by the run; never more than the instances' dense size) */
} sexpm_options;

typedef struct sexpm_plan sexpm_plan_t;
typedef struct sexpm_result sexpm_result_t;

/* Per Taylor term (i = 2..M') or squaring step (i = 1..N) record. */
typedef struct {
  int32_t phase;      /* 0 = Taylor term S^_i, 1 = squaring step T^_i */
  int32_t i;
  int32_t iters;      /* Algorithm 4.1 passes */
  int32_t chunks;     /* row chunks the product was formed in (1: whole) */
  double eps_g;       /* bound on the F-norm of the dropped part */
  double t;           /* final eps_f: stored entries with |v| <= t were dropped */
  double b;           /* F-norm of the dropped part */
  double norm_F;      /* ||I + T~_i||_F (squaring steps; 0 for Taylor terms) */
  int64_t nnz_raw;    /* stored entries before filtering */
  int64_t nnz;        /* stored entries after filtering */
  int64_t products;   /* scalar multiply-adds of the sparse product (all entries) */
  int64_t products_done; /* multiply-adds actually formed (fewer in the symmetric mode) */
  double ms;          /* device time of the step (CUDA events) */
  double ms_symbolic; /* sparse product: row analysis, binning and symbolic pass */
  double ms_numeric;  /* sparse product: numeric pass (fused /i or + 2T) */
  double ms_filter;   /* Algorithm 4.1 passes, row-pointer scan and compaction */
  double flops;       /* FP64 operations of the numeric pass: 2 products_done + the fused term */
  double bytes_filter;/* algorithmic bytes moved by the filter passes, scan and compaction */
  int64_t nnz_stream; /* chunked steps: entries kept by the streaming bound (Algorithm 4.1's input) */
  int64_t rows_class[6]; /* rows of the numeric pass per size class (shared memory 8, 24, 56, 112,
                            220 KB; the last class accumulates in global memory) */
} sexpm_step_stats;

typedef struct {
  int64_t n;
  double norm_H;      /* ||tau H||_F */
  int32_t M, N;       /* Eq. (4.20) */
  int32_t normal;     /* 1 if H was treated as normal */
  int32_t n_steps;    /* entries filled in steps[] (<= max) */
  int32_t symmetric;  /* 1 if the symmetric (upper-triangle) products were used */
  int32_t pad_;
  double a;           /* filter parameter: 1/(N+1) (normal) or 1/||H||_F */
  double r0;          /* Eq. (4.5) at x = ||H 2^-N||_F */
  double eps_g0;      /* a r_0 / (M e^{2 ||H_0||_F}), the Taylor-phase bound */
  int64_t nnz_out;    /* stored entries of e^{tau H} */
  double ms_total;    /* device time of sexpm_compute */
  double ms_taylor;
  double ms_squaring;
  double ms_final;
  int64_t peak_bytes; /* peak device bytes held by the library during compute */
  int64_t launches;   /* kernels enqueued by the library during compute */
} sexpm_stats_t;

/* ------------------------------------------------------------------ calls */

/* Fill *opt with the defaults listed above.  Never fails for non-NULL opt. */
int sexpm_options_default(sexpm_options* opt);

/* Algorithm 4.2 step 1 input: validate H (square, sorted unique columns,
 * finite values), copy it to the device, compute ||H||_F and the normality
 * flag (H == H^T or H == -H^T exactly, else ||H H^T - H^T H||_F <= 64 u ||H||_F^2)
 * on the GPU.  eps is eps_tol of Algorithm 4.2 (> 0, finite).  n must equal
 * H->n.  opt may be NULL (defaults).  On success *out owns device memory. */
int sexpm_plan(const sexpm_csr_view* H, int64_t n, double eps, const sexpm_options* opt,
               void* stream, sexpm_plan_t** out);

/* Algorithm 4.2 for tau*H: (M, N) by Eq. (4.20); a by step 2; the filtered
 * Taylor phase of Eqs. (4.10)-(4.11); N filtered squarings
 * T~_i = 2 T^_{i-1} + T^_{i-1}^2 (Eq. 4.15) each filtered by Algorithm 4.1;
 * e^{tau H} = I + T^_N.  tau must be finite.  *out receives a new result. */
int sexpm_compute(sexpm_plan_t* plan, double tau, sexpm_result_t** out);

/* Dimension and stored-entry count of a result. */
int sexpm_result_info(const sexpm_result_t* res, int64_t* n, int64_t* nnz);

/* ---------------------------------------------------------- complex H
 * The method is stated for H in C^{n x n}.  A complex CSR view has val pointing to 2 nnz doubles,
 * the (re, im) pairs of the entries (the layout of C99 double complex / numpy complex128).
 * Internally Z = X + iY is carried by the rows [X_i | -Y_i] of its real embedding
 * [[X, -Y], [Y, X]] (products of the embedding are the embedding of the products), every
 * product forms those n rows only, and Algorithm 4.1 keeps or drops a complex entry as a whole
 * by its modulus |z| (its sums add |z|^2).  (M, N) come from ||tau H||_F with the complex norm;
 * a = 1/(N+1) when H is normal (H H^* = H^* H: Hermitian and skew-Hermitian H exactly, else
 * ||H H^* - H^* H||_F <= 64 u ||H||_F^2).  tau stays real (put a factor -i into H for e^{-i tau H}).
 * The symmetric mode, the row chunking, the refined scaling (scaling = 1), the batched form,
 * the adjoint and e^H R are real-only.  n <= 2^30.  sexpm_compute computes e^{tau H} of such a
 * plan; its statistics count the real entries and products of the embedding's top rows. */
int sexpm_plan_z(const sexpm_csr_view* H, int64_t n, double eps, const sexpm_options* opt, void* stream,
                 sexpm_plan_t** out);
/* 1 when res holds a complex e^{tau H} (from a plan of sexpm_plan_z). */
int sexpm_result_is_complex(const sexpm_result_t* res, int32_t* is_complex);
/* Copy a complex result: n+1 row pointers, nnz columns, 2 nnz doubles (re, im pairs).
 * SEXPM_EINVAL for a real result (and sexpm_result_copy returns SEXPM_EINVAL for a complex one). */
int sexpm_result_copy_z(const sexpm_result_t* res, int64_t* row_ptr, int32_t* col, double* val, int32_t on_device);

/* Copy a result into caller buffers of n+1 / nnz / nnz elements; on_device
 * selects device (1) or host (0) destination pointers. */
int sexpm_result_copy(const sexpm_result_t* res, int64_t* row_ptr, int32_t* col, double* val,
                      int32_t on_device);

/* Scalars and per-step records of the compute that produced res.  steps may
 * be NULL; otherwise up to max_steps records are written. */
int sexpm_stats(const sexpm_result_t* res, sexpm_stats_t* stats, sexpm_step_stats* steps,
                int32_t max_steps);

void sexpm_result_free(sexpm_result_t* res);
void sexpm_plan_destroy(sexpm_plan_t* plan);

/* Thread-local description of the last failure ("" if none). */
const char* sexpm_last_error(void);

/* Number of kernels the library has enqueued since it was loaded (all threads). */
int64_t sexpm_kernel_launches(void);

/* Return the device memory cached by the library's pool on the current device to
 * the driver (the pool keeps freed blocks for reuse otherwise). */
int sexpm_release_memory(void);

/* Bytes the library currently holds from its device pool (all devices) and the largest
 * value since the last sexpm_compute started (or since load).  Either pointer may be NULL. */
int sexpm_pool_stats(int64_t* live_bytes, int64_t* peak_bytes);

/* Host-only helpers (no GPU needed): the scalar choices of Algorithm 4.2. */

/* Eq. (4.5): (1/M!) sum_k x^{M+1+k} / (k! (M+1+k)). */
double sexpm_rho(int32_t M, double x);

/* Eq. (4.20): minimise M 2^N over N in [N0, N0 + n_extra], N0 = max(ceil(log2 norm_H), 0),
 * M the least positive integer with 2^N rho(M, norm_H 2^-N) <= eps; ties to the smaller
 * M + N, then the smaller N.  norm_H = 0 gives M = N = 0. */
int sexpm_choose_MN(double norm_H, double eps, int32_t n_extra, int32_t max_M, int32_t* M, int32_t* N);

/* ||H^k||_F for k = 1..kmax into out[0..kmax-1], from exact sparse powers H^k = H^{k-1} H formed
 * on the GPU (Sec. 4.2: the norms behind the refined bound h_{M,N} of Eq. 4.9).  The powers
 * widen by the stencil at every step: memory grows like nnz(H^kmax). */
int sexpm_power_norms(const sexpm_csr_view* H, int32_t kmax, void* stream, double* out);

/* alpha^_i of Eq. (4.8) (pnorms NULL) or Eq. (4.9) (pnorms[k-1] = ||H^k||, k <= kmax): the least
 * M1 2^N1 with 2^N1 rho(M1, x) <= r_i = 2^i rho(M, ||H 2^-N||) (Eq. 4.6), x = ||H 2^{i-N-N1}|| or the
 * refined h_{M1, N+N1-i}; alpha^_i lambda(H) bounds the eps-bandwidth of the squaring iterate
 * T_i (Eq. 4.7, Theorem 3.8).  Host only. */
int sexpm_alpha_hat(double norm_H, int32_t M, int32_t N, int32_t i, const double* pnorms, int32_t kmax,
                    int32_t* alpha);

/* Eq. (4.20)'s rule on the refined norm: minimise M 2^N over N in [0, N0 + n_extra] (N0 =
 * max(ceil(log2 norm_H), 0)), M the least positive integer (2M + 1 <= kmax) with
 * 2^N rho(M, h_{M,N}) <= eps and h_{M,N} <= 1; ties to the smaller M + N, then the smaller N.
 * Host only; SEXPM_ENOPARAM when no pair qualifies. */
int sexpm_choose_MN_refined(double norm_H, const double* pnorms, int32_t kmax, double eps, int32_t n_extra,
                            int32_t* M, int32_t* N);

/* ---------------------------------------------------------- batched form */

/* Many independent matrices H_b (b = 0..count-1, sizes may differ) planned together: the
 * instances are stored as one block-diagonal matrix, so every step of Algorithm 4.2 runs as one
 * set of kernel launches for the whole batch (the sparse product's row kernels are persistent
 * over per-size-class row lists that hold the rows of every instance); with
 * sexpm_options.batched_graph = 1 each Taylor term and each squaring step is one replay of a
 * captured CUDA graph.  Validation, symmetry and normality are per
 * instance.  eps is shared.  Not in the paper (a batched form of Algorithm 4.2). */
int sexpm_plan_batched(const sexpm_csr_view* Hs, int32_t count, double eps, const sexpm_options* opt,
                       void* stream, sexpm_plan_t** out);

/* Algorithm 4.2 for every tau_b H_b of a batched plan: each instance gets its own (M_b, N_b)
 * by Eq. (4.20), its own a_b, r_0 and thresholds, and its own Algorithm 4.1 iterations; an
 * instance that has done its N_b squarings is carried unchanged through the remaining
 * steps.  outs[b] receives e^{tau_b H_b} (an n_b x n_b result).  For a plain plan this
 * is sexpm_compute with taus[0]. */
int sexpm_compute_batched(sexpm_plan_t* plan, const double* taus, sexpm_result_t** outs);

/* The captured squaring step of a batched plan (batched_graph = 1): device arena bytes held by
 * the plan, graph captures so far, steps resumed after an arena overflow, squaring steps left to
 * the host-driven launches because device memory ran out, kernels each step launches outside the
 * Algorithm 4.1 loop and per pass of that loop.  Zeros before the first compute.  Any output may
 * be NULL.  Not in the paper. */
int sexpm_batched_graph_info(const sexpm_plan_t* plan, int64_t* arena_bytes, int32_t* captures, int32_t* reruns,
                             int32_t* host_steps, int64_t* kernels_per_step, int64_t* kernels_per_pass);

/* Autotuner of the numeric pass's accumulation layout for a batched plan: runs
 * sexpm_compute_batched(plan, taus) once per candidate (ks_bytes[c]: the shared-memory budget of
 * the k split, 0 = pure column split; wide[c]: 1024-thread blocks for the global-memory class)
 * and keeps the fastest squaring phase for the plan's later computes.  ncand = 0 tries a built-in
 * list (ks_bytes, wide) = (225280, 1), (112640, 1), (0, 1), (225280, 0).  ms_out (ncand entries
 * or 4 for the built-in list; may be NULL) receives each candidate's squaring time, *best (may
 * be NULL) the index chosen.  Results of every candidate agree to rounding (the layouts sum the
 * same products in different orders).  Needs batched_graph = 1.  Not in the paper. */
int sexpm_tune_batched(sexpm_plan_t* plan, const double* taus, int32_t ncand, const int32_t* ks_bytes,
                       const int32_t* wide, double* ms_out, int32_t* best);

/* ---------------------------------------------------------- adjoint form */

/* Gradient of a scalar loss through e^{tau H}: given W = dL/dE for E = e^{tau H} (a sparse
 * matrix; only its entries on the pattern of E matter), returns dL/dH on the stored pattern
 * of H.  The derivative is that of the map the method computes with the scaling N, the Taylor
 * degree and every filter decision (the kept patterns of Algorithm 4.1) held fixed, which is
 * piecewise constant in H: with Y = dL/dT^_k on the pattern of T^_k,
 *   dL/dT^_{k-1} = mask_{k-1}(2 Y + Y T^_{k-1}^T + T^_{k-1}^T Y)     (reverse of Eq. 4.15),
 * then the reverse of the Taylor recursion of Eq. (4.11), and dL/dH = tau 2^-N dL/dH_0.
 * The forward pass is rerun with every product formed; T^_k is kept every ckpt_stride
 * squarings (0: ceil(sqrt(N))) and the iterates in between are recomputed in the reverse pass.
 * *dH receives a result with the pattern of H (its stats are those of the forward run);
 * if expm_out is not NULL it receives e^{tau H} of that forward run.  Not in the paper
 * (the differentiation form of the method). */
int sexpm_adjoint(sexpm_plan_t* plan, double tau, const sexpm_csr_view* W, int32_t ckpt_stride,
                  sexpm_result_t** dH, sexpm_result_t** expm_out);

/* The forward half of sexpm_adjoint, for callers that differentiate later (an autograd
 * function's forward and backward): computes e^{tau H} with every product formed, keeping
 * H_0, the filtered Taylor terms and T^_k at the checkpoints k = 0, ckpt_stride, 2 ckpt_stride,
 * .., N (0: ceil(sqrt(N))) in *tape, which owns that device memory and borrows the plan (the
 * plan must outlive the tape).  *expm_out (may be NULL) receives e^{tau H}.  Not in the paper. */
typedef struct sexpm_tape sexpm_tape_t;
int sexpm_forward_keep(sexpm_plan_t* plan, double tau, int32_t ckpt_stride, sexpm_result_t** expm_out,
                       sexpm_tape_t** tape);

/* The reverse half: dL/dH on the stored pattern of H for W = dL/dE, from a kept forward (the
 * iterates between checkpoints are recomputed).  A tape may serve several calls.  Same result
 * as sexpm_adjoint with the same tau and ckpt_stride. */
int sexpm_adjoint_tape(sexpm_tape_t* tape, const sexpm_csr_view* W, sexpm_result_t** dH);

void sexpm_tape_free(sexpm_tape_t* tape);

/* ------------------------------------------------------------ step calls */
/* The individual steps of the hot path on caller-provided device CSR views,
 * for testing and measurement.  Outputs are new result handles. */

/* One sparse product with the fused scaling and sum of Algorithm 4.2:
 *   C = (A B) / div + beta * D     (D may be NULL; its pattern joins C's).
 * div = i gives the Taylor term S~_i = S^_{i-1} H_0 / i (Eq. 4.10);
 * div = 1, beta = 2, D = A = B = T gives T~ = 2T + T T (Eq. 4.15).
 * Every structurally present entry is stored (exact zeros included).
 * *products receives the number of scalar multiply-adds. */
int sexpm_spgemm(const sexpm_csr_view* A, const sexpm_csr_view* B, const sexpm_csr_view* D,
                 double div, double beta, void* stream, sexpm_result_t** out, int64_t* products);

/* Algorithm 4.1 on the stored values of A with bound eps_g and tolerance e_r:
 * keeps the entries with |v| > t, t the final eps_f.  Writes t, the number of
 * passes and the dropped F-norm b. */
int sexpm_filter(const sexpm_csr_view* A, double eps_g, double e_r, int32_t max_iters, void* stream,
                 sexpm_result_t** out, double* t, int32_t* iters, double* b);

/* A^T of a CSR (columns sorted within every row of the result; rows of any length), as used by
 * the adjoint's reverse pass (Y T^T and T^T Y) and the symmetric part of T^_0. */
int sexpm_transpose(const sexpm_csr_view* A, void* stream, sexpm_result_t** out);

/* One Algorithm 4.1 reduction pass on the stored values of A (device or host view): the sum of
 * v^2 over the entries with |v| <= t (*sum_dropped) and the number of entries with |v| > t
 * (*kept).  With the threshold sequence t_0 = eps_g, t_{j+1} = eps_g t_j / b_j driven by the caller,
 * this is the pass a multi-process run all-reduces across its row blocks.  t >= 0. */
int sexpm_filter_pass(const sexpm_csr_view* A, double t, void* stream, double* sum_dropped, int64_t* kept);

/* A~ = A - b_n of Algorithm 4.1 at a given final threshold: the entries of A with |v| > t. */
int sexpm_filter_apply(const sexpm_csr_view* A, double t, void* stream, sexpm_result_t** out);

/* sum over the rows r0 <= i < r1 of A of sum_j (delta_ij + a_ij)^2, the part of ||I + A||_F^2
 * (the relative threshold of the squaring steps, Sec. 4.2) that those rows hold. */
int sexpm_norm2_I_plus_rows(const sexpm_csr_view* A, int64_t r0, int64_t r1, void* stream, double* out);

/* ------------------------------------------------- applying e^{tau H} to vectors */

/* Y = E X for a result E (n x n) and a block X of r vectors: X and Y are device arrays of n x r
 * doubles, row-major (vector c of row k at X[k r + c]); X and Y must not overlap.  This is how
 * the computed exponential is used (Sec. 5.3 applies it to a block of random vectors). */
int sexpm_result_spmm(const sexpm_result_t* E, const double* X, int64_t r, double* Y, void* stream);

/* Time stepping with a computed propagator (Eq. 2.2): U_k = E U_{k-1}, k = 1..steps, from U_0;
 * U0 and U are device arrays of n x r doubles (row-major, may be the same array).  One n x r
 * work array comes from the library's pool. */
int sexpm_propagate(const sexpm_result_t* E, const double* U0, int64_t r, int32_t steps, double* U, void* stream);

/* Y = A X for a borrowed CSR view (copied to the device first) and device X, Y as above. */
int sexpm_spmm(const sexpm_csr_view* A, const double* X, int64_t r, double* Y, void* stream);

/* ------------------------------------------------------- no-allocation call */

/* Largest number of rows sexpm_filter_noalloc accepts (its fixed scratch size). */
#define SEXPM_NOALLOC_MAX_ROWS 1048576

/* Algorithm 4.1 and the compaction of the kept entries, like sexpm_filter, but without
 * allocating any memory: no cudaMalloc/cudaFree, no pool, no pinned host buffer.  The paper
 * has no counterpart; this call exists for callers that cannot allocate device memory when
 * they filter, e.g. because another allocator already owns all of the GPU's memory or
 * because they run under a fixed memory budget.
 *
 * A must be a device CSR (on_device = 1) with at most SEXPM_NOALLOC_MAX_ROWS rows (larger
 * inputs return SEXPM_EOVERFLOW with a message).  The caller provides the outputs on the
 * device: out_row_ptr (n+1 entries) and out_col / out_val with room for out_capacity
 * entries (nnz(A) always suffices; if the kept part is larger, SEXPM_EOVERFLOW and none of
 * the three output arrays is written).  On success *nnz_out is the number of kept entries
 * and t, iters and b are as for sexpm_filter.
 *
 * Scratch (per-row kept counts, per-block partial sums, scan tile sums; about 4.2 MB) lives
 * in one static device array that every GPU loading the library holds until the process
 * exits.  The first call on a device looks up its address (cudaGetSymbolAddress, once per
 * device); make that first call before any stream capture.  The address stays cached for
 * the process: after a cudaDeviceReset of a device, do not call this entry point on it
 * again.  `stream` must belong to the current device (SEXPM_EINVAL otherwise).  All calls
 * share the array: calls that overlap on the GPU race on it, so the caller must serialise
 * them.  The call synchronises `stream` before it returns. */
int sexpm_filter_noalloc(const sexpm_csr_view* A, double eps_g, double e_r, int32_t max_iters, void* stream,
                         int64_t* out_row_ptr, int32_t* out_col, double* out_val, int64_t out_capacity,
                         int64_t* nnz_out, double* t, int32_t* iters, double* b);

#ifdef __cplusplus
}
#endif
#endif /* SEXPM_H_ */
