/*
 * mc.h -- C ABI of the GB300 fast-SVT matrix-completion library (libmc.so).
 *
 * The library computes, on one GPU, the hot path of accelerated singular value
 * thresholding (Feng, Yu & Li, "Faster Matrix Completion Using Randomized
 * SVD", arXiv 1810.06860):
 *   - randomized truncated SVDs of a sparse matrix Y held as CSR plus a CSC
 *     copy: rSVD-PI (Alg. 4) and rSVD-BKI (Alg. 5), built from eigSVD (Alg. 3);
 *   - the SVT iteration of Alg. 6 (Sec. IV.C): rank growth, shrink, the update
 *     Y^i = Y^{i-1} + delta P_Phi(M - X^i) evaluated only on the observed set
 *     Phi, subspace recycling (Sec. IV.B) and the adaptive power parameter p.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major.  An m x k factor U is U[i*k + j].
 *   - Singular values are returned in descending order.
 *   - Pointer arguments marked "host or device" may point to either; the
 *     library asks the CUDA runtime which one it is.  Output buffers are
 *     allocated by the caller.
 *   - Every call returns an mc_status; nothing throws across the ABI.  On
 *     failure mc_last_error() returns a message for the calling thread.
 *   - A handle is used by one host thread at a time.  All device work of a
 *     handle is issued on its stream; calls return after the results they
 *     report are on the host (they synchronise that stream).
 *   - Sizes: m, n >= 1, nnz < 2^31 (indices are stored as int32 on the GPU).
 */
#ifndef MC_H_
#define MC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MC_OK = 0,
  MC_EINVAL = 1,          /* bad argument or input (nothing launched) */
  MC_ENOMEM = 2,          /* device allocation failed */
  MC_ECUDA = 3,           /* a CUDA call failed */
  MC_ENOTCONVERGED = 4,   /* SVT hit i_max; results are still filled */
  MC_EBUSY = 5,           /* server queue full / job not admitted */
  MC_PENDING = 6,         /* job not finished yet (mc_poll) */
  MC_ETIMEOUT = 7,        /* a bounded wait expired */
  MC_ECANCELLED = 8,      /* job was cancelled */
  MC_EINTERNAL = 9        /* internal consistency check failed */
} mc_status;

typedef struct mc_handle_s *mc_handle;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer aligned to 256 bytes or NULL; free releases
 * it.  Both are called on the host thread that calls the library. */
typedef struct {
  void *ctx;
  void *(*alloc)(void *ctx, size_t bytes, void *stream);
  void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
} mc_allocator;

/* Parameters of Alg. 6 (Sec. IV.C) and of the internal settings of Alg. 2 it
 * inherits (Sec. II.C).  mc_params_default fills the paper's values. */
typedef struct {
  double tau;     /* threshold; <= 0 selects 5*sqrt(m*n) (Sec. II.C's 5n for square) */
  double delta;   /* step size delta of eq. (6) */
  double eps;     /* tolerance on ||P_Phi(X - M)||_F / ||P_Phi(M)||_F (Alg. 6 step 16) */
  int l;          /* rank increment (5) */
  int s;          /* oversampling (10) */
  int p0;         /* initial power parameter (3, Alg. 6 step 1) */
  int p_min;      /* lower bound of p (3) */
  int p_max;      /* upper bound of p (20) */
  int i_max;      /* iteration cap (1000) */
  int i_reuse;    /* first iteration allowed to recycle (50) */
  int q_reuse;    /* recycled SVD calls per subspace (10) */
  int recycle;    /* 0 none, 1 reuse Q, 2 reuse U (Sec. IV.B), 3 warm-start Omega with V */
  int k_max;      /* cap on the SVD rank (0 = min(m,n) - s) */
  int precision;  /* 0 plain float32, 1 bf16 panels in the Krylov products */
  int inner;      /* SVD of each fresh call: 0 rSVD-BKI (Alg. 5, Alg. 6 step 6), 1 rSVD-PI (Alg. 4) */
  uint64_t seed;  /* key of the Philox stream that draws Omega */
} mc_params;

/* Per-iteration record of mc_svt_step. */
typedef struct {
  int i;            /* iteration index (1-based) */
  int k;            /* rank requested from the last SVD of the repeat loop */
  int r;            /* r_i = #{sigma_j > tau} */
  int p;            /* power parameter used */
  int nsvd;         /* SVD calls in this iteration's repeat loop */
  int recycled;     /* 1 if any of them recycled a subspace */
  int converged;    /* 1 if err < eps (Y was not advanced) */
  int reserved;
  double err;       /* ||P_Phi(X^i - M)||_F / ||P_Phi(M)||_F */
  double sigma_last;/* last singular value computed (the repeat test) */
  double sigma_max; /* largest singular value of Y^{i-1} */
  double c;         /* c = ceil(tau / (delta ||P_Phi M||_2)) of Y^0 = c delta P_Phi(M) */
  double norm2;     /* the ||P_Phi(M)||_2 estimate behind c */
} mc_iter_info;

void mc_params_default(mc_params *p);
const char *mc_last_error(void);
/* Number of kernels this library has launched in the process so far. */
int64_t mc_launch_count(void);
const char *mc_status_str(mc_status s);

/* mc_create: ingest the observed entries P_Phi(M) (problem (5), Sec. II.C).
 * row_ptr int64[m+1], col int32[nnz], val float32[nnz] in CSR order; columns
 * strictly increasing within a row; values finite.  Host or device pointers.
 * The library copies them into handle-owned device memory and builds the CSC
 * copy and its permutation.  stream: a cudaStream_t or NULL (the handle
 * creates its own).  alloc: NULL for cudaMallocAsync on the stream.
 * Errors: MC_EINVAL for bad shapes, unsorted or duplicate columns, indices out
 * of range or non-finite values; MC_ENOMEM; MC_ECUDA. */
mc_status mc_create(mc_handle *out, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col, const float *val, void *stream, const mc_allocator *alloc);
/* mc_create_coo: as mc_create, from coordinates in any order: rows int64[nnz],
 * cols int32[nnz], vals float32[nnz] (host or device).  The entries are
 * sorted on the device by (row, column) with a stable radix sort into the CSR
 * that mc_create takes.  MC_EINVAL also for a repeated (row, column) pair. */
mc_status mc_create_coo(mc_handle *out, int64_t m, int64_t n, int64_t nnz, const int64_t *rows,
                        const int32_t *cols, const float *vals, void *stream, const mc_allocator *alloc);
void mc_destroy(mc_handle h);

/* Set the values of the sparse iterate Y (CSR order, nnz floats, host or
 * device).  mc_create initialises Y = P_Phi(M). */
mc_status mc_set_values(mc_handle h, const float *val);

/* mc_rsvd_bki: rank-k truncated SVD of the current Y by rSVD-BKI (Alg. 5):
 * Gaussian Omega (n x (k+s)) drawn from Philox(seed, call_id); p block-Krylov
 * steps; B^T = Y^T Q; eigSVD(B^T); the k largest triplets.
 * (k, p) are clamped so that (p+1)(k+s) <= min(m,n) (k+s itself must fit).
 * U: m x k_out, S: k_out, V: n x k_out, row-major, host or device; each may be
 * NULL.  k_out (host) receives the rank returned (k after clamping, fewer if Y
 * has lower rank).  Buffers must hold k columns. */
mc_status mc_rsvd_bki(mc_handle h, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U,
                      float *S, float *V, int *k_out);

/* Precision of the randomized SVDs of this handle: 0 plain float32 (default);
 * 1 mixed: the panels that feed the Krylov / power products (Omega, A^T Q and
 * Q) are read as bf16 with float32 sums, the basis is orthonormalised in
 * float32, and the final projection B^T = Y^T Q uses the float32 basis (one
 * float32 pass over the Krylov block).  mc_svt_step sets it from
 * params->precision.  MC_EINVAL for other values. */
mc_status mc_set_precision(mc_handle h, int precision);

/* mc_rsvd_pi: as mc_rsvd_bki but by rSVD-PI (Alg. 4): p power steps with a
 * block normalisation between them, eigSVD of the last block, B^T = Y^T Q. */
mc_status mc_rsvd_pi(mc_handle h, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U,
                     float *S, float *V, int *k_out);

/* mc_rsvd_basic: as mc_rsvd_bki but by the basic randomized SVD with power
 * iteration (Alg. 1, Sec. II.B): Q = orth(Y Omega), then p times
 * G = orth(Y^T Q), Q = orth(Y G) -- an orthonormalisation after every
 * product -- then B^T = Y^T Q and the SVD of B (computed by eigSVD, which
 * Lemma 1 shows equal to svd()).  The cost reference of Table I. */
mc_status mc_rsvd_basic(mc_handle h, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U,
                        float *S, float *V, int *k_out);

/* mc_svt_step: one outer iteration of Alg. 6 (steps 3-17).  The first call on
 * a handle (or the first after mc_svt_reset) also performs step 1: estimates
 * ||P_Phi(M)||_2, sets c and Y^0 = c delta P_Phi(M).  params is read at that
 * first call only.  out (host) receives the iteration record.  Returns MC_OK
 * (also when the tolerance was met: out->converged = 1).  The copy of the
 * updated Y into CSC order (the values the Y^T X products read) is left
 * running on a second stream of the handle when the call returns; the
 * library's own calls wait for it where they need it. */
mc_status mc_svt_step(mc_handle h, const mc_params *params, mc_iter_info *out);
mc_status mc_svt_reset(mc_handle h);

/* mc_join: orders the handle's stream after the work the handle left on its
 * second stream (the copy of Y into CSC order after mc_svt_step), so that an
 * event recorded on the handle's stream afterwards, or a synchronisation of
 * it, covers all of the handle's work.  Enqueues a wait only; does not block. */
mc_status mc_join(mc_handle h);

/* mc_svt_solve: run mc_svt_step until err < eps or i_max.  Returns MC_OK or
 * MC_ENOTCONVERGED (results still available).  out (host, may be NULL)
 * receives the last iteration's record. */
mc_status mc_svt_solve(mc_handle h, const mc_params *params, mc_iter_info *out);

/* Factors of the current SVT estimate X = Us V^T with Us = U diag(sigma - tau)
 * (Alg. 6 step 15).  r_out (host) receives r.  Us: m x r, V: n x r, sigma: r
 * (the singular values before shrinking); host or device; any may be NULL;
 * buffers must hold max_r columns (MC_EINVAL if r > max_r). */
mc_status mc_svt_factors(mc_handle h, int max_r, float *Us, float *V, float *sigma, int *r_out);

/* Evaluate the current X at count positions (rows[i], cols[i]) (host or
 * device int64 arrays) into out (host or device float32). */
mc_status mc_svt_sample(mc_handle h, int64_t count, const int64_t *rows, const int64_t *cols,
                        float *out);

/* Values of the current iterate Y in CSR order (nnz floats, host or device). */
mc_status mc_get_values(mc_handle h, float *val);

/* ---- device timing -------------------------------------------------------
 * Per kernel class: CUDA-event time on the handle's stream, launches, and the
 * algorithmic bytes / flops of those launches (compulsory traffic: for a
 * sparse x panel product 8 nnz + 4 (rows+1) + 4 (rows_in + rows_out) K bytes
 * and 2 nnz K flops; for the fused update 16 bytes per observed entry plus
 * the two factor panels).  Off by default; enabling resets the counters. */
enum {
  MC_T_SPMM = 0,      /* Y X over CSR */
  MC_T_SPMM_T = 1,    /* Y^T X over the CSC copy */
  MC_T_GRAM = 2,      /* X^T X and X^T Y panel products */
  MC_T_GEMM = 3,      /* panel x small products */
  MC_T_SMALL = 4,     /* Cholesky / inverse of small Grams */
  MC_T_EIG = 5,       /* small symmetric eigensolver */
  MC_T_SDDMM = 6,     /* fused evaluation on Phi + update of Y */
  MC_T_OTHER = 7,     /* Omega, mirror of Y into CSC order, reductions */
  MC_T_COUNT = 8
};
typedef struct {
  double ms;
  double bytes;
  double flops;
  int64_t launches;
} mc_timing;
/* on: 0 off, 1 every class, 2 the two sparse-product classes only (two
 * events per product instead of two per launch of every class: the lighter
 * form for a timed region).  Synchronises the handle's stream and resets
 * the counters. */
mc_status mc_timing_enable(mc_handle h, int on);
/* out: MC_T_COUNT entries (host).  Synchronises the handle's stream. */
mc_status mc_timing_read(mc_handle h, mc_timing *out);

/* ---- serving: many completion jobs on one GPU ---------------------------
 *
 * A server runs whole SVT solves (Alg. 6 until err < eps or i_max) for jobs
 * submitted at any time.  Jobs are admitted in arrival order as soon as a
 * slot is free and the job's device-memory footprint fits the budget
 * (continuous batching: jobs that arrive while others run join them).  Each
 * admitted job keeps its sparse iterate Y, recycled subspace and factors
 * resident on the device and issues its kernels on its own CUDA stream, so
 * the work of different jobs overlaps on the GPU.  Results do not depend on
 * what else runs: every kernel is deterministic.  The paper solves one
 * problem at a time; this form has no counterpart there. */
typedef struct mc_server_s *mc_server;

typedef struct {
  int64_t m, n, nnz;          /* job shape; nnz observed entries */
  const int64_t *row_ptr;     /* host, m+1 entries, CSR of P_Phi(M) */
  const int32_t *col;         /* host, nnz column indices, sorted within rows */
  const float *val;           /* host, nnz observed values M_ij */
  mc_params params;           /* tau, delta, eps, i_max, ... of Alg. 6 */
} mc_job_desc;

typedef struct {
  mc_status status;           /* MC_OK (converged), MC_ENOTCONVERGED, MC_ECANCELLED or the failure */
  int iters, r, converged;
  double err;                 /* last ||P_Phi(X - M)||_F / ||P_Phi(M)||_F */
  int64_t m, n;
  const float *Us;            /* host m x r, U diag(sigma - tau) (row-major); owned by the server */
  const float *V;             /* host n x r */
  const float *sigma;         /* host r singular values before shrinking, descending */
  double queue_s;             /* seconds from mc_submit to admission */
  double latency_s;           /* seconds from mc_submit to completion */
  size_t footprint_bytes;     /* admission estimate */
  size_t device_bytes_peak;   /* device memory the job held at its peak */
  const char *message;        /* failure message ("" on success); owned by the server */
} mc_result;

typedef struct {
  size_t budget_bytes, in_use_bytes, peak_in_use_bytes;
  int active, peak_active, queued, slots;
  int64_t admitted, completed;
} mc_server_info;

/* mc_server_create: budget_bytes of device memory for admitted jobs' estimated
 * footprints (0: half of the free memory of the device at creation);
 * max_active concurrent jobs (1..256), each driven by one host worker thread;
 * device: CUDA device ordinal.  simulate != 0 runs no GPU work: a job takes
 * params.i_max microseconds and returns no factors (tests of the scheduling
 * logic on hosts without a GPU). */
mc_status mc_server_create(mc_server *out, size_t budget_bytes, int max_active, int device, int simulate);

/* mc_server_destroy: cancels queued and running jobs, waits for the workers
 * (a running job stops after its current iteration) and frees everything. */
void mc_server_destroy(mc_server s);

/* mc_submit: copies the job's host arrays and queues it; returns at once with
 * its id.  MC_EINVAL for bad shapes or pointers; the CSR itself is checked
 * when the job starts (its result then carries MC_EINVAL).  A job whose
 * footprint exceeds the whole budget runs alone when nothing else does. */
mc_status mc_submit(mc_server s, const mc_job_desc *job, uint64_t *job_id);

/* mc_poll: non-blocking.  MC_PENDING while the job is queued or running;
 * otherwise fills out and returns MC_OK (out->status holds the job's own
 * outcome) or MC_ECANCELLED.  MC_EINVAL for an unknown id.  The pointers in
 * out stay valid until mc_result_release or mc_server_destroy. */
mc_status mc_poll(mc_server s, uint64_t job_id, mc_result *out);

/* mc_wait: blocks until the job has finished or timeout_s has passed
 * (MC_ETIMEOUT). */
mc_status mc_wait(mc_server s, uint64_t job_id, double timeout_s);

/* mc_cancel: a queued job is dropped; a running one stops after its current
 * iteration.  Its result has status MC_ECANCELLED. */
mc_status mc_cancel(mc_server s, uint64_t job_id);

/* mc_result_release: frees a finished job's result (MC_EBUSY if not finished). */
mc_status mc_result_release(mc_server s, uint64_t job_id);

/* mc_server_stats: occupancy counters.  mc_server_admit_order writes up to
 * cap job ids in the order they were admitted and returns how many there are. */
mc_status mc_server_stats(mc_server s, mc_server_info *out);
int64_t mc_server_admit_order(mc_server s, uint64_t *ids, int64_t cap);

/* ---- building blocks, exposed for testing and reuse -------------------- */

/* Omega (n x k) of Alg. 1/4/5 step 1 drawn from Philox4x32-10 with counter
 * (row, col0 + col, call_lo, call_hi) and key (seed_lo, seed_hi), Box-Muller
 * z = sqrt(-2 ln u1) cos(2 pi u2), u1 = (x0+1) 2^-32, u2 = x1 2^-32.
 * out: n x k row-major (host or device).  words (optional, host or device,
 * uint32 n x k x 2) receives (x0, x1). */
mc_status mc_omega(int64_t n, int k, uint64_t seed, uint64_t call_id, int col0, float *out,
                   uint32_t *words);

/* Sparse products with the current Y (the A X and A^T X products of Alg. 5):
 * trans = 0: out (m x k) = Y X with X n x k;  trans = 1: out (n x k) = Y^T X
 * with X m x k.  Row-major, host or device. */
mc_status mc_spmm(mc_handle h, int trans, int k, const float *X, float *out);

/* Symmetric eigen-decomposition of a dense K x K matrix A (row-major, host or
 * device; only its lower triangle is read): the kw largest eigenvalues in
 * descending order into lam (kw floats) and their eigenvectors into W
 * (K x kw row-major).  The eig() step of eigSVD (Alg. 3).  K <= 1024. */
mc_status mc_eig_sym(int K, int kw, const float *A, float *lam, float *W);

/* One Krylov block of the orthonormal basis of Alg. 5 (its orth(), built a
 * block at a time; the span is that of Theorem 2): out (R x K) = an
 * orthonormal basis of (I - Qp Qp^T) X.  X is projected against the cols
 * earlier orthonormal columns Qp twice (block classical Gram-Schmidt with
 * reorthogonalisation), then passed through CholeskyQR steps (the first
 * with a shift of 1e-6 trace/K, then plain ones: two, or one when the block
 * is already orthonormal to within 1e-2 after the first, for blocks of at
 * most 32 columns that take the one-launch kernel).  A column whose
 * squared norm after the projection is at most 1e-10 of its squared norm
 * before (a dependent direction), or whose Cholesky pivot falls to the
 * float32 noise floor, is returned as a zero column.  These are the kernels
 * the rSVD-BKI steps use.
 *   - Device pointers, row-major: X (R x K, leading dimension ldx),
 *     Qp (R x cols, ldq), out (R x K, ldo); 16-byte aligned.  X is
 *     overwritten; out must not overlap X or Qp.
 *   - K and cols multiples of 4 (zero columns pad a block), K <= 1024;
 *     ldx, ldq and ldo multiples of 4.  Anything else: MC_EINVAL.
 *   - Enqueued on stream (a cudaStream_t, NULL for the legacy default
 *     stream); scratch comes from cudaMallocAsync on that stream; returns
 *     after the stream has reached the end of the work. */
mc_status mc_orth_block(int64_t R, int K, float *X, int ldx, const float *Qp, int ldq, int cols, float *out, int ldo,
                        void *stream);

/* Gram matrix G = X^T X (K x K) of a tall X (R x K row-major), the B = A^T A
 * step of eigSVD (Alg. 3).  Host or device. */
mc_status mc_gram(int64_t R, int K, const float *X, float *G);

/* As mc_gram on the tensor cores (tcgen05, TF32 split into hi and lo parts
 * for float32 accuracy); K <= 256.  Returns MC_ETIMEOUT if a bounded wait on
 * a TMA or MMA barrier expired. */
mc_status mc_gram_tc(int64_t R, int K, const float *X, float *G);

/* mc_panel_gram: C = X1^T X2 (K1 x K2, row-major) of two tall panels X1 (R x
 * K1) and X2 (R x K2), row-major: the Grams of the block orthonormalisation
 * and the Ritz Gram B B^T (Alg. 3 step 1, Alg. 5 steps 3-9) and the
 * projections Q_prev^T X.  tensor_cores = 1 runs the tcgen05 kernel (TF32
 * operands split into hi and lo parts, float32 accumulation; K1, K2 <= 256,
 * else MC_EINVAL with nothing run); 0 runs the SIMT kernels.  Host or device
 * pointers; synchronous; MC_ETIMEOUT if a bounded wait of the tensor-core
 * kernel expired. */
mc_status mc_panel_gram(int64_t R, int K1, int K2, const float *X1, const float *X2, float *C, int tensor_cores);

/* mc_gather_rate: the rate (GB/s, gathered bytes) at which this GPU loads the
 * panel rows the sparse products of Alg. 5 gather -- rows idx[e] of an
 * n x k (trans = 0: the CSR column indices) or m x k (trans = 1: the CSC row
 * indices) panel, k rounded up to 4, in the SpMM's 16-byte lane slices and
 * entry order -- with no arithmetic or stores: the ceiling of the sparse
 * products' gathers on this matrix.  k <= 128; reps timed launches after one
 * warm-up (CUDA events on the handle's stream).  The paper has no counterpart
 * (a measurement aid). */
mc_status mc_gather_rate(mc_handle h, int trans, int k, int reps, double *gbs);

/* mc_panel_gemm: Z = X W of a tall X (R x K, row-major) and a small W (K x N,
 * row-major) into Z (R x N, row-major): the panel products of the block
 * orthonormalisation (X R^{-1} of a CholeskyQR pass, X - Q_prev C of a
 * projection) and of the Ritz factors (U = Q W of Alg. 5 step 11, V = B^T W
 * S^{-1} of Alg. 3 step 4).  tensor_cores = 1 runs the tcgen05 kernel (TF32
 * operands split into hi and lo parts, float32 accumulation: about float32
 * accuracy); it takes N <= 256 with K and N rounded up to 32 and 16 of product
 * at most 16384, else MC_EINVAL (nothing run).  tensor_cores = 0 runs the SIMT
 * kernels.  Host or device pointers; synchronous; MC_ETIMEOUT if a bounded
 * wait of the tensor-core kernel expired. */
mc_status mc_panel_gemm(int64_t R, int K, int N, const float *X, const float *W, float *Z, int tensor_cores);

/* mc_gram_noalloc: G = X^T X (K x K, leading dimension ldg) of a tall device
 * matrix X (R rows, K columns, leading dimension ld, ld a multiple of 4, base
 * address 16-byte aligned), like mc_gram but without allocating any device
 * memory.  Columns K..ld-1 of X are never combined into G.  The paper has no
 * counterpart; it exists for callers that cannot allocate while they call:
 * code between cudaStreamBeginCapture and cudaStreamEndCapture, host
 * callbacks and allocator hooks, and hosts whose device memory is entirely
 * owned by their own pool.
 *   - X and G must be device pointers; the call only enqueues work on stream
 *     (a cudaStream_t, NULL for the legacy default stream) and returns; G is
 *     ready when the stream reaches that point.
 *   - Scratch is one fixed 4 MiB device array inside the library, held by
 *     every GPU that loads it until the process exits.  K > 1024 is rejected
 *     with MC_EINVAL (the array must hold one 1024 x 1024 partial tile).
 *   - The first call on a device looks up that array's device address with
 *     cudaGetSymbolAddress (with the device current) and caches it; make that
 *     first call before any stream capture.  The cached address belongs to
 *     the device's primary context: after cudaDeviceReset the library must
 *     not be called again in that process.
 *   - MC_EINVAL (nothing enqueued) for R or K < 1, null, host or unaligned
 *     pointers, ld < K or not a multiple of 4, ldg < K, K > 1024.
 *   - All calls share the array and each overwrites it: calls that can
 *     overlap on the GPU (different streams, no ordering between them) race
 *     and give wrong results.  Order them on one stream or with events. */
mc_status mc_gram_noalloc(int64_t R, int K, const float *X, int ld, float *G, int ldg, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MC_H_ */
