/*
 * rpod.h -- C ABI of librpod: randomized POD (rPOD) of tall-skinny snapshot
 * matrices on one GB300 (sm_103a).
 *
 * The method is Alg. 1 of Sec. 4.2 ("randomized POD with subspace
 * iterations") of Besabe, Girfoglio, Quaini, Rozza, "Randomized POD-LSTM
 * ROMs for the quasi-geostrophic equations" (arXiv 2504.15350):
 *   Lambda (m x l) ~ N(0, 1)        Gaussian sketching matrix
 *   P = S Lambda                    sampled matrix
 *   P <- (S S^T)^q P                subspace iterations, orthonormalised after
 *                                   every product with S or S^T
 *   P = Q R                         QR (CholeskyQR on the GPU)
 *   T = Q^T S                       l x m
 *   T = Uhat Sigma V^T              small SVD
 *   U = Q Uhat                      basis (first k columns)
 * with n = N_C grid cells, m = N^s snapshots, k = N^r, l = k + p, plus the
 * modal coefficients C = U_k^T S of Sec. 4.3.
 *
 * Conventions for every entry point
 *   - Matrices are column-major with an explicit leading dimension (element
 *     (i, j) of S is S[i + j * lds]).  All matrix pointers are DEVICE pointers
 *     owned by the caller; the library never allocates device memory.  Work
 *     memory is a caller-allocated device buffer of rpod_workspace_bytes()
 *     bytes, 256-byte aligned.
 *   - Everything is enqueued asynchronously on `stream` (a cudaStream_t, NULL
 *     for the legacy default stream).  Argument errors are detected on the
 *     host and returned synchronously; errors detected on the device
 *     (non-finite input, no convergence, wait timeout) are recorded in a
 *     status word inside the workspace and reported by rpod_status_sync().
 *     rpod_basis clears the workspace's status block when it starts; the
 *     word then collects that call's errors and those of later
 *     rpod_project/rpod_sample calls until rpod_status_sync clears it.
 *   - Return values are rpod_status codes (0 = success).
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     call returns RPOD_ERR_CUDA.
 */
#ifndef RPOD_H
#define RPOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types.  RPOD_F64/RPOD_F32 select the plain paths; RPOD_BF16 and
 * RPOD_F16 select the tensor-core precision forms (passes over a 16-bit S,
 * FP32 accumulation).  Small steps by form:
 *   F64:         FP64 Grams and Cholesky factors (a shifted first round,
 *                CholeskyQR3); the small SVD is one-sided Jacobi in FP64 on
 *                the transposed Cholesky factor of T T^T (relative accuracy
 *                of small singular values).
 *   F32, 16-bit: Gram partials added as compensated FP32 sums, an FP32
 *                Cholesky factor with a device-gated FP64 refactorization of
 *                an exact-product Gram when a pivot shows a condition number
 *                beyond FP32 reach (F32 form: also in the second CholeskyQR
 *                round when its basis has kappa^2 > 2); the small SVD is the
 *                FP32 eigen start of the Gram T T^T (FP32 products, FP64
 *                sums) refined in FP64, where eigenvalue pairs closer than
 *                the FP32 Gram's rounding level (100 u_32 ||T T^T||_F) keep
 *                an orthonormal basis of their common span. */
typedef enum { RPOD_F64 = 0, RPOD_F32 = 1, RPOD_BF16 = 2, RPOD_F16 = 3 } rpod_dtype;

typedef enum {
  RPOD_OK = 0,
  RPOD_ERR_INVALID_ARG = 1,   /* a size, leading dimension or pointer is invalid */
  RPOD_ERR_UNSUPPORTED = 2,   /* valid but not supported by this build */
  RPOD_ERR_NONFINITE = 3,     /* S holds NaN or Inf (device-detected) */
  RPOD_ERR_BREAKDOWN = 4,     /* every column of a Gram matrix vanished */
  RPOD_ERR_NO_CONVERGENCE = 5,/* small SVD did not converge */
  RPOD_ERR_TIMEOUT = 6,       /* a device-side wait gave up */
  RPOD_ERR_CUDA = 7,          /* a CUDA runtime call failed */
  RPOD_ERR_WORKSPACE = 8,     /* workspace missing, too small or misaligned */
  RPOD_ERR_IO = 9,            /* a model file could not be read or written, or is not one */
  RPOD_ERR_EXCHANGE = 10      /* the exchange callback of rpod_basis_rows reported a failure */
} rpod_status;

/* Warning bits returned through rpod_status_sync()'s flags_out. */
enum {
  RPOD_WARN_RANK_DEFICIENT = 1u  /* a Gram matrix had numerically dependent
                                    columns; the matching basis columns are 0 */
};

/* Plan flags. */
enum {
  RPOD_FLAG_REFINE_FP32 = 1u,  /* 16-bit forms: T = Q^T S reads an FP32 copy */
  RPOD_FLAG_RETURN_ALL_L = 4u, /* U gets all l = k + p columns, not k */
  RPOD_FLAG_HOST_IO = 8u       /* rpod_basis takes HOST pointers for S, U, sigma and
                                  C: S is copied into the workspace (which then holds
                                  room for it, see rpod_workspace_bytes), the outputs
                                  are copied back, all asynchronously on the stream
                                  (host buffers must stay valid until it completes);
                                  S in the compute type (FP32 for the 16-bit forms,
                                  which then refine from it); no S_refine */
};

typedef struct rpod_plan rpod_plan;

/* Creates a plan for one rPOD of an n x m matrix (Alg. 1 inputs: target rank
 * k = N^r >= 1, oversampling p >= 0, subspace iterations q >= 0 -- the paper
 * asks q >= 1; q = 0 is the plain randomized range finder).  Requires
 * l = k + p <= min(n, m, 128).  `seed` keys the Philox4x64-10 stream of the
 * sketch: entry (i, j) of Lambda uses the counter (e/2, 0, 0, 0), e = i + j*m,
 * under the key (seed, 0), and a Box-Muller transform (z0 for even e, z1 for
 * odd e).  `compute` is an rpod_dtype.  The plan owns no device memory; a
 * plan of a 16-bit compute type holds a CUDA stream and two events of the
 * device current at creation (the last CholeskyQR round runs on that stream
 * beside the refinement pass) and is used on that device.
 * Errors: RPOD_ERR_INVALID_ARG for bad sizes or a NULL `out`. */
int rpod_plan_create(rpod_plan** out, int64_t n, int64_t m, int32_t k, int32_t p,
                     int32_t q, uint64_t seed, int32_t compute, uint32_t flags);

/* Caps the one-sided Jacobi sweeps of the FP64 form's small SVD (Alg. 1,
 * SVD of T; default 30, 1 <= max_sweeps <= 1000).  A sweep visits every
 * pair of columns once; the iteration has converged when a sweep rotates no
 * pair.  When the cap is reached first, rpod_basis still writes its outputs
 * (from the last sweep) and rpod_status_sync reports
 * RPOD_ERR_NO_CONVERGENCE.  Errors: RPOD_ERR_INVALID_ARG for a NULL plan or a
 * cap outside the range; RPOD_ERR_UNSUPPORTED for a plan whose compute type
 * is not RPOD_F64 (those forms take no Jacobi sweeps). */
int rpod_plan_set_svd_sweeps(rpod_plan* plan, int32_t max_sweeps);

/* Graph replay of repeated rpod_basis calls (on by default).  The second
 * consecutive call with the same S, S_refine, U, sigma, C and workspace
 * pointers, leading dimensions, s_dtype and workspace size records the
 * call's kernel sequence into one CUDA graph (captured on a stream the plan
 * creates), and later calls with those arguments launch that graph on their
 * stream instead of launching each kernel: the same kernels, arguments and
 * results, without the host work and the gaps between kernels.  A call with
 * other arguments launches directly and starts the count again.  Direct
 * launches are also used while pass profiling is enabled, for row-sharded
 * plans, and when the caller's stream is itself being captured.  The graph
 * reads the buffers at their addresses when it runs, so new contents of S
 * are seen; freeing and reallocating a buffer at the same address is safe.
 * enable = 0 drops the graph and launches directly from then on.  If a
 * capture fails the plan falls back to direct launches for good.
 * Errors: RPOD_ERR_INVALID_ARG for a NULL plan or enable not 0 or 1. */
int rpod_plan_set_graph(rpod_plan* plan, int32_t enable);

/* Bytes of device workspace the plan needs (for any of its calls). */
int rpod_workspace_bytes(const rpod_plan* plan, size_t* bytes);

/* Alg. 1 on S (n x m, element type s_dtype, leading dimension lds >= n).
 *   s_dtype:   RPOD_F64 for compute F64; RPOD_F32 for compute F32; for the
 *              16-bit forms either that 16-bit type or RPOD_F32 (converted
 *              into the workspace on the first pass).
 *   S_refine:  FP32 copy of S (ldr >= n) read by T = Q^T S when
 *              RPOD_FLAG_REFINE_FP32 is set and S itself is 16-bit; ignored
 *              otherwise (an FP32 S is its own refinement copy).
 *   U:         n x k (or n x l with RPOD_FLAG_RETURN_ALL_L), ldu >= n; double
 *              for compute F64, float otherwise.
 *   sigma:     l singular values of T, descending, double.
 *   C:         k x m modal coefficients U_k^T S, ldc >= k; double for F64,
 *              float otherwise.
 * Column signs: each column of U has its largest-magnitude entry positive;
 * C's rows follow.  Columns of U that belong to numerically rank-deficient
 * directions are zero (flagged by RPOD_WARN_RANK_DEFICIENT). */
int rpod_basis(rpod_plan* plan, const void* S, int64_t lds, int32_t s_dtype,
               const float* S_refine, int64_t ldr,
               void* U, int64_t ldu, double* sigma, void* C, int64_t ldc,
               void* workspace, size_t workspace_bytes, void* stream);

/* Galerkin projection of new snapshots on a basis (Sec. 4.3 coefficient
 * matrix applied to held-out data): C' = U^T S', U n x kc (kc <= l), S'
 * n x m_new.  U and C' are double for compute F64, float otherwise; S' has
 * type s_dtype as for rpod_basis.  m_new may exceed the plan's m. */
int rpod_project(const rpod_plan* plan, const void* U, int64_t ldu, int32_t kc,
                 const void* S_new, int64_t lds, int64_t m_new, int32_t s_dtype,
                 void* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                 void* stream);

/* The plan's Gaussian sketch Lambda (Alg. 1, first step) alone: writes the
 * m x l matrix (element type `dtype`, leading dimension ld >= m) to the device
 * buffer Lam.  Same Philox counters as rpod_basis. */
int rpod_sketch(const rpod_plan* plan, void* Lam, int64_t ld, int32_t dtype, void* stream);

/* The sampled matrix of Alg. 1 (second step) for a caller-given sketch, on
 * the tensor-core path of a 16-bit plan: Y = S A with S n x m (ld lds) and
 * A m x l (ld lda >= m), both of the plan's 16-bit type, Y n x l FP32
 * (ld ldy >= n).  S must start on a 16-byte boundary with lds * 2 a multiple
 * of 16 (else RPOD_ERR_UNSUPPORTED).  Uses the workspace. */
int rpod_sample(const rpod_plan* plan, const void* A, int64_t lda, const void* S, int64_t lds,
                int32_t s_dtype, float* Y, int64_t ldy, void* workspace,
                size_t workspace_bytes, void* stream);

/* Pass profiling.  rpod_profile_enable(plan, 1) creates CUDA events and
 * resets the counters; from then on rpod_basis records events on its stream
 * around every pass over S (the products S Lambda, S^T Q, S Z and Q^T S), up
 * to 1024 passes in total.  rpod_profile_read synchronises on the last recorded
 * event and returns, summed over the recorded passes, their number, their
 * device time in ms and their algorithmic bytes and flops (bytes of S and of
 * the skinny operands read or written; 2 n m l flops per product). */
int rpod_profile_enable(rpod_plan* plan, int enable);
int rpod_profile_read(const rpod_plan* plan, int* passes, double* pass_ms, double* bytes,
                      double* flops);

/* Allocation-free variant of rpod_project (the paper has no counterpart; this
 * is a deployment convenience).  For callers that cannot call cudaMalloc or
 * supply a workspace -- a host framework that owns all device memory through
 * its own pool, a plugin whose execute callback may not allocate, a loop that
 * must avoid the device synchronisation an allocation can cause.  The caller
 * still passes U, S' and C' (same meaning, layout and types as rpod_project;
 * compute F64 with double data, otherwise FP32 U, S' and C').  The split-K
 * partial sums live in a 16 MiB array inside the library that every GPU which
 * loads the library holds until the process exits; nothing is allocated.
 * Limit: kc * m_new * sizeof(element) <= 16 MiB, else RPOD_ERR_UNSUPPORTED
 * (project larger S' in column blocks).  Every call outside a stream capture
 * looks up the array's device address (cudaGetSymbolAddress), so a device
 * reset is followed correctly; a call during a capture reuses the address
 * the last call outside one found, so make one call on the device before
 * capturing.  All calls share the array: calls whose kernels
 * overlap on the GPU (several streams or host threads) race and must be
 * serialised by the caller.  No part of the array needs clearing between
 * calls.  Asynchronous on `stream`; argument errors are returned at once. */
int rpod_project_static(const rpod_plan* plan, const void* U, int64_t ldu, int32_t kc,
                        const void* S_new, int64_t lds, int64_t m_new, int32_t s_dtype,
                        void* C, int64_t ldc, void* stream);

/* ---- Row-sharded rPOD --------------------------------------------------
 * Alg. 1 on a matrix whose rows (grid cells) are split into contiguous
 * blocks held by different calls -- one per GPU, each in its own process or
 * host thread.  Every call runs the passes over its own block; at each point
 * where Alg. 1 needs a quantity of the whole matrix the call hands a partial
 * result to the caller's exchange callback, which must combine it with the
 * other blocks' and leave the combined values in place on every block:
 *   the l x l Gram P^T P of each CholeskyQR round   sum   (l^2 values)
 *   Z = S^T Q of each subspace iteration            sum   (m l values)
 *   T = Q^T S                                       sum   (m l values)
 *   the sign rule (largest-magnitude entry of each column of U over all
 *   rows, ties to the lowest global row)            max, min, sum (ku values each)
 * so a pass over S costs one exchange of its small result.  The sketch, the
 * QR of Z, the small SVD and C = Uhat_k^T T are computed identically by
 * every call; U's rows stay with their block.  With q subspace iterations
 * the FP64 form makes 3q + 7 exchanges, in the same order on every block:
 * the Grams of two CholeskyQR rounds per intermediate basis and of three
 * for the final one (2q + 3), Z (q), T (1) and the signs (3).
 *
 * The callback runs on the calling host thread after the work producing
 * buf was enqueued on `stream` (buf is a device pointer into the
 * workspace, `count` values of `dtype` RPOD_F64 or RPOD_F32).  It must
 * complete the combination before later work on `stream` reads buf, e.g.
 * by ncclAllReduce(buf, buf, count, ..., stream) on a communicator over the
 * blocks, or by synchronising the stream and combining on the host.  It
 * returns 0 on success; any other value makes rpod_basis_rows return
 * RPOD_ERR_EXCHANGE at once (the other blocks' calls then wait on their
 * next exchange: the caller must fail them too). */
enum { RPOD_REDUCE_SUM = 0, RPOD_REDUCE_MAX = 1, RPOD_REDUCE_MIN = 2 };
typedef int (*rpod_exchange_fn)(void* ctx, void* buf, int64_t count, int32_t dtype, int32_t op,
                                void* stream);

/* Plan for the row block row0 .. row0 + n_rows - 1 (1 <= n_rows,
 * row0 + n_rows <= n_total) of an n_total x m matrix; k, p, q, seed, compute
 * and flags as for rpod_plan_create, with l <= min(n_total, m, 128).
 * Supported: compute RPOD_F64 (RPOD_ERR_UNSUPPORTED otherwise), flags 0 or
 * RPOD_FLAG_RETURN_ALL_L.  Every block's plan must use the same n_total, m,
 * k, p, q, seed, compute and flags.  Use with rpod_basis_rows only
 * (rpod_basis and rpod_project refuse it with RPOD_ERR_INVALID_ARG). */
int rpod_rows_plan_create(rpod_plan** out, int64_t n_total, int64_t row0, int64_t n_rows,
                          int64_t m, int32_t k, int32_t p, int32_t q, uint64_t seed,
                          int32_t compute, uint32_t flags);

/* Alg. 1 on this plan's row block S_rows (n_rows x m, leading dimension
 * lds >= n_rows, type RPOD_F64).  Writes this block's rows of U (n_rows x ku,
 * ldu >= n_rows), and the whole sigma (l) and C (k x m), identical on every
 * block.  Workspace as for rpod_basis (rpod_workspace_bytes of this plan).
 * Errors: RPOD_ERR_INVALID_ARG for a plan not made by
 * rpod_rows_plan_create, NULL pointers or short leading dimensions;
 * RPOD_ERR_EXCHANGE when the callback fails; device errors through
 * rpod_status_sync as for rpod_basis. */
int rpod_basis_rows(rpod_plan* plan, const void* S_rows, int64_t lds, int32_t s_dtype, void* U_rows,
                    int64_t ldu, double* sigma, void* C, int64_t ldc, void* workspace,
                    size_t workspace_bytes, void* stream, rpod_exchange_fn exchange, void* ctx);

/* ---- Batched rPOD ------------------------------------------------------
 * Many independent instances of Alg. 1 (e.g. the 4 fields psi_1, psi_2, q_1,
 * q_2 of Sec. 2 times the parameter samples mu_k of Sec. 4.1, each with its
 * own snapshot count and rank) run as one unit.  The first rpod_batch_run
 * captures every instance's pipeline into one CUDA graph (instances spread
 * over worker streams inside the graph, costliest first, each to the least
 * loaded stream) and launches it; later runs with the
 * same workspace pointer replay the graph with a single launch.  All
 * pointers in the instance table are device pointers owned by the caller and
 * must stay valid (the graph bakes them in); the data they point to may
 * change between runs. */
typedef struct rpod_instance {
  int64_t n, m;               /* S is n x m */
  int32_t k, p, q;            /* target rank, oversampling, subspace iterations */
  uint64_t seed;              /* Philox key of this instance's sketch */
  const void* S;              /* n x m, ld lds, element type s_dtype of the batch */
  int64_t lds;
  const float* S_refine;      /* FP32 copy for RPOD_FLAG_REFINE_FP32 with 16-bit S, else NULL */
  int64_t ldr;
  void* U;                    /* n x k (n x l with RPOD_FLAG_RETURN_ALL_L) */
  int64_t ldu;
  double* sigma;              /* l values */
  void* C;                    /* k x m */
  int64_t ldc;
} rpod_instance;

typedef struct rpod_batch rpod_batch;

/* Creates a batch of `count` instances (copied; compute and flags as for
 * rpod_plan_create, s_dtype as for rpod_basis).  No device memory (16-bit
 * instances hold a stream and two events each, as their plans do).
 * RPOD_ERR_INVALID_ARG if any instance is invalid for rpod_plan_create. */
int rpod_batch_create(rpod_batch** out, int32_t count, const rpod_instance* inst,
                      int32_t compute, uint32_t flags, int32_t s_dtype);
int rpod_batch_workspace_bytes(const rpod_batch* batch, size_t* bytes);
/* Enqueues the whole batch on `stream` (graph capture on first use). */
int rpod_batch_run(rpod_batch* batch, void* workspace, size_t workspace_bytes, void* stream);
/* Autotuner: times the candidate launch configurations -- worker streams in
 * {1, 2, 4, 8, 16, 32, 64} (up to the instance count) x split-K scale in
 * {1/4, 1/2, 1, 2} of the passes' default split x, for the 16-bit forms, the
 * tensor-core passes' pipeline depth in {2, 4} stages -- as `trials` separately
 * timed replays each (CUDA events on `stream`, synchronising; a point's time
 * is the fastest replay), keeps the fastest point, re-captures, and returns
 * it through best_streams, best_split_pct and best_stages (each may be
 * NULL).  Runs the batch many times: outputs hold the last run's results. */
int rpod_batch_tune(rpod_batch* batch, void* workspace, size_t workspace_bytes, void* stream,
                    int32_t trials, int32_t* best_streams, int32_t* best_split_pct,
                    int32_t* best_stages);
/* Pipeline depth of every instance's tensor-core W- and Y-passes: 0 (the
 * default) chooses by pass size -- two 96 KB stages below 1 GiB, so that two
 * CTAs share an SM, four above -- while 2 or 4 force it (e.g. from a cached
 * tuning).  Errors: RPOD_ERR_INVALID_ARG for other values. */
int rpod_batch_set_pass_stages(rpod_batch* batch, int32_t stages);
/* Sets the launch configuration directly (e.g. from a cached tuning):
 * 1..64 worker streams, split_pct in 10..200. */
int rpod_batch_configure(rpod_batch* batch, int32_t streams, int32_t split_pct);
/* Synchronises, reads and clears every instance's status word; returns the
 * first error found (and its instance index through first_bad, -1 if none)
 * and ORs the warning bits into *flags_out. */
int rpod_batch_status_sync(const rpod_batch* batch, void* workspace, void* stream,
                           int32_t* first_bad, uint32_t* flags_out);
int rpod_batch_last_launch_count(const rpod_batch* batch);
void rpod_batch_destroy(rpod_batch* batch);

/* ---- LSTM on modal coefficients (Sec. 4.3) ------------------------------
 * Maps a window of `window` (= sigma_L) time steps of inputs [mu, alpha_1..N]
 * (Eq. (input); `in_dim` features, the first in_dim - out_dim of them the
 * physical parameters) to the next coefficients (`out_dim` = N features).
 * Cell: gates [i, f, g, o] = W_x x_t + W_h h_{t-1} + b, i, f, o logistic,
 * g tanh, c_t = f c_{t-1} + i g, h_t = o tanh(c_t), h_0 = c_0 = 0; `layers`
 * stacked cells of `hidden` units; linear head y = W_y h_T + b_y.  Loss MSE
 * (mean over batch and outputs); Adam (beta 0.9 / 0.999, eps 1e-8) with the
 * weight decay added to the gradient (Table tab:hyperparam: lr 1e-3, weight
 * decay 1e-5).  Parameters use one flat FP32 vector: per layer W_x
 * (4H x I_l, row-major), W_h (4H x H), b (4H); then W_y (O x H), b_y (O).
 * The weight matrices enter every product as BF16 copies; activations and
 * accumulation are FP32.
 * The caller's workspace (rpod_lstm_workspace_bytes) holds the parameters,
 * the Adam moments and all activations: keep it for the life of the model.
 * Inputs X are row-major (batch, window, in_dim) FP32 device arrays, targets
 * and outputs row-major (batch, out_dim). */
typedef struct rpod_lstm rpod_lstm;

/* rpod_lstm_create flags */
enum {
  RPOD_LSTM_FP32_WEIGHTS = 1u  /* products read the FP32 master weights, not BF16 copies */
};

int rpod_lstm_create(rpod_lstm** out, int32_t in_dim, int32_t hidden, int32_t layers,
                     int32_t out_dim, int32_t window, int32_t max_batch, uint32_t flags);
int64_t rpod_lstm_param_count(const rpod_lstm* net);
int rpod_lstm_workspace_bytes(const rpod_lstm* net, size_t* bytes);
/* Copies the flat parameter vector (host or device pointer) into the
 * workspace and resets Adam's moments and step count. */
int rpod_lstm_set_params(rpod_lstm* net, const float* theta, void* workspace,
                         size_t workspace_bytes, void* stream);
int rpod_lstm_get_params(const rpod_lstm* net, float* theta, void* workspace,
                         size_t workspace_bytes, void* stream);
/* y = net(X) for B <= max_batch windows. */
int rpod_lstm_forward(rpod_lstm* net, const float* X, int32_t B, float* Y, void* workspace,
                      size_t workspace_bytes, void* stream);
/* MSE loss against Y_target and its gradient (flat layout) by
 * backpropagation through time; loss and grad may be NULL (kept in the
 * workspace). */
int rpod_lstm_loss_grad(rpod_lstm* net, const float* X, const float* Y_target, int32_t B,
                        float* loss, float* grad, void* workspace, size_t workspace_bytes,
                        void* stream);
/* loss_grad followed by one Adam update of the parameters. */
int rpod_lstm_train_step(rpod_lstm* net, const float* X, const float* Y_target, int32_t B,
                         float lr, float weight_decay, float* loss, void* workspace,
                         size_t workspace_bytes, void* stream);
/* Training windows from coefficient series: series (n_series, t_len, out_dim)
 * and mu (n_series, d) row-major, idx (B, 2) = (series, first step); writes
 * X[b][t] = [mu[s], series[s][t0 + t]] for t < window and Y[b] =
 * series[s][t0 + window].  Requires d + out_dim == in_dim. */
int rpod_lstm_gather(const rpod_lstm* net, const float* series, const float* mu,
                     int32_t n_series, int32_t t_len, int32_t d, const int32_t* idx, int32_t B,
                     float* X, float* Y, void* stream);
/* Autoregressive prediction (the online stage): from the window (B, window,
 * in_dim), predict, append [mu of the newest row, prediction] as the newest
 * row, drop the oldest, `steps` times; out (B, steps, out_dim).  Runs as one
 * persistent cooperative kernel when the network fits (at most 4 layers; the
 * gate rows of a CTA's hidden units plus the staged inputs of B windows
 * within 200 KB of shared memory): the weights stay in shared memory for all
 * steps, and a grid barrier separates the anti-diagonal phases of the
 * layer x time cells; every barrier wait is limited to 2 s, after which the
 * kernel records RPOD_ERR_TIMEOUT (read by rpod_lstm_status_sync) and
 * returns.  Otherwise one series of kernels per step. */
int rpod_lstm_rollout(rpod_lstm* net, const float* window, int32_t B, int32_t mu_cols,
                      int32_t steps, float* out, void* workspace, size_t workspace_bytes,
                      void* stream);
/* One training epoch: for each of the floor(n_windows / batch) full
 * batches of the window list idx (device, n_windows x 2 int32 pairs
 * (series, first step) in the order to train -- shuffle it beforehand),
 * gather the windows (as rpod_lstm_gather) into the workspace and take one
 * training step (as rpod_lstm_train_step); the last n_windows mod batch
 * windows are left out.  *loss_out (device or host float; may be NULL)
 * receives the mean of the batch losses.  Each pair must satisfy series <
 * n_series and first step + window < t_len (not checked).  Requires
 * batch <= max_batch.  Errors as for rpod_lstm_gather and
 * rpod_lstm_train_step, and RPOD_ERR_INVALID_ARG when no full batch fits. */
int rpod_lstm_train_epoch(rpod_lstm* net, const float* series, const float* mu, int32_t n_series,
                          int32_t t_len, int32_t d, const int32_t* idx, int32_t n_windows,
                          int32_t batch, float lr, float weight_decay, float* loss_out,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Model files.  rpod_lstm_save synchronises `stream` and writes the network's
 * dimensions (in_dim, hidden, layers, out_dim, window, max_batch, flags), its
 * Adam step count, dropout settings, flat FP32 parameters and both Adam
 * moments to `path` (little-endian binary, magic "RPODLSTM", version 1).
 * rpod_lstm_load creates a network of the file's dimensions and keeps the
 * file's state on the host; rpod_lstm_restore then copies that state into a
 * workspace of rpod_lstm_workspace_bytes for the new network, after which
 * it continues exactly where the saved one stopped.  Errors: RPOD_ERR_IO
 * when the file cannot be opened, read or written, or is not a model file of
 * this version; RPOD_ERR_INVALID_ARG for NULL arguments or, for restore, a
 * network without loaded state. */
int rpod_lstm_save(const rpod_lstm* net, const char* path, void* workspace, size_t workspace_bytes,
                   void* stream);
int rpod_lstm_load(rpod_lstm** out, const char* path);
int rpod_lstm_restore(rpod_lstm* net, void* workspace, size_t workspace_bytes, void* stream);
/* dims[0..6] = in_dim, hidden, layers, out_dim, window, max_batch, flags. */
int rpod_lstm_dims(const rpod_lstm* net, int32_t* dims);

/* Dropout between stacked layers (Table tab:hyperparam: 0.1 for the
 * stream-function networks), 0 <= p < 1 (0 switches it off).  In every later
 * training pass (rpod_lstm_loss_grad, rpod_lstm_train_step) the input of each
 * layer above the first is multiplied by keep / (1 - p); forward and
 * rollout never mask.  keep for element e = (t B + b) H + j of the input to
 * layer l (t < window, b < B, j < hidden) at training pass s (counted from 0
 * by this call) is word e mod 4 of the Philox4x64-10 block with counter
 * (e div 4, l, s, 0) and key (seed, 1): kept when that word shifted right by
 * 11 bits is at least ceil(p 2^53).  Errors: RPOD_ERR_INVALID_ARG for a NULL
 * net or p outside [0, 1). */
int rpod_lstm_set_dropout(rpod_lstm* net, double p, uint64_t seed);
int rpod_lstm_last_launch_count(const rpod_lstm* net);
/* Synchronises `stream`, reads and clears the network's device status word
 * (set by a persistent rollout whose barrier wait ran out): RPOD_ERR_TIMEOUT
 * or RPOD_OK.  Errors: RPOD_ERR_INVALID_ARG for NULL arguments. */
int rpod_lstm_status_sync(const rpod_lstm* net, void* workspace, void* stream);

/* Self-test of the persistent rollout's grid barrier (failure detection
 * without a GPU fault): a cooperative kernel of two CTAs in which one never
 * arrives, so the other's bounded wait runs out after `seconds`
 * (0 < seconds <= 2); it records the timeout in a status word of the library
 * and returns.  The call synchronises `stream` and returns RPOD_ERR_TIMEOUT
 * (the designed outcome).  The context stays usable.  Errors:
 * RPOD_ERR_INVALID_ARG for seconds outside (0, 2]. */
int rpod_selftest_grid_barrier(double seconds, void* stream);
void rpod_lstm_destroy(rpod_lstm* net);

/* ---- Time averages, fluctuations and rank selection (Sec. 4.1) ----------
 * The snapshot matrix S (n x m, element type s_dtype, leading dimension
 * lds >= n) holds M = m / nt parameter samples of nt consecutive snapshots
 * each (columns ordered by sample, then time, as in the matrix after
 * Eq. (fluct_psi)); nt must divide m.  Computes the time average of every
 * sample, Eq. (time_av),
 *   Sbar(:, g) = (1/nt) sum_{p < nt} S(:, g nt + p),   g < M,
 * into Sbar (n x M, ldb >= n; double for an FP64 S, float otherwise; rows
 * summed with compensation in that type), and the fluctuation snapshots of
 * Eqs. (fluct_q), (fluct_psi),
 *   F(:, g nt + p) = S(:, g nt + p) - Sbar(:, g),
 * (the difference formed in Sbar's type, then rounded to the output type)
 * into F (ldf >= n, type f_dtype) and/or H (ldh >= n, type h_dtype); either
 * may be NULL (Sbar alone when both are).  Supported types:
 *   s_dtype F64:       F in F64; no H
 *   s_dtype F32:       F in F32, BF16 or F16; H in BF16 or F16 (the 16-bit
 *                      copy the tensor-core forms of rpod_basis read while F
 *                      stays their FP32 refinement copy)
 *   s_dtype BF16/F16:  F in the same type; no H
 * F may be S itself (in place: same type and leading dimension); otherwise
 * F, H, Sbar and S must not overlap.  One kernel, enqueued on `stream`; it
 * reads S once from HBM (a tile of rows of one sample at a time staged in
 * shared memory) unless a 128-byte-high tile of nt snapshots exceeds
 * shared memory (about 1600 FP32 snapshots per sample), when S is read a
 * second time for the write.  Non-finite entries propagate into the means of
 * their rows.  Errors: RPOD_ERR_INVALID_ARG for bad sizes, leading dimensions,
 * types or NULL S/Sbar, or F == S with another type or leading dimension;
 * RPOD_ERR_UNSUPPORTED for a type combination not listed; RPOD_ERR_CUDA when
 * the launch fails. */
int rpod_fluctuations(int64_t n, int64_t m, int64_t nt, const void* S, int64_t lds,
                      int32_t s_dtype, void* F, int64_t ldf, int32_t f_dtype, void* H,
                      int64_t ldh, int32_t h_dtype, void* Sbar, int64_t ldb, void* stream);

/* Energy-based rank of Eq. (energy) on the device: from `count` singular
 * values (device array, double, descending, e.g. rpod_basis's sigma) writes
 * to the device int *rank the smallest N with c_N / c_count >= delta, where
 * c_N = sigma_1 + ... + sigma_N are summed sequentially in double; 0 when
 * c_count is not positive.  With the l values of an rPOD the denominator is
 * the energy of those l values only (the full sum over min(n, m) values of
 * Eq. (energy) is exact when rank(S) <= l).  0 < delta <= 1.  One
 * single-thread kernel on `stream`.  Errors: RPOD_ERR_INVALID_ARG for NULL
 * pointers, count < 1 or delta outside (0, 1]. */
int rpod_energy_rank(const double* sigma, int32_t count, double delta, int32_t* rank,
                     void* stream);

/* Basis files (checkpoints of Alg. 1's output).  rpod_basis_save
 * synchronises `stream` and writes the plan's parameters (n, m, k, p, q,
 * seed, compute, flags) and the outputs of rpod_basis -- U (n x ku, ku = k or
 * l with RPOD_FLAG_RETURN_ALL_L), sigma (l), C (k x m), in the plan's output
 * type, ldu/ldc as for rpod_basis, device or host pointers -- to `path`
 * (little-endian binary, magic "RPODBASE", version 1, column-major packed).
 * rpod_basis_file_info reads info[0..8] = n, m, k, p, q, seed (the 64 bits),
 * compute, flags, ku, enough to allocate the outputs and to recreate the
 * plan; rpod_basis_load copies the three arrays into caller buffers (device
 * or host, leading dimensions >= n and >= k) and synchronises `stream`.
 * Errors: RPOD_ERR_IO for a file that cannot be opened, read or written or
 * is not a basis file of this version; RPOD_ERR_INVALID_ARG for NULL
 * pointers or short leading dimensions; RPOD_ERR_CUDA for a failed copy. */
int rpod_basis_save(const rpod_plan* plan, const char* path, const void* U, int64_t ldu,
                    const double* sigma, const void* C, int64_t ldc, void* stream);
int rpod_basis_file_info(const char* path, int64_t* info);
int rpod_basis_load(const char* path, void* U, int64_t ldu, double* sigma, void* C, int64_t ldc,
                    void* stream);

/* Self-test of the device-side bounded waits (failure detection without a
 * GPU fault): one CTA waits on an mbarrier that nothing arrives on, with the
 * bounded-wait helper of the staged kernels limited to `seconds` (0 < seconds
 * <= 2), records the timeout in a status word of the library and returns;
 * the call synchronises `stream` and returns RPOD_ERR_TIMEOUT (the designed
 * outcome) or RPOD_OK if the wait completed.  The context stays usable.
 * Errors: RPOD_ERR_INVALID_ARG for seconds outside (0, 2]. */
int rpod_selftest_wait_timeout(double seconds, void* stream);

/* Synchronises `stream`, reads and clears the workspace status word.  Returns
 * the device-detected error (RPOD_OK if none) and stores warning bits in
 * *flags_out when it is not NULL. */
int rpod_status_sync(const rpod_plan* plan, void* workspace, void* stream,
                     uint32_t* flags_out);

void rpod_plan_destroy(rpod_plan* plan);

/* Static string for a status code. */
const char* rpod_strerror(int status);

/* Number of kernels the last rpod_basis/rpod_project call on this plan
 * enqueued (for launch accounting). */
int rpod_last_launch_count(const rpod_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* RPOD_H */
