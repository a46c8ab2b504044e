// Internal declarations shared by the librpod translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rpod.h"

namespace rpod {

// NVTX ranges for profilers (ncu --nvtx, nsys): the kernels a call launches
// are attributed to the range open on the calling thread; without a
// profiler attached a push or pop does nothing.  Pass ranges are counted so
// that an entry point's range closes any left open by an error return.
inline thread_local int g_nvtx_passes = 0;
inline void nvtx_pass_push() { nvtxRangePushA("pass"); ++g_nvtx_passes; }
inline void nvtx_pass_pop() {
  if (g_nvtx_passes > 0) { nvtxRangePop(); --g_nvtx_passes; }
}
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() {
    while (g_nvtx_passes > 0) nvtx_pass_pop();
    nvtxRangePop();
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device status word bits (first 32-bit word of the workspace).
enum : unsigned {
  ST_NONFINITE = 1u << 0,
  ST_RANK_DEF = 1u << 1,
  ST_NO_CONV = 1u << 2,
  ST_TIMEOUT = 1u << 3,
  ST_BREAKDOWN = 1u << 4,
};

constexpr int kMaxL = 128;  // one-block limit of the small dense kernels

// Philox4x64-10 (Salmon et al., SC'11): the counter c becomes the block's
// four output words under the key (k0, k1).  Used by the sketch and by the
// LSTM's dropout masks.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    const uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// Kernels enqueued by the calling host thread since the last reset (the
// C ABI reports it per call).
extern thread_local int g_launches;
inline void note_launch() { ++g_launches; }

// ---- generic SIMT GEMM --------------------------------------------------
// C_z = sum_{k in split z} A(i, k) B(k, j) for i < M, j < N,
//   A(i, k) = a_kcontig ? A[k + i*lda] : A[i + k*lda]
//   B(k, j) = B[k + j*ldb]
// Split z covers k in [z*kchunk, min(K, (z+1)*kchunk)) and is stored at
// C + z*csplit + i*ci + j*cj.  TA/TB: stored types, TC: multiply-accumulate
// type, TO: output type.  `check` flags non-finite A entries in *status.
template <typename TA, typename TB, typename TC, typename TO>
cudaError_t gemm(cudaStream_t st, bool a_kcontig, int64_t M, int64_t N, int64_t K,
                 int nsplit, const TA* A, int64_t lda, const TB* B, int64_t ldb,
                 TO* C, int64_t ci, int64_t cj, int64_t csplit,
                 unsigned* status, bool check);

// As gemm, with B(k, j) = bkc ? B[k + j*ldb] : B[k*ldb + j].
template <typename TA, typename TB, typename TC, typename TO>
cudaError_t gemm_ex(cudaStream_t st, bool a_kcontig, bool b_kcontig, int64_t M, int64_t N,
                    int64_t K, int nsplit, const TA* A, int64_t lda, const TB* B, int64_t ldb,
                    TO* C, int64_t ci, int64_t cj, int64_t csplit, unsigned* status, bool check);

// out[i*oi + j*oj] = sum_z part[z*M*N + i + j*M] (summed in double)
template <typename TP, typename TO>
cudaError_t reduce_splits(cudaStream_t st, int64_t M, int64_t N, int nsplit,
                          const TP* part, TO* out, int64_t oi, int64_t oj);

// Lambda (m x l) Philox sketch, stored at Lam[i + j*ld]; caller zeroes padding.
template <typename T>
cudaError_t sketch(cudaStream_t st, uint64_t seed, uint64_t stream_id, int64_t m,
                   int l, T* Lam, int64_t ld);

// One-block Cholesky G = R^T R of the Gram G (l x l, ld = l; FP64 for an
// FP64 TW, FP32 for an FP32 TW; the FP32 kernel reads its upper triangle)
// with a rank-revealing pivot threshold, then X = R^{-1} on the kept
// directions (zero rows and columns for dropped ones), written in TW and,
// when X is not null, in double.  `round` is the CholeskyQR round
// (0 = first): for FP32 working types the first round factors in FP32 and,
// when a pivot signals a condition number beyond FP32 reach, a device-gated
// FP64 factorization takes over -- of the Gram recomputed with exact
// products from Y (rows x l, ld ldy, rows when 0) into the nsplit partials at
// `part`.  FP64 working type only: shift_coef > 0 factors G + shift_coef *
// trace(G) * I (the shifted first round of a shifted CholeskyQR3; only
// exactly vanishing columns are dropped), and flag_tiny raises
// ST_RANK_DEF, without dropping, for columns of squared norm below 1e-16
// (rounds after a shifted one, whose basis is near orthonormal).
// gate_second (FP32 working type, round 1): the second round takes the same
// gated FP64 factorization when its FP32 pivots show kappa(Q1)^2 > 2.
template <typename TW>
cudaError_t cholesky(cudaStream_t st, int l, const void* G, double tol, int round,
                     double* X, TW* Xw, int ldxw, unsigned* status, const float* Y = nullptr,
                     int64_t rows = 0, double* part = nullptr, int nsplit = 0, int64_t ldy = 0,
                     double shift_coef = 0.0, bool flag_tiny = false, bool gate_second = false);

// Symmetric eigen-decomposition of G (l x l, FP64): an FP32 start from the
// tridiagonal reduction, then FP64 Ogita-Aishima refinement.  Outputs
// eigenvalues (descending, as sigma = sqrt(max(lambda, 0))) and eigenvectors
// Uhat (l x l).
cudaError_t sym_eig(cudaStream_t st, int l, const double* G, double* sigma,
                    double* Uhat, double* work, unsigned* status, int refine_iters);

// FP32 starting eigenvectors X (l x l, FP64, column-major, ascending
// eigenvalues) of the symmetric G (l x l, FP64; column i is read as row i) from
// one CTA: Householder tridiagonalization, multisection, twisted
// factorizations.  Writes the number of replaced vectors of multiple
// eigenvalues to status[4] (diagnostic).
cudaError_t tridiag_eig32(cudaStream_t st, int l, const double* G, double* X, float* scratch,
                          unsigned* status);
size_t eig_scratch_floats(int l);
size_t sym_eig_work_doubles(int l);

// Relatively accurate small SVD from the Gram G = T T^T (l x l, FP64) of a
// row-graded T: FP64 Cholesky G = R^T R, then one-sided Jacobi sweeps on the
// columns of L = R^T.  Writes the left singular vectors of T to Uhat (l x l)
// and the singular values to sigma (descending); ST_NO_CONV when max_sweeps
// sweeps still rotate; the sweep count goes to status[5] (diagnostic).
cudaError_t jacobi_svd(cudaStream_t st, int l, const double* G, double* Uhat, double* sigma,
                       unsigned* status, int max_sweeps);
void prepare_jacobi_kernels();

// Column-sign convention: per column c < ncols of U (rows n, ld ldu) find the
// largest |entry| (ties: lowest row) and multiply the column by its sign; the
// same sign is applied to column c of Uhat (l rows, ld l).
template <typename T>
cudaError_t sign_fix(cudaStream_t st, int64_t n, int ncols, T* U, int64_t ldu,
                     double* Uhat, int l, void* scratch, size_t scratch_bytes);
size_t sign_fix_scratch_bytes(int64_t n, int ncols);

// The sign rule when the rows of U are split over row blocks held by
// different calls (row0: this block's first global row).  xb holds 6 ncols
// doubles; between the steps the caller combines over all blocks: xb[0, nc)
// by max after sign_rows_candidates, xb[nc, 2nc) by min after
// sign_rows_step(1), xb[2nc, 3nc) by sum after sign_rows_step(2); then
// sign_rows_apply flips the columns of U and Uhat whose chosen entry is
// negative.  Ties go to the lowest global row, as in sign_fix.
template <typename T>
cudaError_t sign_rows_candidates(cudaStream_t st, int64_t n, int ncols, const T* U, int64_t ldu,
                                 int64_t row0, double* xb, void* scratch, size_t scratch_bytes);
cudaError_t sign_rows_step(cudaStream_t st, int ncols, double* xb, int step);
template <typename T>
cudaError_t sign_rows_apply(cudaStream_t st, int64_t n, int ncols, T* U, int64_t ldu, double* Uhat,
                            int l, double* xb);

template <typename TS, typename TD>
cudaError_t convert_matrix(cudaStream_t st, int64_t rows, int64_t cols, const TS* src,
                           int64_t lds, TD* dst, int64_t ldd);

template <typename T>
cudaError_t check_finite(cudaStream_t st, int64_t rows, int64_t cols, const T* S,
                         int64_t lds, unsigned* status);

// FP32 snapshot matrix -> 16-bit copy (round to nearest), flagging
// non-finite entries; TD is __nv_bfloat16 or __half.
template <typename TD>
cudaError_t convert_snapshots(cudaStream_t st, int64_t rows, int64_t cols, const float* S,
                              int64_t lds, TD* D, int64_t ldd, unsigned* status);

// FP32 copy rounded to TF32 (10-bit mantissa, round to nearest, ties away).
cudaError_t round_tf32(cudaStream_t st, int64_t rows, int64_t cols, const float* src, int64_t lds,
                       float* dst, int64_t ldd);

// FP64 partial Gram matrices part[z] = Y_z^T Y_z of nsplit row chunks of the
// FP32 matrix Y (rows x l, l <= 128), products and chunk sums in FP32.
cudaError_t gram_f32(cudaStream_t st, int64_t rows, int l, const float* Y, int64_t ldy, int nsplit,
                     double* part);

// Persistent LSTM rollout (rpod_rollout.cu): one cooperative launch for all
// `steps` predictions; ring: the window (T x B x I, time-major), hbuf: L x T x
// B x H states, count/abort_word/status: zeroed words (barrier arrivals, the
// abort word, the status word).  rollout_units: hidden units per CTA;
// rollout_smem_bytes: dynamic shared memory of one CTA (the caller checks it
// against the device limit).  grid_sync_selftest: the barrier with one CTA
// that never arrives, limited to `seconds`; returns the status word left.
int rollout_units(int H, int sms);
size_t rollout_smem_bytes(int I, int H, int L, int O, int B, int U);
cudaError_t rollout_persistent(cudaStream_t st, bool bf16_weights, int I, int H, int L, int O, int T,
                               int B, int d, int steps, const float* theta, const void* wbf,
                               const int64_t (*off_w)[3], int64_t off_wy, int64_t off_by,
                               float* ring, float* hbuf, float* out, unsigned* count,
                               int* abort_word, unsigned* status, int sms);
cudaError_t grid_sync_selftest(cudaStream_t st, double seconds, unsigned* status_out);

// Sets every kernel attribute the library needs (dynamic shared memory
// limits) once per process, so that no attribute call happens during a
// stream capture.
void prepare_kernels();
void prepare_kernels_tc();
void prepare_eig_kernels();

// Flags ST_NONFINITE if any of the l values is NaN or Inf.
cudaError_t check_finite_vec(cudaStream_t st, int l, const double* v, unsigned* status);

}  // namespace rpod
