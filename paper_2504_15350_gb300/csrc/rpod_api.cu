// C ABI of librpod (declared in include/rpod.h): plans, workspace layout and
// the host-side orchestration of Alg. 1 (Sec. 4.2) on one CUDA stream.
#include <float.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "rpod_internal.cuh"
#include "rpod_tc.cuh"

using namespace rpod;

namespace rpod {
thread_local int g_launches = 0;
}

struct rpod_plan {
  int64_t n, m;
  int k, p, q, l;
  uint64_t seed;
  int compute;
  uint32_t flags;
  // workspace layout (byte offsets)
  size_t off_status, off_lam, off_y, off_q, off_z, off_zq, off_tt, off_part, off_gpart, off_g,
      off_x, off_xw, off_xu, off_eig, off_sigma, off_uhat, off_sign, total;
  // tensor-core forms: 16-bit copy of S, 16-bit operands (128 columns, zero
  // padded), TF32-rounded basis, split-K partials of the W-pass
  size_t off_sb, off_qb, off_zb, off_atf, off_wpart;
  // RPOD_FLAG_HOST_IO: staging copies of S (ld ld_hs) and of U, sigma, C
  size_t off_hs, off_hu, off_hsig, off_hc;
  int64_t ld_hs;
  int64_t n_ld, m_ld;
  int nsplit_z, nsplit_t, nsplit_w;
  int nsz_def, nsw_def, split_cap;  // default split counts and the scale the buffers allow
  size_t part_elems, gpart_elems, sign_bytes, wpart_elems;
  int last_launches;
  int svd_sweeps;  // cap on the FP64 form's one-sided Jacobi sweeps
  int pass_stages;  // 16-bit passes' pipeline depth: 0 by pass size, else 2 or 4
  // row-sharded plans (rpod_rows_plan_create): this plan's rows are rows
  // row0 .. row0 + n - 1 of an n_total x m matrix whose other row blocks
  // belong to other calls; the exchange callback is set for one
  // rpod_basis_rows call at a time
  int rows_mode;
  int64_t n_total, row0;
  rpod_exchange_fn xch;
  void* xch_ctx;
  size_t off_xch;  // 3 l doubles: the sign rule's exchanged candidates
  // pass profiling
  int prof_on;
  int prof_n;
  cudaEvent_t* prof_ev;  // 2 * kProfPasses events while profiling
  double prof_bytes, prof_flops;
  // side stream and fork/join events (16-bit forms: the last CholeskyQR
  // round runs beside the refinement pass); null when they could not be made
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // graph replay of repeated basis calls: the second call with the same
  // buffers captures the launch sequence (on gcap) into gexec, later calls
  // with those buffers launch the graph on the caller's stream
  int graph_on;
  int graph_calls;  // consecutive calls seen with gkey
  uintptr_t gkey[12];
  cudaStream_t gcap;
  cudaGraphExec_t gexec;
  int graph_launches;  // kernels in the captured graph
};

namespace rpod {
// Passes a profiled plan records (begin and end event each); later passes
// are not recorded.
constexpr int kProfPasses = 1024;

// Read-only view of a plan for the allocation-free projection.
__attribute__((visibility("hidden"))) void plan_shape(const rpod_plan* P, int64_t* n, int32_t* l,
                                                      int32_t* compute, int32_t* nsplit) {
  *n = P->n;
  *l = P->l;
  *compute = P->compute;
  *nsplit = P->nsplit_z;
}

// Pass profiling hooks used by the pipelines; each pass over S is also an
// NVTX range named "pass" (one left open by an error return is closed by the
// entry point's range).
void prof_begin(rpod_plan* P, cudaStream_t st) {
  nvtx_pass_push();
  if (!P->prof_on || P->prof_n >= kProfPasses) return;
  cudaEventRecord(P->prof_ev[2 * P->prof_n], st);
}
void prof_end(rpod_plan* P, cudaStream_t st, double bytes, double flops) {
  nvtx_pass_pop();
  if (!P->prof_on || P->prof_n >= kProfPasses) return;
  cudaEventRecord(P->prof_ev[2 * P->prof_n + 1], st);
  ++P->prof_n;
  P->prof_bytes += bytes;
  P->prof_flops += flops;
}
}  // namespace rpod

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool is16(int dt) { return dt == RPOD_BF16 || dt == RPOD_F16; }

int splits_for(int64_t K, int64_t chunk, int maxs) {
  int64_t s = (K + chunk - 1) / chunk;
  if (s < 1) s = 1;
  if (s > maxs) s = maxs;
  return (int)s;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

#define CK(x)                                        \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return RPOD_ERR_CUDA;     \
  } while (0)
#define CR(x)                                        \
  do {                                               \
    int r_ = (x);                                    \
    if (r_ != RPOD_OK) return r_;                    \
  } while (0)

// ---------------------------------------------------------------------------
// Pipelines on working type W (double for RPOD_F64, float otherwise).
template <typename W>
struct Run {
  rpod_plan* P;
  char* ws;
  cudaStream_t st;
  unsigned* status;

  W* buf(size_t off) { return (W*)(ws + off); }
  double* dbuf(size_t off) { return (double*)(ws + off); }

  // Row-sharded plans: combine `count` values at the device pointer p with
  // every other row block through the caller's exchange callback (after the
  // work that produced them was enqueued on st); no-op otherwise.
  int exchange(void* p, int64_t count, int dtype, int op) {
    if (!P->rows_mode) return RPOD_OK;
    return P->xch(P->xch_ctx, p, count, dtype, op, (void*)st) == 0 ? RPOD_OK : RPOD_ERR_EXCHANGE;
  }

  // Gram G = A^T A (A rows x l, ld lda) in FP64: products in W, summed in W
  // within a split of rows, then in FP64 across splits.  FP32 (when A is
  // TMA-addressable): the tensor-core split-TF32 kernel, with a two-part
  // split when `fast` (only the conditioning of the basis depends on it)
  // and an exact three-part split otherwise; else FP32 products on the SIMT
  // pipes.
  int gram(const W* A, int64_t rows, int64_t lda, double* G, int nsplit, bool fast) {
    const int l = P->l;
    if (sizeof(W) == 4) {
      // the exact kernel holds one CTA per SM: one wave of partials
      const int ns = fast ? nsplit : std::min(nsplit, tc_sm_count());
      float* fpart = (float*)dbuf(P->off_gpart);
      int rc = tc_gram(st, (const float*)A, lda, rows, l, fpart, ns, status, !fast);
      // FP32 working type: FP32 partials summed in FP64, the Gram stored in
      // FP32 for the FP32 Cholesky
      if (rc == RPOD_OK) {
        CK((reduce_splits<float, float>(st, l, l, ns, fpart, (float*)G, 1, l)));
        return RPOD_OK;
      }
      if (rc == RPOD_ERR_CUDA) return rc;
      CK(gram_f32(st, rows, l, (const float*)A, lda, nsplit, dbuf(P->off_gpart)));
      CK((reduce_splits<double, float>(st, l, l, nsplit, dbuf(P->off_gpart), (float*)G, 1, l)));
      return RPOD_OK;
    } else
      CK((gemm<W, W, W, double>(st, true, l, l, rows, nsplit, A, lda, A, lda, dbuf(P->off_gpart), 1,
                                l, (int64_t)l * l, status, false)));
    CK((reduce_splits<double, double>(st, l, l, nsplit, dbuf(P->off_gpart), G, 1, l)));
    return RPOD_OK;
  }

  // CholeskyQR with `rounds` passes (CholeskyQR2 for rounds = 2); returns the
  // buffer holding Q (in or tmp).  Only the conditioning of an intermediate
  // basis matters (its span comes from the FP32 product Y R^{-1}), so its
  // Gram may take the split-TF32 tensor path; with `exact_last` the last
  // round, which fixes the orthogonality of the returned basis, keeps FP32
  // products.
  // With `defer` the last round stops after its Cholesky factor: the
  // returned buffer holds the previous round's basis Q1 and the final basis
  // is Q1 X with X = R^{-1} left in off_x (FP64) and off_xw (W); the caller
  // folds X into the small matrices (T = X^T Q1^T S, U = Q1 (X Uhat)), which
  // saves one n x l x l product.
  // Outputs of the last apply of a CholeskyQR on the tensor-core path:
  // the basis rounded to the 16-bit type (h16) and/or to TF32 (tf), the
  // FP32 basis itself only when f32 is set; `used` reports whether the
  // tensor-core apply ran (else the FP32 basis was formed on the SIMT path
  // and the rounded copies were not written).
  struct TcOut {
    void* h16;
    float* tf;
    bool f32;
    bool used;
    int64_t ldo = 0;  // leading dimension of h16 and tf (P->n_ld when 0)
  };

  // `ld`: leading dimension of in and tmp (rows when 0).
  // `dist`: the rows are this plan's block of a row-sharded matrix, so each
  // round's Gram is summed over the row blocks before its factorization.
  int orth(W* in, W* tmp, int64_t rows, int rounds, W** out, bool exact_last, bool defer = false,
           TcOut* tco = nullptr, int64_t ld = 0, bool dist = false) {
    if (ld == 0) ld = rows;
    const int l = P->l;
    const double tol = sizeof(W) == 8 ? 1e-13 : 1e-5;
    // FP32 Gram: two row chunks per SM (the kernel fits two blocks per SM).
    // FP64 Gram: 32-row chunks -- GB300 issues about two FP64 FMAs per clock
    // per SM, so the l^2 x rows products must spread over many SMs
    const int ns = sizeof(W) == 8 ? splits_for(rows, 32, 256)
                                  : (int)std::max<int64_t>(1, std::min<int64_t>(2 * 152, rows / 256));
    W* src = in;
    W* dst = tmp;
    // FP64 form: shifted CholeskyQR (the first round factors G + s I), so
    // that sampled matrices whose condition number reaches u^-1 keep every
    // direction; the callers add one round for it
    const double grows = (dist && P->rows_mode) ? (double)P->n_total : (double)rows;
    const double shift_coef =
        sizeof(W) == 8 ? 11.0 * (grows * l + (double)l * (l + 1)) * (DBL_EPSILON / 2) : 0.0;
    for (int r = 0; r < rounds; ++r) {
      double* G = dbuf(P->off_g);
      CR(gram(src, rows, ld, G, ns, !(exact_last && r == rounds - 1)));
      if (dist) CR(exchange(G, (int64_t)l * l, sizeof(W) == 8 ? RPOD_F64 : RPOD_F32, RPOD_REDUCE_SUM));
      // the FP64 copy of R^-1 is read only for a deferred last round (and
      // by the FP64 form)
      double* xd = (sizeof(W) == 8 || (defer && r == rounds - 1)) ? dbuf(P->off_x) : nullptr;
      CK((cholesky<W>(st, l, G, tol, r, xd, buf(P->off_xw), l, status,
                      sizeof(W) == 4 ? (const float*)src : nullptr, rows, dbuf(P->off_gpart), ns, ld,
                      r == 0 ? shift_coef : 0.0, sizeof(W) == 8 && r > 0,
                      P->compute == RPOD_F32 && r == 1)));
      if (defer && r == rounds - 1) break;
      const bool last_apply = r == rounds - 1 - (defer ? 1 : 0);
      int rc = RPOD_ERR_UNSUPPORTED;
      if (sizeof(W) == 4 && tco && last_apply)
        rc = tc_apply(st, (const float*)src, ld, rows, l, (const float*)buf(P->off_xw), l,
                      tco->f32 ? (float*)dst : nullptr, rows, P->compute, tco->h16,
                      tco->ldo ? tco->ldo : P->n_ld, tco->tf, tco->ldo ? tco->ldo : P->n_ld,
                      status);
      if (rc == RPOD_ERR_CUDA) return rc;
      if (tco && last_apply) tco->used = rc == RPOD_OK;
      if (rc != RPOD_OK)
        CK((gemm<W, W, W, W>(st, false, rows, l, l, 1, src, ld, buf(P->off_xw), l, dst, 1, ld, 0,
                             status, false)));
      W* t = src; src = dst; dst = t;
    }
    *out = src;
    return RPOD_OK;
  }

  // The deferred last CholeskyQR round of the basis Q1 (rows x l, ld rows):
  // exact Gram and its factor X2 = R2^{-1} (in off_x and off_xw), no apply.
  int last_factor(const W* Q1, int64_t rows) {
    const int l = P->l;
    const double tol = sizeof(W) == 8 ? 1e-13 : 1e-5;
    const int ns = sizeof(W) == 8 ? splits_for(rows, 4096, 256)
                                  : (int)std::max<int64_t>(1, std::min<int64_t>(2 * 152, rows / 256));
    double* G = dbuf(P->off_g);
    CR(gram(Q1, rows, rows, G, ns, false));
    CK((cholesky<W>(st, l, G, tol, 1, dbuf(P->off_x), buf(P->off_xw), l, status,
                    sizeof(W) == 4 ? (const float*)Q1 : nullptr, rows, dbuf(P->off_gpart), ns, rows)));
    return RPOD_OK;
  }

  // Fold a deferred last CholeskyQR factor into T: Tt (m x l) = Tt1 X,
  // written to `out` (m x l).
  int fold_t(const W* Tt1, W* out) {
    const int64_t m = P->m;
    const int l = P->l;
    // 16-bit forms: the two-part TF32 tensor-core product (about 2^-21
    // relative error per entry, as the lift); else, or when Tt1 is not
    // addressable by TMA, the SIMT product
    int rc = RPOD_ERR_UNSUPPORTED;
    if (sizeof(W) == 4 && is16(P->compute))
      rc = tc_apply(st, (const float*)Tt1, m, m, l, (const float*)buf(P->off_xw), l, (float*)out, m,
                    0, nullptr, 0, nullptr, 0, status, 0, true);
    if (rc == RPOD_ERR_CUDA) return rc;
    if (rc != RPOD_OK)
      CK((gemm<W, W, W, W>(st, false, m, l, l, 1, Tt1, m, buf(P->off_xw), l, out, 1, m, 0, status,
                           false)));
    return RPOD_OK;
  }

  // After T (as Tt, m x l): small SVD, lift, signs, coefficients.  With
  // `deferred` the basis is Q X (X from the deferred last CholeskyQR round)
  // and the lift uses X Uhat.
  int finish(const W* Q, const W* Tt, W* U, int64_t ldu, double* sigma, W* C, int64_t ldc,
             bool deferred = false) {
    const int64_t n = P->n, m = P->m;
    const int l = P->l, k = P->k;
    // Alg. 1: SVD of T via the eigenpairs of T T^T (FP64 Gram)
    double* GT = dbuf(P->off_g);
    const int ns = P->nsplit_t;
    CK((gemm<W, W, W, double>(st, true, l, l, m, ns, Tt, m, Tt, m, dbuf(P->off_gpart), 1, l,
                              (int64_t)l * l, status, false)));
    CK((reduce_splits<double, double>(st, l, l, ns, dbuf(P->off_gpart), GT, 1, l)));
    double* Uhat = dbuf(P->off_uhat);
    if (sizeof(W) == 8) {
      // FP64 form: one-sided Jacobi sweeps on the transposed Cholesky factor
      // of the Gram, which keep the relative accuracy of small singular
      // values (an eigen-decomposition of the Gram is accurate only
      // relative to sigma_1^2)
      CK(jacobi_svd(st, l, GT, Uhat, sigma, status, P->svd_sweeps));
    } else {
      // FP32 and 16-bit forms: FP32 start from the tridiagonal reduction
      // (eigenvectors to about 1e-5), then FP64 refinement passes, each of
      // which squares the eigenvector error outside clusters and restores
      // orthogonality; the cluster threshold of a pass scales with the norm
      // of all remaining off-diagonal terms, so eigenvalues closer than that
      // are separated only by a later pass, and never below the rounding
      // level of the FP32 Gram (100 u_32 ||A||).  The 16-bit forms, whose passes
      // over S hold sigma to 1e-4 (BF16) or 1e-5 (FP16), take one pass
      // (eigenvector error near 1e-10); the FP32 form takes two.
      CK((sym_eig(st, l, GT, sigma, Uhat, dbuf(P->off_eig), status, is16(P->compute) ? 1 : 2)));
    }
    CK((check_finite_vec(st, l, sigma, status)));
    // Alg. 1: lift U = Q Uhat (first k or all l columns), then the sign rule
    const int ku = (P->flags & RPOD_FLAG_RETURN_ALL_L) ? l : k;
    const double* Ul = Uhat;
    if (deferred) {
      double* XU = dbuf(P->off_xu);
      CK((gemm<double, double, double, double>(st, false, l, ku, l, 1, dbuf(P->off_x), l, Uhat, l, XU,
                                               1, l, 0, status, false)));
      Ul = XU;
    }
    // The small factor enters the n- and m-sized products in W: converted
    // once here rather than per tile load (FP64 conversions are slow on
    // GB300).  off_xw (l x l in W) is free after fold_t.
    W* Uw = buf(P->off_xw);
    CK((convert_matrix<double, W>(st, l, ku, Ul, l, Uw, l)));
    // 16-bit forms: the lift on the tensor cores with a hi/lo TF32 split of
    // both operands (about 2^-21 relative error); the plain forms, or a basis
    // that TMA cannot address, on the SIMT pipes
    int rc = RPOD_ERR_UNSUPPORTED;
    if (sizeof(W) == 4 && is16(P->compute))
      rc = tc_apply(st, (const float*)Q, n, n, l, (const float*)Uw, l, (float*)U, ldu, 0, nullptr, 0,
                    nullptr, 0, status, ku, true);
    if (rc == RPOD_ERR_CUDA) return rc;
    if (rc != RPOD_OK)
      CK((gemm<W, W, W, W>(st, false, n, ku, l, 1, Q, n, Uw, l, U, 1, ldu, 0, status, false)));
    if (P->rows_mode) {
      // the largest-magnitude entry of each column over all row blocks (ties
      // to the lowest global row) decides its sign: three exchanges of l
      // values -- the largest magnitude, the lowest row holding it, the sign
      // of the entry there
      double* xb = dbuf(P->off_xch);
      CK((sign_rows_candidates<W>(st, n, ku, U, ldu, P->row0, xb, ws + P->off_sign, P->sign_bytes)));
      CR(exchange(xb, ku, RPOD_F64, RPOD_REDUCE_MAX));
      CK(sign_rows_step(st, ku, xb, 1));
      CR(exchange(xb + ku, ku, RPOD_F64, RPOD_REDUCE_MIN));
      CK(sign_rows_step(st, ku, xb, 2));
      CR(exchange(xb + 2 * ku, ku, RPOD_F64, RPOD_REDUCE_SUM));
      CK((sign_rows_apply<W>(st, n, ku, U, ldu, Uhat, l, xb)));
    } else {
      CK((sign_fix<W>(st, n, ku, U, ldu, Uhat, l, ws + P->off_sign, P->sign_bytes)));
    }
    // Sec. 4.3 coefficients C = U_k^T S = Uhat_k^T T (k x m), Uhat with the signs
    CK((convert_matrix<double, W>(st, l, k, Uhat, l, Uw, l)));
    CK((gemm<W, W, W, W>(st, false, m, k, l, 1, Tt, m, Uw, l, C, ldc, 1, 0, status, false)));
    return RPOD_OK;
  }

  int run(const W* S, int64_t lds, W* U, int64_t ldu, double* sigma, W* C, int64_t ldc) {
    const int64_t n = P->n, m = P->m;
    const int l = P->l, q = P->q;
    W* Lam = buf(P->off_lam);
    W* Y = buf(P->off_y);
    W* Qb = buf(P->off_q);
    W* Z = buf(P->off_z);
    W* Zq = buf(P->off_zq);
    W* Tt = buf(P->off_tt);
    W* part = buf(P->off_part);
    const double sw = sizeof(W);
    const double pass_bytes = sw * ((double)n * m + (double)n * l + (double)m * l);
    const double pass_flops = 2.0 * n * m * l;
    // the shifted first CholeskyQR round of the FP64 form (see orth)
    const int extra = sizeof(W) == 8 ? 1 : 0;
    // Alg. 1: Gaussian sketch
    CK((sketch<W>(st, P->seed, 0, m, l, Lam, m)));
    // Alg. 1: P = S Lambda (pass over S; flags non-finite input)
    prof_begin(P, st);
    CK((gemm<W, W, W, W>(st, false, n, l, m, 1, S, lds, Lam, m, Y, 1, n, 0, status, true)));
    prof_end(P, st, pass_bytes, pass_flops);
    W* Q = nullptr;
    for (int it = 0; it <= q; ++it) {
      if (it > 0) {
        // Alg. 1 subspace iteration: Z = S^T Q, orthonormalise, Y = S Z
        prof_begin(P, st);
        CK((gemm<W, W, W, W>(st, true, m, l, n, P->nsplit_z, S, lds, Q, n, part, 1, m, m * l,
                             status, false)));
        prof_end(P, st, pass_bytes, pass_flops);
        CK((reduce_splits<W, W>(st, m, l, P->nsplit_z, part, Z, 1, m)));
        CR(exchange(Z, m * l, sizeof(W) == 8 ? RPOD_F64 : RPOD_F32, RPOD_REDUCE_SUM));
        W* Zo = nullptr;
        CR(orth(Z, Zq, m, 1 + extra, &Zo, false));
        prof_begin(P, st);
        CK((gemm<W, W, W, W>(st, false, n, l, m, 1, S, lds, Zo, m, Y, 1, n, 0, status, false)));
        prof_end(P, st, pass_bytes, pass_flops);
      }
      // Alg. 1 QR of the sampled matrix (CholeskyQR2 for the final basis);
      // Y's buffer is free again once Z = S^T Q is formed
      CR(orth(Y, Qb, n, (it == q ? 2 : 1) + extra, &Q, it == q, it == q, nullptr, 0, true));
    }
    // Alg. 1: T = Q^T S, stored transposed (m x l), with the deferred last
    // CholeskyQR factor folded in afterwards
    prof_begin(P, st);
    CK((gemm<W, W, W, W>(st, true, m, l, n, P->nsplit_z, S, lds, Q, n, part, 1, m, m * l, status,
                         false)));
    prof_end(P, st, pass_bytes, pass_flops);
    CK((reduce_splits<W, W>(st, m, l, P->nsplit_z, part, Zq, 1, m)));
    CR(exchange(Zq, m * l, sizeof(W) == 8 ? RPOD_F64 : RPOD_F32, RPOD_REDUCE_SUM));
    CR(fold_t(Zq, Tt));
    return finish(Q, Tt, U, ldu, sigma, C, ldc, true);
  }

  // Tensor-core form (W = float): passes over a 16-bit S on tcgen05, the
  // final T = Q^T S on TF32 from an FP32 copy when refining.
  int run_tc(const void* S_in, int64_t lds_in, int s_dtype, const float* Sref, int64_t ldr,
             float* U, int64_t ldu, double* sigma, float* C, int64_t ldc) {
    const int64_t n = P->n, m = P->m;
    const int l = P->l, q = P->q;
    const int dt = P->compute;  // RPOD_BF16 or RPOD_F16
    float* Y = (float*)buf(P->off_y);
    float* Qbuf = (float*)buf(P->off_q);
    float* Z = (float*)buf(P->off_z);
    float* Zq = (float*)buf(P->off_zq);
    float* Tt = (float*)buf(P->off_tt);
    float* wpart = (float*)(ws + P->off_wpart);
    void* Qh = ws + P->off_qb;   // n_ld x 128, 16-bit
    void* Zh = ws + P->off_zb;   // m_ld x 128, 16-bit
    const int64_t nld = P->n_ld, mld = P->m_ld;
    // Columns l..127 of the 16-bit operand buffers are never read: the tensor
    // maps span l columns and TMA fills the rest of each 128-wide box with 0.
    // the 16-bit S read by the passes
    const void* Sh = S_in;
    int64_t ldh = lds_in;
    const double pass_flops = 2.0 * n * m * l;
    const double pb16 = 2.0 * ((double)n * m + (double)n * l + (double)m * l);
    auto to16 = [&](const float* src, int64_t rows, int64_t ldsrc, void* dst, int64_t ldd) -> cudaError_t {
      if (dt == RPOD_BF16)
        return convert_matrix<float, __nv_bfloat16>(st, rows, l, src, ldsrc, (__nv_bfloat16*)dst, ldd);
      return convert_matrix<float, __half>(st, rows, l, src, ldsrc, (__half*)dst, ldd);
    };
    // Alg. 1: Gaussian sketch, directly in the 16-bit operand layout
    if (dt == RPOD_BF16)
      CK((sketch<__nv_bfloat16>(st, P->seed, 0, m, l, (__nv_bfloat16*)Zh, mld)));
    else
      CK((sketch<__half>(st, P->seed, 0, m, l, (__half*)Zh, mld)));
    // Alg. 1: P = S Lambda.  An FP32 S is rounded to the 16-bit type by the
    // same pass, which also leaves the 16-bit copy for the later passes.
    if (s_dtype == RPOD_F32) {
      void* Sb = ws + P->off_sb;
      prof_begin(P, st);
      int rc = tc_ypass_cvt(st, dt, Zh, mld, (const float*)S_in, lds_in, n, m, l, Y, n, Sb, nld,
                            status, wpart, P->wpart_elems);
      if (rc == RPOD_ERR_UNSUPPORTED) {
        if (dt == RPOD_BF16)
          CK(convert_snapshots<__nv_bfloat16>(st, n, m, (const float*)S_in, lds_in,
                                              (__nv_bfloat16*)Sb, nld, status));
        else
          CK(convert_snapshots<__half>(st, n, m, (const float*)S_in, lds_in, (__half*)Sb, nld,
                                       status));
        rc = tc_ypass(st, dt, Zh, mld, Sb, nld, n, m, l, Y, n, status, wpart, P->wpart_elems, P->pass_stages);
        CR(rc);
        prof_end(P, st, 6.0 * (double)n * m + pb16, pass_flops);
      } else {
        CR(rc);
        prof_end(P, st, 6.0 * (double)n * m + 2.0 * (double)m * l + 4.0 * (double)n * l, pass_flops);
      }
      Sh = Sb;
      ldh = nld;
      if (!Sref) { Sref = (const float*)S_in; ldr = lds_in; }
    } else {
      prof_begin(P, st);
      CR(tc_ypass(st, dt, Zh, mld, Sh, ldh, n, m, l, Y, n, status, wpart, P->wpart_elems, P->pass_stages));
      prof_end(P, st, pb16, pass_flops);
    }
    float* Q = nullptr;
    const bool refine_req = (P->flags & RPOD_FLAG_REFINE_FP32) && Sref;
    // BF16: the refinement pass on the TF32 tensor path (S and Q rounded to
    // TF32, about 2e-5 relative error in sigma, below the form's 1e-4 bound).
    // FP16 stores S to 2^-11 and is held to 1e-5: its refinement pass keeps
    // exact FP32 products (SIMT), which the TF32 rounding would not
    const bool refine_tma = refine_req && dt == RPOD_BF16 && (((uintptr_t)Sref & 15) == 0) &&
                            ((ldr * 4) % 16 == 0);
    float* const Atf = (float*)(ws + P->off_atf);
    bool tf_ready = false;
    for (int it = 0; it <= q; ++it) {
      if (it > 0) {
        // Alg. 1 subspace iteration: Z = S^T Q, orthonormalise, Y = S Z
        prof_begin(P, st);
        CR(tc_wpass(st, dt, Qh, nld, n, l, Sh, ldh, m, wpart, P->nsplit_w, status, P->pass_stages));
        prof_end(P, st, pb16, pass_flops);
        // Z with a 16-byte aligned leading dimension, so that its Gram
        // takes the tensor-core path at any m
        const int64_t m4 = round_up(m, 4);
        CK((reduce_splits<float, float>(st, m, l, P->nsplit_w, wpart, Z, 1, m4)));
        // the orthonormal Z goes straight to its 16-bit copy for the Y-pass
        // (the tensor-core apply; the SIMT product and a conversion when Z
        // is not addressable by TMA)
        float* Zo = nullptr;
        TcOut tz{Zh, nullptr, false, false, mld};
        CR(orth(Z, Zq, m, 1, &Zo, false, false, &tz, m4));
        if (!tz.used) CK(to16(Zo, m, m4, Zh, mld));
        prof_begin(P, st);
        CR(tc_ypass(st, dt, Zh, mld, Sh, ldh, n, m, l, Y, n, status, wpart, P->wpart_elems, P->pass_stages));
        prof_end(P, st, pb16, pass_flops);
      }
      // the final basis is kept in FP32 (lift, Gram of the deferred round)
      // and rounded to TF32 for the refinement pass; intermediate ones are
      // needed only as the 16-bit operand of the next W-pass
      TcOut tco{it < q ? Qh : nullptr, it == q && refine_tma ? Atf : nullptr, it == q, false};
      if (it == q && P->side) {
        // first round only: the exact second round (which fixes the returned
        // basis' orthogonality, not the span the refinement pass reads) runs
        // on the side stream beside the refinement pass
        CR(orth(Y, Qbuf, n, 1, &Q, false, false, &tco));
      } else {
        CR(orth(Y, Qbuf, n, it == q ? 2 : 1, &Q, it == q, it == q, &tco));
      }
      if (it < q && !tco.used) CK(to16(Q, n, n, Qh, nld));
      tf_ready = it == q && tco.used && refine_tma;
    }
    bool forked = false;
    if (P->side) {
      CK(cudaEventRecord(P->ev_fork, st));
      CK(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
      cudaStream_t main_st = st;
      st = P->side;
      const int rc = last_factor(Q, n);
      st = main_st;
      CR(rc);
      CK(cudaEventRecord(P->ev_join, P->side));
      forked = true;
    }
    // join before the factor is used (fold_t, finish)
    auto join = [&]() -> cudaError_t {
      return forked ? cudaStreamWaitEvent(st, P->ev_join, 0) : cudaSuccess;
    };
    // Alg. 1: T = Q^T S (TF32 from the FP32 copy when refining)
    const bool refine = refine_req;
    const bool ref_tma = refine_tma;
    if (refine && !ref_tma) {
      // FP32 copy not addressable by TMA: the SIMT FP32 pass computes T
      prof_begin(P, st);
      CK((gemm<float, float, float, float>(st, true, m, l, n, P->nsplit_z, Sref, ldr, Q, n,
                                           (float*)buf(P->off_part), 1, m, m * l, status, false)));
      prof_end(P, st, 4.0 * ((double)n * m + (double)n * l + (double)m * l), pass_flops);
      CK((reduce_splits<float, float>(st, m, l, P->nsplit_z, (float*)buf(P->off_part), Zq, 1, m)));
      CK(join());
      CR(fold_t(Zq, Tt));
      return finish(Q, Tt, U, ldu, sigma, C, ldc, true);
    }
    if (refine) {
      if (!tf_ready) CK(round_tf32(st, n, l, Q, n, Atf, nld));
      prof_begin(P, st);
      CR(tc_wpass(st, RPOD_F32, Atf, nld, n, l, Sref, ldr, m, wpart, P->nsplit_w, status, P->pass_stages));
      prof_end(P, st, 4.0 * ((double)n * m + (double)n * l + (double)m * l), pass_flops);
    } else {
      CK(to16(Q, n, n, Qh, nld));
      prof_begin(P, st);
      CR(tc_wpass(st, dt, Qh, nld, n, l, Sh, ldh, m, wpart, P->nsplit_w, status, P->pass_stages));
      prof_end(P, st, pb16, pass_flops);
    }
    CK((reduce_splits<float, float>(st, m, l, P->nsplit_w, wpart, Zq, 1, m)));
    CK(join());
    CR(fold_t(Zq, Tt));
    return finish(Q, Tt, U, ldu, sigma, C, ldc, true);
  }

  int project(const W* U, int64_t ldu, int kc, const W* Sn, int64_t lds, int64_t mn, W* C,
              int64_t ldc) {
    const int64_t n = P->n;
    // C'^T (mn x kc) = S'^T U, split over n, chunked over snapshots so the
    // partial buffer of the plan suffices
    const int64_t per = (int64_t)(P->part_elems / ((size_t)P->nsplit_z * (size_t)kc));
    const int64_t cols = per < 1 ? 1 : per;
    for (int64_t j0 = 0; j0 < mn; j0 += cols) {
      const int64_t mc = (mn - j0 < cols) ? (mn - j0) : cols;
      W* part = buf(P->off_part);
      CK((gemm<W, W, W, W>(st, true, mc, kc, n, P->nsplit_z, Sn + j0 * lds, lds, U, ldu, part, 1, mc,
                           mc * kc, status, false)));
      CK((reduce_splits<W, W>(st, mc, kc, P->nsplit_z, part, C + j0 * ldc, ldc, 1)));
    }
    return RPOD_OK;
  }

  // 16-bit S': the W-pass with U converted to the 16-bit operand layout.
  int project_tc(const float* U, int64_t ldu, int kc, const void* Sn, int64_t lds, int64_t mn,
                 float* C, int64_t ldc) {
    const int64_t n = P->n;
    const int dt = P->compute;
    void* Qh = ws + P->off_qb;
    float* wpart = (float*)(ws + P->off_wpart);
    if (dt == RPOD_BF16)
      CK((convert_matrix<float, __nv_bfloat16>(st, n, kc, U, ldu, (__nv_bfloat16*)Qh, P->n_ld)));
    else
      CK((convert_matrix<float, __half>(st, n, kc, U, ldu, (__half*)Qh, P->n_ld)));
    const int64_t per = (int64_t)(P->wpart_elems / ((size_t)64 * (size_t)kc));
    const int64_t cols = std::max<int64_t>(256, per / 256 * 256);
    for (int64_t j0 = 0; j0 < mn; j0 += cols) {
      const int64_t mc = std::min(mn - j0, cols);
      const int ns = tc_wpass_splits(n, mc, dt);
      if ((size_t)ns * kc * mc > P->wpart_elems) return RPOD_ERR_WORKSPACE;
      CR(tc_wpass(st, dt, Qh, P->n_ld, n, kc, (const char*)Sn + (size_t)j0 * lds * 2, lds, mc, wpart,
                  ns, status));
      CK((reduce_splits<float, float>(st, mc, kc, ns, wpart, C + j0 * ldc, ldc, 1)));
    }
    return RPOD_OK;
  }
};

}  // namespace

extern "C" {

const char* rpod_strerror(int s) {
  switch (s) {
    case RPOD_OK: return "ok";
    case RPOD_ERR_INVALID_ARG: return "invalid argument";
    case RPOD_ERR_UNSUPPORTED: return "unsupported";
    case RPOD_ERR_NONFINITE: return "non-finite input";
    case RPOD_ERR_BREAKDOWN: return "Gram matrix breakdown";
    case RPOD_ERR_NO_CONVERGENCE: return "small SVD did not converge";
    case RPOD_ERR_TIMEOUT: return "device wait timed out";
    case RPOD_ERR_CUDA: return "CUDA error";
    case RPOD_ERR_WORKSPACE: return "workspace missing or too small";
    case RPOD_ERR_IO: return "file could not be read or written";
    case RPOD_ERR_EXCHANGE: return "exchange callback failed";
    default: return "unknown status";
  }
}

// split_cap: the split-K counts of the passes may later be scaled up to this
// factor (the batch autotuner), so the partial buffers are sized for it.
// n_rank: the row count that bounds l (n, or n_total for a row block).
static int plan_create_impl(rpod_plan** out, int64_t n, int64_t m, int32_t k, int32_t p,
                            int32_t q, uint64_t seed, int32_t compute, uint32_t flags,
                            int split_cap, int64_t n_rank = 0) {
  if (!out) return RPOD_ERR_INVALID_ARG;
  *out = nullptr;
  const int64_t l = (int64_t)k + p;
  if (n_rank == 0) n_rank = n;
  if (n < 1 || m < 1 || k < 1 || p < 0 || q < 0 || l > n_rank || l > m || l > kMaxL)
    return RPOD_ERR_INVALID_ARG;
  if (compute < RPOD_F64 || compute > RPOD_F16) return RPOD_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(RPOD_FLAG_REFINE_FP32 | RPOD_FLAG_RETURN_ALL_L | RPOD_FLAG_HOST_IO))
    return RPOD_ERR_INVALID_ARG;
  if (n > ((int64_t)1 << 31) - 1024 || m > ((int64_t)1 << 31) - 1024) return RPOD_ERR_UNSUPPORTED;
  rpod_plan* P = new (std::nothrow) rpod_plan();
  if (!P) return RPOD_ERR_INVALID_ARG;
  P->n = n; P->m = m; P->k = k; P->p = p; P->q = q; P->l = (int)l;
  P->seed = seed; P->compute = compute; P->flags = flags;
  const size_t w = (compute == RPOD_F64) ? 8 : 4;
  const size_t L = (size_t)l;
  // split-K counts of the S^T Q products (over n) and of the Gram T T^T
  // (over m): the FP64 form splits finely (its products run at the narrow
  // FP64 rate, so they need many SMs even for small matrices)
  P->nsplit_z = splits_for(n, compute == RPOD_F64 ? 256 : 8192, 64);
  P->nsplit_t = splits_for(m, compute == RPOD_F64 ? 32 : 256, 512);
  const int nsg = 2 * 152;
  P->split_cap = split_cap < 1 ? 1 : split_cap;
  P->nsz_def = P->nsplit_z;
  P->part_elems = std::max((size_t)P->nsplit_z * P->split_cap * m * L, (size_t)1);
  P->gpart_elems = std::max((size_t)nsg, (size_t)P->nsplit_t) * L * L;
  P->sign_bytes = sign_fix_scratch_bytes(n, (int)L);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  P->off_status = take(256);
  P->off_lam = take(w * m * L);
  P->off_y = take(w * n * L);
  P->off_q = take(w * n * L);
  P->off_z = take(w * round_up(m, 4) * L);
  P->off_zq = take(w * round_up(m, 4) * L);
  P->off_tt = take(w * m * L);
  P->off_part = take(w * P->part_elems);
  P->off_gpart = take(8 * P->gpart_elems);
  P->off_g = take(8 * L * L);
  P->off_x = take(8 * L * L);
  P->off_xw = take(w * L * L);
  P->off_xu = take(8 * L * L);
  P->off_eig = take(8 * sym_eig_work_doubles((int)L));
  P->off_sigma = take(8 * L);
  P->off_uhat = take(8 * L * L);
  P->off_sign = take(P->sign_bytes);
  P->off_xch = take(8 * 6 * L);
  P->n_ld = round_up(n, 64);
  P->m_ld = round_up(m, 64);
  P->off_sb = P->off_qb = P->off_zb = P->off_atf = P->off_wpart = 0;
  P->nsplit_w = 0;
  P->wpart_elems = 0;
  if (is16(compute)) {
    P->nsplit_w = std::max(tc_wpass_splits(n, m, compute), tc_wpass_splits(n, m, RPOD_F32));
    P->nsw_def = P->nsplit_w;
    // room for the project of up to 64 splits x 256 snapshots as well
    P->wpart_elems = std::max((size_t)P->nsplit_w * P->split_cap * L * m, (size_t)64 * L * 256);
    P->off_sb = take((size_t)2 * P->n_ld * m);
    P->off_qb = take((size_t)2 * P->n_ld * 128);
    P->off_zb = take((size_t)2 * P->m_ld * 128);
    P->off_atf = take((size_t)4 * P->n_ld * 128);
    P->off_wpart = take(4 * P->wpart_elems);
  }
  P->off_hs = P->off_hu = P->off_hsig = P->off_hc = 0;
  P->ld_hs = 0;
  if (flags & RPOD_FLAG_HOST_IO) {
    // S staged in the compute type (FP32 for the 16-bit forms, converted on
    // the first pass), 16-element-aligned columns so the tensor maps apply
    const size_t es = compute == RPOD_F64 ? 8 : 4;
    P->ld_hs = round_up(n, 16);
    P->off_hs = take(es * (size_t)P->ld_hs * m);
    P->off_hu = take(w * n * L);
    P->off_hsig = take(8 * L);
    P->off_hc = take(w * (size_t)k * m);
  }
  P->total = off;
  P->side = nullptr;
  if (is16(compute)) {
    // made here (not during a call, which may be inside a stream capture);
    // without a device the fork is skipped
    cudaStream_t ss = nullptr;
    if (cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) == cudaSuccess) {
      if (cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
          cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) == cudaSuccess)
        P->side = ss;
      else
        cudaStreamDestroy(ss);
    }
    cudaGetLastError();
  }
  P->last_launches = 0;
  P->svd_sweeps = 30;
  P->pass_stages = 0;
  P->graph_on = 1;
  *out = P;
  return RPOD_OK;
}

int rpod_plan_create(rpod_plan** out, int64_t n, int64_t m, int32_t k, int32_t p, int32_t q,
                     uint64_t seed, int32_t compute, uint32_t flags) {
  return plan_create_impl(out, n, m, k, p, q, seed, compute, flags, 1);
}

int rpod_rows_plan_create(rpod_plan** out, int64_t n_total, int64_t row0, int64_t n_rows, int64_t m,
                          int32_t k, int32_t p, int32_t q, uint64_t seed, int32_t compute,
                          uint32_t flags) {
  if (!out) return RPOD_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_rows < 1 || row0 < 0 || n_total < 1 || row0 + n_rows > n_total) return RPOD_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)RPOD_FLAG_RETURN_ALL_L) return RPOD_ERR_UNSUPPORTED;
  if (compute != RPOD_F64) return (compute >= RPOD_F64 && compute <= RPOD_F16) ? RPOD_ERR_UNSUPPORTED
                                                                              : RPOD_ERR_INVALID_ARG;
  rpod_plan* P = nullptr;
  const int rc = plan_create_impl(&P, n_rows, m, k, p, q, seed, compute, flags, 1, n_total);
  if (rc != RPOD_OK) return rc;
  P->rows_mode = 1;
  P->n_total = n_total;
  P->row0 = row0;
  *out = P;
  return RPOD_OK;
}

static void drop_plan_graph(rpod_plan* P) {
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  P->gexec = nullptr;
  P->graph_calls = 0;
}

int rpod_plan_set_svd_sweeps(rpod_plan* P, int32_t max_sweeps) {
  if (!P || max_sweeps < 1 || max_sweeps > 1000) return RPOD_ERR_INVALID_ARG;
  if (P->compute != RPOD_F64) return RPOD_ERR_UNSUPPORTED;
  P->svd_sweeps = max_sweeps;
  drop_plan_graph(P);
  return RPOD_OK;
}

int rpod_plan_set_graph(rpod_plan* P, int32_t enable) {
  if (!P || (enable != 0 && enable != 1)) return RPOD_ERR_INVALID_ARG;
  P->graph_on = enable;
  drop_plan_graph(P);
  return RPOD_OK;
}

int rpod_workspace_bytes(const rpod_plan* P, size_t* bytes) {
  if (!P || !bytes) return RPOD_ERR_INVALID_ARG;
  *bytes = P->total;
  return RPOD_OK;
}

int rpod_profile_enable(rpod_plan* P, int enable);

void rpod_plan_destroy(rpod_plan* P) {
  if (P && P->prof_on) rpod_profile_enable(P, 0);
  if (P) drop_plan_graph(P);
  if (P && P->gcap) cudaStreamDestroy(P->gcap);
  if (P && P->side) {
    cudaEventDestroy(P->ev_fork);
    cudaEventDestroy(P->ev_join);
    cudaStreamDestroy(P->side);
  }
  delete P;
}

int rpod_last_launch_count(const rpod_plan* P) { return P ? P->last_launches : -1; }

static int check_ws(const rpod_plan* P, void* ws, size_t bytes) {
  if (!ws || bytes < P->total || ((uintptr_t)ws & 255)) return RPOD_ERR_WORKSPACE;
  return RPOD_OK;
}

static int basis_device(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype,
                        const float* S_refine, int64_t ldr, void* U, int64_t ldu, double* sigma,
                        void* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                        void* stream);

int rpod_basis_rows(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype, void* U, int64_t ldu,
                    double* sigma, void* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                    void* stream, rpod_exchange_fn exchange, void* ctx) {
  rpod::NvtxRange nv("rpod_basis_rows");
  if (!P || !P->rows_mode || !S || !U || !sigma || !C || !exchange) return RPOD_ERR_INVALID_ARG;
  if (s_dtype != P->compute) return RPOD_ERR_INVALID_ARG;
  P->xch = exchange;
  P->xch_ctx = ctx;
  const int rc = basis_device(P, S, lds, s_dtype, nullptr, 0, U, ldu, sigma, C, ldc, workspace,
                              workspace_bytes, stream);
  P->xch = nullptr;
  P->xch_ctx = nullptr;
  return rc;
}

int rpod_basis(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype, const float* S_refine,
               int64_t ldr, void* U, int64_t ldu, double* sigma, void* C, int64_t ldc,
               void* workspace, size_t workspace_bytes, void* stream) {
  rpod::NvtxRange nv("rpod_basis");
  if (!P || !S || !U || !sigma || !C) return RPOD_ERR_INVALID_ARG;
  if (P->rows_mode) return RPOD_ERR_INVALID_ARG;  // needs the exchange: rpod_basis_rows
  if (!(P->flags & RPOD_FLAG_HOST_IO))
    return basis_device(P, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, workspace,
                        workspace_bytes, stream);
  // host buffers: S in (the compute type, or FP32 for the 16-bit forms),
  // U, sigma, C out, through the workspace's staging copies
  const int c = P->compute;
  const int want = (c == RPOD_F64) ? RPOD_F64 : RPOD_F32;
  if (s_dtype != want || S_refine) return RPOD_ERR_UNSUPPORTED;
  if (lds < P->n || ldc < P->k || ldu < P->n) return RPOD_ERR_INVALID_ARG;
  if (int rc = check_ws(P, workspace, workspace_bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const size_t es = c == RPOD_F64 ? 8 : 4;
  const int ku = (P->flags & RPOD_FLAG_RETURN_ALL_L) ? P->l : P->k;
  if (cudaMemcpy2DAsync(ws + P->off_hs, P->ld_hs * es, S, lds * es, P->n * es, P->m,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  const int rc = basis_device(P, ws + P->off_hs, P->ld_hs, s_dtype, nullptr, 0, ws + P->off_hu,
                              P->n, (double*)(ws + P->off_hsig), ws + P->off_hc, P->k, workspace,
                              workspace_bytes, stream);
  if (rc) return rc;
  if (cudaMemcpy2DAsync(U, ldu * es, ws + P->off_hu, P->n * es, P->n * es, ku,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(sigma, ws + P->off_hsig, 8 * (size_t)P->l, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpy2DAsync(C, ldc * es, ws + P->off_hc, P->k * es, P->k * es, P->m,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  return RPOD_OK;
}

static int basis_direct(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype,
                        const float* S_refine, int64_t ldr, void* U, int64_t ldu, double* sigma,
                        void* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                        void* stream);

// A repeated basis call with unchanged buffers replays one CUDA graph of its
// launches (no host work per kernel, no launch gaps).  Direct launches for:
// the first call with a set of buffers, row-sharded plans (their exchange
// callback runs on the host between kernels), profiled plans (their events
// time each pass), and a caller's stream that is itself being captured.
static int basis_device(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype,
                        const float* S_refine, int64_t ldr, void* U, int64_t ldu, double* sigma,
                        void* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                        void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!P->graph_on || P->rows_mode || P->prof_on || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return basis_direct(P, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, workspace,
                        workspace_bytes, stream);
  }
  const uintptr_t key[12] = {(uintptr_t)S, (uintptr_t)lds, (uintptr_t)s_dtype, (uintptr_t)S_refine,
                             (uintptr_t)ldr, (uintptr_t)U, (uintptr_t)ldu, (uintptr_t)sigma,
                             (uintptr_t)C, (uintptr_t)ldc, (uintptr_t)workspace,
                             (uintptr_t)workspace_bytes};
  const bool same = P->graph_calls > 0 && std::equal(key, key + 12, P->gkey);
  if (same && P->gexec) {
    if (cudaGraphLaunch(P->gexec, st) != cudaSuccess) return RPOD_ERR_CUDA;
    P->last_launches = P->graph_launches;
    return RPOD_OK;
  }
  if (!same) {
    drop_plan_graph(P);
    std::copy(key, key + 12, P->gkey);
    P->graph_calls = 1;
    return basis_direct(P, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, workspace,
                        workspace_bytes, stream);
  }
  // second call with these buffers: capture on the plan's own stream (the
  // caller's may be the legacy default stream, which cannot capture)
  if (!P->gcap && cudaStreamCreateWithFlags(&P->gcap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    P->gcap = nullptr;
    P->graph_on = 0;
    return basis_direct(P, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, workspace,
                        workspace_bytes, stream);
  }
  int rc = RPOD_ERR_CUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(P->gcap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    rc = basis_direct(P, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, workspace,
                      workspace_bytes, P->gcap);
    const cudaError_t ec = cudaStreamEndCapture(P->gcap, &g);
    if (rc == RPOD_OK && ec != cudaSuccess) rc = RPOD_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (rc == RPOD_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    ex = nullptr;
    rc = RPOD_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  if (rc == RPOD_OK) {
    P->gexec = ex;
    P->graph_launches = P->last_launches;
    if (cudaGraphLaunch(P->gexec, st) != cudaSuccess) return RPOD_ERR_CUDA;
    return RPOD_OK;
  }
  cudaGetLastError();  // leave no capture error behind
  if (rc != RPOD_ERR_CUDA) return rc;  // an argument error: the same as a direct call
  // the launch sequence could not be captured: direct launches from now on
  P->graph_on = 0;
  return basis_direct(P, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, workspace,
                      workspace_bytes, stream);
}

static int basis_direct(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype,
                        const float* S_refine, int64_t ldr, void* U, int64_t ldu, double* sigma,
                        void* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                        void* stream) {
  if (lds < P->n || ldc < P->k || ldu < P->n) return RPOD_ERR_INVALID_ARG;
  if (int rc = check_ws(P, workspace, workspace_bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int c = P->compute;
  g_launches = 0;
  if ((c == RPOD_F64 || c == RPOD_F32) ? (s_dtype != c) : !(s_dtype == c || s_dtype == RPOD_F32))
    return RPOD_ERR_INVALID_ARG;
  if (is16(c) && (P->flags & RPOD_FLAG_REFINE_FP32) && s_dtype != RPOD_F32 &&
      (!S_refine || ldr < P->n))
    return RPOD_ERR_INVALID_ARG;
  // a basis call starts from a clear status block (status word, FP64 gate)
  if (cudaMemsetAsync(ws + P->off_status, 0, 256, st) != cudaSuccess) return RPOD_ERR_CUDA;
  int rc;
  if (c == RPOD_F64 || c == RPOD_F32) {
    if (s_dtype != c) return RPOD_ERR_INVALID_ARG;
    if (c == RPOD_F64) {
      Run<double> R{P, ws, st, (unsigned*)(ws + P->off_status)};
      rc = R.run((const double*)S, lds, (double*)U, ldu, sigma, (double*)C, ldc);
    } else {
      Run<float> R{P, ws, st, (unsigned*)(ws + P->off_status)};
      rc = R.run((const float*)S, lds, (float*)U, ldu, sigma, (float*)C, ldc);
    }
  } else {
    // 16-bit tensor-core forms
    if (!(s_dtype == c || s_dtype == RPOD_F32)) return RPOD_ERR_INVALID_ARG;
    const bool want_ref = (P->flags & RPOD_FLAG_REFINE_FP32) && s_dtype != RPOD_F32;
    if (want_ref && (!S_refine || ldr < P->n)) return RPOD_ERR_INVALID_ARG;
    Run<float> R{P, ws, st, (unsigned*)(ws + P->off_status)};
    rc = R.run_tc(S, lds, s_dtype, want_ref ? S_refine : nullptr, ldr, (float*)U, ldu, sigma,
                  (float*)C, ldc);
  }
  P->last_launches = g_launches;
  return rc;
}

int rpod_project(const rpod_plan* P, const void* U, int64_t ldu, int32_t kc, const void* S_new,
                 int64_t lds, int64_t m_new, int32_t s_dtype, void* C, int64_t ldc, void* workspace,
                 size_t workspace_bytes, void* stream) {
  rpod::NvtxRange nv("rpod_project");
  if (!P || !U || !S_new || !C || kc < 1 || kc > P->l || m_new < 1) return RPOD_ERR_INVALID_ARG;
  if (P->rows_mode || ldu < P->n || lds < P->n || ldc < kc) return RPOD_ERR_INVALID_ARG;
  if (int rc = check_ws(P, workspace, workspace_bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  rpod_plan* Pm = const_cast<rpod_plan*>(P);
  g_launches = 0;
  int rc = RPOD_ERR_INVALID_ARG;
  if (P->compute == RPOD_F64) {
    if (s_dtype != RPOD_F64) return RPOD_ERR_INVALID_ARG;
    Run<double> R{Pm, ws, st, (unsigned*)(ws + P->off_status)};
    rc = R.project((const double*)U, ldu, kc, (const double*)S_new, lds, m_new, (double*)C, ldc);
  } else if (s_dtype == RPOD_F32) {
    Run<float> R{Pm, ws, st, (unsigned*)(ws + P->off_status)};
    rc = R.project((const float*)U, ldu, kc, (const float*)S_new, lds, m_new, (float*)C, ldc);
  } else if (is16(P->compute) && s_dtype == P->compute) {
    Run<float> R{Pm, ws, st, (unsigned*)(ws + P->off_status)};
    rc = R.project_tc((const float*)U, ldu, kc, S_new, lds, m_new, (float*)C, ldc);
  } else {
    return RPOD_ERR_INVALID_ARG;
  }
  Pm->last_launches = g_launches;
  return rc;
}

int rpod_sketch(const rpod_plan* P, void* Lam, int64_t ld, int32_t dtype, void* stream) {
  if (!P || !Lam || ld < P->m) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (dtype) {
    case RPOD_F64: e = sketch<double>(st, P->seed, 0, P->m, P->l, (double*)Lam, ld); break;
    case RPOD_F32: e = sketch<float>(st, P->seed, 0, P->m, P->l, (float*)Lam, ld); break;
    case RPOD_BF16: e = sketch<__nv_bfloat16>(st, P->seed, 0, P->m, P->l, (__nv_bfloat16*)Lam, ld); break;
    case RPOD_F16: e = sketch<__half>(st, P->seed, 0, P->m, P->l, (__half*)Lam, ld); break;
    default: return RPOD_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}

int rpod_sample(const rpod_plan* P, const void* A, int64_t lda, const void* S, int64_t lds,
                int32_t s_dtype, float* Y, int64_t ldy, void* workspace, size_t workspace_bytes,
                void* stream) {
  if (!P || !A || !S || !Y || lda < P->m || lds < P->n || ldy < P->n) return RPOD_ERR_INVALID_ARG;
  if (!is16(P->compute) || s_dtype != P->compute) return RPOD_ERR_INVALID_ARG;
  if (int rc = check_ws(P, workspace, workspace_bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  void* Zh = ws + P->off_zb;
  if (cudaMemcpy2DAsync(Zh, (size_t)P->m_ld * 2, A, (size_t)lda * 2, (size_t)P->m * 2, (size_t)P->l,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  g_launches = 0;
  const int rc = tc_ypass(st, P->compute, Zh, P->m_ld, S, lds, P->n, P->m, P->l, Y, ldy,
                          (unsigned*)(ws + P->off_status));
  const_cast<rpod_plan*>(P)->last_launches = g_launches;
  return rc;
}

int rpod_profile_enable(rpod_plan* P, int enable) {
  if (!P) return RPOD_ERR_INVALID_ARG;
  if (enable && !P->prof_on) {
    P->prof_ev = new (std::nothrow) cudaEvent_t[2 * kProfPasses];
    if (!P->prof_ev) return RPOD_ERR_INVALID_ARG;
    for (int i = 0; i < 2 * kProfPasses; ++i)
      if (cudaEventCreate(&P->prof_ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(P->prof_ev[j]);
        delete[] P->prof_ev;
        P->prof_ev = nullptr;
        return RPOD_ERR_CUDA;
      }
    P->prof_on = 1;
  } else if (!enable && P->prof_on) {
    for (int i = 0; i < 2 * kProfPasses; ++i) cudaEventDestroy(P->prof_ev[i]);
    delete[] P->prof_ev;
    P->prof_ev = nullptr;
    P->prof_on = 0;
  }
  P->prof_n = 0;
  P->prof_bytes = 0.0;
  P->prof_flops = 0.0;
  return RPOD_OK;
}

int rpod_profile_read(const rpod_plan* P, int* passes, double* pass_ms, double* bytes, double* flops) {
  if (!P || !passes || !pass_ms || !bytes || !flops) return RPOD_ERR_INVALID_ARG;
  *passes = P->prof_n;
  *pass_ms = 0.0;
  *bytes = P->prof_bytes;
  *flops = P->prof_flops;
  if (!P->prof_on || P->prof_n == 0) return RPOD_OK;
  if (cudaEventSynchronize(P->prof_ev[2 * P->prof_n - 1]) != cudaSuccess) return RPOD_ERR_CUDA;
  for (int i = 0; i < P->prof_n; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P->prof_ev[2 * i], P->prof_ev[2 * i + 1]) != cudaSuccess)
      return RPOD_ERR_CUDA;
    *pass_ms += ms;
  }
  return RPOD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched rPOD: per-instance pipelines on worker streams, captured into one
// CUDA graph.
struct rpod_batch {
  int count = 0;
  int compute = 0;
  uint32_t flags = 0;
  int s_dtype = 0;
  std::vector<rpod_plan*> plans;
  std::vector<rpod_instance> inst;
  std::vector<size_t> ws_off;
  size_t total = 0;
  int nstreams = 4;
  int split_pct = 100;
  int stages = 0;  // pipeline depth of the instances' passes (0: by pass size)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // capture origin (the legacy default stream cannot capture)
  cudaGraphExec_t exec = nullptr;
  void* graph_ws = nullptr;
  int last_launches = 0;
};

namespace {

void apply_split(rpod_plan* P, int pct) {
  auto scale = [&](int def) {
    if (def <= 0) return def;
    int s = (int)((int64_t)def * pct / 100);
    if (s < 1) s = 1;
    if (s > def * P->split_cap) s = def * P->split_cap;
    return s;
  };
  P->nsplit_z = scale(P->nsz_def);
  if (P->nsw_def > 0) P->nsplit_w = scale(P->nsw_def);
}

void drop_graph(rpod_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  B->exec = nullptr;
  B->graph_ws = nullptr;
}

constexpr int kMaxBatchStreams = 64;

int ensure_streams(rpod_batch* B) {
  while ((int)B->streams.size() < kMaxBatchStreams) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RPOD_ERR_CUDA;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return RPOD_ERR_CUDA;
    B->streams.push_back(s);
    B->join.push_back(e);
  }
  if (!B->fork && cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess)
    return RPOD_ERR_CUDA;
  if (!B->cap && cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess)
    return RPOD_ERR_CUDA;
  return RPOD_OK;
}

// Captures every instance's pipeline into B->exec, starting from the batch's
// own stream; the graph is then launched on the caller's stream.
int capture(rpod_batch* B, char* ws) {
  CR(ensure_streams(B));
  prepare_kernels();
  drop_graph(B);
  cudaStream_t stream = B->cap;
  const int ns = std::max(1, std::min(B->nstreams, std::min(kMaxBatchStreams, B->count)));
  // Longest-processing-time assignment of instances to worker streams: the
  // costliest instances first, each to the stream with the least work so
  // far.  Cost = pass bytes (2q + 2 passes over n x m) plus a fixed share for
  // the latency-bound small-matrix steps, which scale with l.
  std::vector<int> order(B->count), where(B->count);
  std::vector<double> cost(B->count), load(ns, 0.0);
  for (int i = 0; i < B->count; ++i) {
    const rpod_instance& I = B->inst[i];
    const double l = (double)(I.k + I.p);
    cost[i] = (2.0 * I.q + 2.0) * (double)I.n * (double)I.m + 4.0e6 * l;
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (int i : order) {
    int best = 0;
    for (int s2 = 1; s2 < ns; ++s2)
      if (load[s2] < load[best]) best = s2;
    where[i] = best;
    load[best] += cost[i];
  }
  if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return RPOD_ERR_CUDA;
  int rc = RPOD_OK;
  int launches = 0;
  if (cudaEventRecord(B->fork, stream) != cudaSuccess) rc = RPOD_ERR_CUDA;
  for (int s = 0; s < ns && rc == RPOD_OK; ++s)
    if (cudaStreamWaitEvent(B->streams[s], B->fork, 0) != cudaSuccess) rc = RPOD_ERR_CUDA;
  for (int oi = 0; oi < B->count && rc == RPOD_OK; ++oi) {
    const int i = order[oi];
    const rpod_instance& I = B->inst[i];
    rc = rpod_basis(B->plans[i], I.S, I.lds, B->s_dtype, I.S_refine, I.ldr, I.U, I.ldu, I.sigma,
                    I.C, I.ldc, ws + B->ws_off[i], B->plans[i]->total, B->streams[where[i]]);
    launches += B->plans[i]->last_launches;
  }
  for (int s = 0; s < ns && rc == RPOD_OK; ++s) {
    if (cudaEventRecord(B->join[s], B->streams[s]) != cudaSuccess ||
        cudaStreamWaitEvent(stream, B->join[s], 0) != cudaSuccess)
      rc = RPOD_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(stream, &g);
  if (rc == RPOD_OK && ec != cudaSuccess) rc = RPOD_ERR_CUDA;
  if (rc != RPOD_OK) cudaGetLastError();  // do not leave a capture error behind
  if (rc == RPOD_OK && cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) {
    B->exec = nullptr;
    rc = RPOD_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  if (rc == RPOD_OK) {
    B->graph_ws = ws;
    B->last_launches = launches;
  }
  return rc;
}

}  // namespace

extern "C" {

int rpod_batch_create(rpod_batch** out, int32_t count, const rpod_instance* inst, int32_t compute,
                      uint32_t flags, int32_t s_dtype) {
  if (!out || count < 1 || !inst) return RPOD_ERR_INVALID_ARG;
  *out = nullptr;
  // batch instances live in device memory (one graph over all of them)
  if (flags & RPOD_FLAG_HOST_IO) return RPOD_ERR_UNSUPPORTED;
  if ((compute == RPOD_F64 || compute == RPOD_F32) ? (s_dtype != compute)
                                                   : !(s_dtype == compute || s_dtype == RPOD_F32))
    return RPOD_ERR_INVALID_ARG;
  rpod_batch* B = new (std::nothrow) rpod_batch();
  if (!B) return RPOD_ERR_INVALID_ARG;
  B->count = count;
  B->compute = compute;
  B->flags = flags;
  B->s_dtype = s_dtype;
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    const rpod_instance& I = inst[i];
    rpod_plan* P = nullptr;
    const int rc = plan_create_impl(&P, I.n, I.m, I.k, I.p, I.q, I.seed, compute, flags, 2);
    if (rc != RPOD_OK || !I.S || !I.U || !I.sigma || !I.C || I.lds < I.n || I.ldu < I.n ||
        I.ldc < I.k) {
      if (P) rpod_plan_destroy(P);
      rpod_batch_destroy(B);
      return rc != RPOD_OK ? rc : RPOD_ERR_INVALID_ARG;
    }
    B->plans.push_back(P);
    B->inst.push_back(I);
    B->ws_off.push_back(off);
    off = align256(off + P->total);
  }
  B->total = off;
  *out = B;
  return RPOD_OK;
}

int rpod_batch_workspace_bytes(const rpod_batch* B, size_t* bytes) {
  if (!B || !bytes) return RPOD_ERR_INVALID_ARG;
  *bytes = B->total;
  return RPOD_OK;
}

int rpod_batch_configure(rpod_batch* B, int32_t streams, int32_t split_pct) {
  if (!B || streams < 1 || streams > kMaxBatchStreams || split_pct < 10 || split_pct > 200)
    return RPOD_ERR_INVALID_ARG;
  B->nstreams = streams;
  B->split_pct = split_pct;
  for (rpod_plan* P : B->plans) apply_split(P, split_pct);
  drop_graph(B);
  return RPOD_OK;
}

int rpod_batch_set_pass_stages(rpod_batch* B, int32_t stages) {
  if (!B || !(stages == 0 || stages == 2 || stages == 4)) return RPOD_ERR_INVALID_ARG;
  B->stages = stages;
  for (rpod_plan* P : B->plans) P->pass_stages = stages;
  drop_graph(B);
  return RPOD_OK;
}

int rpod_batch_run(rpod_batch* B, void* workspace, size_t workspace_bytes, void* stream) {
  rpod::NvtxRange nv("rpod_batch_run");
  if (!B) return RPOD_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < B->total || ((uintptr_t)workspace & 255))
    return RPOD_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  if (!B->exec || B->graph_ws != workspace) CR(capture(B, (char*)workspace));
  if (cudaGraphLaunch(B->exec, st) != cudaSuccess) return RPOD_ERR_CUDA;
  return RPOD_OK;
}

int rpod_batch_tune(rpod_batch* B, void* workspace, size_t workspace_bytes, void* stream,
                    int32_t trials, int32_t* best_streams, int32_t* best_split_pct,
                    int32_t* best_stages) {
  rpod::NvtxRange nv("rpod_batch_tune");
  if (!B || trials < 1) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int stream_opts[7] = {1, 2, 4, 8, 16, 32, 64};
  const int split_opts[4] = {25, 50, 100, 200};
  // the passes' pipeline depth matters only for the tensor-core forms
  const bool tc16 = B->compute == RPOD_BF16 || B->compute == RPOD_F16;
  const int stage_opts[2] = {2, 4};
  const int nstage = tc16 ? 2 : 1;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RPOD_ERR_CUDA;
  float best = 1e30f;
  int bs = B->nstreams, bp = B->split_pct, bg = B->stages;
  int rc = RPOD_OK;
  for (int g = 0; g < nstage && rc == RPOD_OK; ++g) {
    if (tc16) rc = rpod_batch_set_pass_stages(B, stage_opts[g]);
    for (int a = 0; a < 7 && rc == RPOD_OK; ++a) {
      if (stream_opts[a] > std::max(1, B->count)) continue;
      for (int b = 0; b < 4 && rc == RPOD_OK; ++b) {
        rc = rpod_batch_configure(B, stream_opts[a], split_opts[b]);
        if (rc == RPOD_OK) rc = rpod_batch_run(B, workspace, workspace_bytes, stream);  // capture + warm
        if (rc != RPOD_OK) break;
        // `trials` separately timed replays; the point's time is their minimum
        float pt = 1e30f;
        for (int t = 0; t < trials && rc == RPOD_OK; ++t) {
          cudaEventRecord(e0, st);
          rc = rpod_batch_run(B, workspace, workspace_bytes, stream);
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = RPOD_ERR_CUDA;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          pt = std::min(pt, ms);
        }
        if (rc == RPOD_OK && pt < best) {
          best = pt;
          bs = stream_opts[a];
          bp = split_opts[b];
          bg = tc16 ? stage_opts[g] : B->stages;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RPOD_OK) return rc;
  CR(rpod_batch_set_pass_stages(B, bg));
  CR(rpod_batch_configure(B, bs, bp));
  if (best_streams) *best_streams = bs;
  if (best_split_pct) *best_split_pct = bp;
  if (best_stages) *best_stages = bg;
  return RPOD_OK;
}

int rpod_batch_status_sync(const rpod_batch* B, void* workspace, void* stream, int32_t* first_bad,
                           uint32_t* flags_out) {
  if (!B || !workspace) return RPOD_ERR_INVALID_ARG;
  int first = RPOD_OK;
  int bad = -1;
  uint32_t fl = 0;
  for (int i = 0; i < B->count; ++i) {
    uint32_t f = 0;
    const int rc = rpod_status_sync(B->plans[i], (char*)workspace + B->ws_off[i], stream, &f);
    fl |= f;
    if (rc != RPOD_OK && first == RPOD_OK) { first = rc; bad = i; }
  }
  if (first_bad) *first_bad = bad;
  if (flags_out) *flags_out = fl;
  return first;
}

int rpod_batch_last_launch_count(const rpod_batch* B) { return B ? B->last_launches : -1; }

void rpod_batch_destroy(rpod_batch* B) {
  if (!B) return;
  drop_graph(B);
  for (rpod_plan* P : B->plans) rpod_plan_destroy(P);
  for (cudaStream_t s : B->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->join) cudaEventDestroy(e);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
}

int rpod_status_sync(const rpod_plan* P, void* workspace, void* stream, uint32_t* flags_out) {
  if (!P || !workspace) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  unsigned* d = (unsigned*)((char*)workspace + P->off_status);
  if (cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return RPOD_ERR_CUDA;
  if (cudaMemsetAsync(d, 0, sizeof(unsigned), st) != cudaSuccess) return RPOD_ERR_CUDA;
  if (flags_out) *flags_out = (h & ST_RANK_DEF) ? RPOD_WARN_RANK_DEFICIENT : 0u;
  if (h & ST_NONFINITE) return RPOD_ERR_NONFINITE;
  if (h & ST_TIMEOUT) return RPOD_ERR_TIMEOUT;
  if (h & ST_BREAKDOWN) return RPOD_ERR_BREAKDOWN;
  if (h & ST_NO_CONV) return RPOD_ERR_NO_CONVERGENCE;
  return RPOD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Basis files: "RPODBASE", version 1, the plan's parameters, then U (n x ku),
// sigma (l) and C (k x m), column-major and packed.
namespace {
constexpr char kBasisMagic[8] = {'R', 'P', 'O', 'D', 'B', 'A', 'S', 'E'};
constexpr uint32_t kBasisVersion = 1;
struct BasisHeader {
  char magic[8];
  uint32_t version;
  int32_t compute;
  uint32_t flags;
  int32_t k, p, q, ku, elem;
  int64_t n, m;
  uint64_t seed;
};

int read_basis_header(FILE* f, BasisHeader* h) {
  if (fread(h, sizeof(*h), 1, f) != 1 || memcmp(h->magic, kBasisMagic, 8) != 0 ||
      h->version != kBasisVersion || h->n < 1 || h->m < 1 || h->k < 1 || h->p < 0 || h->q < 0 ||
      h->ku < h->k || h->ku > h->k + h->p || (h->elem != 4 && h->elem != 8))
    return RPOD_ERR_IO;
  return RPOD_OK;
}
}  // namespace

extern "C" {

int rpod_basis_save(const rpod_plan* P, const char* path, const void* U, int64_t ldu,
                    const double* sigma, const void* C, int64_t ldc, void* stream) {
  if (!P || !path || !U || !sigma || !C) return RPOD_ERR_INVALID_ARG;
  const int ku = (P->flags & RPOD_FLAG_RETURN_ALL_L) ? P->l : P->k;
  const size_t es = P->compute == RPOD_F64 ? 8 : 4;
  if (ldu < P->n || ldc < P->k) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<char> u, c;
  std::vector<double> s;
  try {
    u.resize((size_t)P->n * ku * es);
    c.resize((size_t)P->k * P->m * es);
    s.resize(P->l);
  } catch (...) {
    return RPOD_ERR_INVALID_ARG;
  }
  if (cudaMemcpy2DAsync(u.data(), P->n * es, U, ldu * es, P->n * es, ku, cudaMemcpyDefault, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(s.data(), sigma, 8 * (size_t)P->l, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaMemcpy2DAsync(c.data(), P->k * es, C, ldc * es, P->k * es, P->m, cudaMemcpyDefault, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  BasisHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kBasisMagic, 8);
  h.version = kBasisVersion;
  h.compute = P->compute;
  h.flags = P->flags;
  h.k = P->k;
  h.p = P->p;
  h.q = P->q;
  h.ku = ku;
  h.elem = (int32_t)es;
  h.n = P->n;
  h.m = P->m;
  h.seed = P->seed;
  FILE* f = fopen(path, "wb");
  if (!f) return RPOD_ERR_IO;
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(u.data(), 1, u.size(), f) == u.size() &&
            fwrite(s.data(), sizeof(double), s.size(), f) == s.size() &&
            fwrite(c.data(), 1, c.size(), f) == c.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? RPOD_OK : RPOD_ERR_IO;
}

int rpod_basis_file_info(const char* path, int64_t* info) {
  if (!path || !info) return RPOD_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return RPOD_ERR_IO;
  BasisHeader h;
  const int rc = read_basis_header(f, &h);
  fclose(f);
  if (rc) return rc;
  const int64_t v[9] = {h.n, h.m, h.k, h.p, h.q, (int64_t)h.seed, h.compute, (int64_t)h.flags, h.ku};
  memcpy(info, v, sizeof(v));
  return RPOD_OK;
}

int rpod_basis_load(const char* path, void* U, int64_t ldu, double* sigma, void* C, int64_t ldc,
                    void* stream) {
  if (!path || !U || !sigma || !C) return RPOD_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return RPOD_ERR_IO;
  BasisHeader h;
  if (int rc = read_basis_header(f, &h)) {
    fclose(f);
    return rc;
  }
  if (ldu < h.n || ldc < h.k) {
    fclose(f);
    return RPOD_ERR_INVALID_ARG;
  }
  const size_t es = (size_t)h.elem;
  const int l = h.k + h.p;
  std::vector<char> u, c;
  std::vector<double> s;
  try {
    u.resize((size_t)h.n * h.ku * es);
    c.resize((size_t)h.k * h.m * es);
    s.resize(l);
  } catch (...) {
    fclose(f);
    return RPOD_ERR_INVALID_ARG;
  }
  const bool ok = fread(u.data(), 1, u.size(), f) == u.size() &&
                  fread(s.data(), sizeof(double), s.size(), f) == s.size() &&
                  fread(c.data(), 1, c.size(), f) == c.size();
  fclose(f);
  if (!ok) return RPOD_ERR_IO;
  cudaStream_t st = (cudaStream_t)stream;
  // the host buffers live until the copies are done
  if (cudaMemcpy2DAsync(U, ldu * es, u.data(), h.n * es, h.n * es, h.ku, cudaMemcpyDefault, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(sigma, s.data(), 8 * (size_t)l, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaMemcpy2DAsync(C, ldc * es, c.data(), h.k * es, h.k * es, h.m, cudaMemcpyDefault, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  return RPOD_OK;
}

}  // extern "C"
