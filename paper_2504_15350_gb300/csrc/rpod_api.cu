// C ABI of librpod (declared in include/rpod.h): plans, workspace layout and
// the host-side orchestration of Alg. 1 (Sec. 4.2) on one CUDA stream.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

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
      off_x, off_xw, off_eig, off_sigma, off_uhat, off_sign, off_lowp, total;
  int nsplit_z, nsplit_g, nsplit_t;
  size_t part_elems, gpart_elems, sign_bytes;
  int last_launches;
  // pass profiling
  int prof_on;
  int prof_n;
  cudaEvent_t prof_ev[2 * 64];
  double prof_bytes, prof_flops;
};

namespace rpod {
// Pass profiling hooks used by the pipelines.
void prof_begin(rpod_plan* P, cudaStream_t st) {
  if (!P->prof_on || P->prof_n >= 64) return;
  cudaEventRecord(P->prof_ev[2 * P->prof_n], st);
}
void prof_end(rpod_plan* P, cudaStream_t st, double bytes, double flops) {
  if (!P->prof_on || P->prof_n >= 64) return;
  cudaEventRecord(P->prof_ev[2 * P->prof_n + 1], st);
  ++P->prof_n;
  P->prof_bytes += bytes;
  P->prof_flops += flops;
}
}  // namespace rpod

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int elem_size(int dt) {
  switch (dt) {
    case RPOD_F64: return 8;
    case RPOD_F32: return 4;
    case RPOD_BF16: case RPOD_F16: return 2;
    default: return 0;
  }
}

bool is16(int dt) { return dt == RPOD_BF16 || dt == RPOD_F16; }

int splits_for(int64_t K, int64_t chunk, int maxs) {
  int64_t s = (K + chunk - 1) / chunk;
  if (s < 1) s = 1;
  if (s > maxs) s = maxs;
  return (int)s;
}

#define CK(x)                                        \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return RPOD_ERR_CUDA;     \
  } while (0)

// ---------------------------------------------------------------------------
// SIMT pipeline on working type W (double for RPOD_F64, float for RPOD_F32).
template <typename W>
struct SimtRun {
  rpod_plan* P;
  char* ws;
  cudaStream_t st;
  unsigned* status;

  W* buf(size_t off) { return (W*)(ws + off); }
  double* dbuf(size_t off) { return (double*)(ws + off); }

  // Gram G = A^T A (A rows x l, ld = rows) in FP64 (products in W, summed in
  // W over chunks, then in FP64)
  int gram(const W* A, int64_t rows, int64_t lda, double* G, int nsplit) {
    const int l = P->l;
    CK((gemm<W, W, W, double>(st, true, l, l, rows, nsplit, A, lda, A, lda, dbuf(P->off_gpart), 1, l,
                              (int64_t)l * l, status, false)));
    CK((reduce_splits<double, double>(st, l, l, nsplit, dbuf(P->off_gpart), G, 1, l)));
    return 0;
  }

  // CholeskyQR with `rounds` passes: returns the buffer holding Q (in or tmp)
  int orth(W* in, W* tmp, int64_t rows, int rounds, W** out) {
    const int l = P->l;
    const double tol = sizeof(W) == 8 ? 1e-13 : 1e-5;
    const int64_t chunk = sizeof(W) == 8 ? 4096 : 1024;
    const int ns = splits_for(rows, chunk, 256);
    W* src = in;
    W* dst = tmp;
    for (int r = 0; r < rounds; ++r) {
      double* G = dbuf(P->off_g);
      if (int rc = gram(src, rows, rows, G, ns)) return rc;
      CK((cholesky<W>(st, l, G, tol, nullptr, dbuf(P->off_x), buf(P->off_xw), l, status)));
      CK((gemm<W, W, W, W>(st, false, rows, l, l, 1, src, rows, buf(P->off_xw), l, dst, 1, rows, 0,
                           status, false)));
      W* t = src; src = dst; dst = t;
    }
    *out = src;
    return 0;
  }

  int run(const W* S, int64_t lds, const W* Sref, int64_t ldr, W* U, int64_t ldu, double* sigma,
          W* C, int64_t ldc) {
    const int64_t n = P->n, m = P->m;
    const int l = P->l, k = P->k, q = P->q;
    W* Lam = buf(P->off_lam);
    W* Y = buf(P->off_y);
    W* Qb = buf(P->off_q);
    W* Z = buf(P->off_z);
    W* Zq = buf(P->off_zq);
    W* Tt = buf(P->off_tt);
    W* part = buf(P->off_part);
    // Alg. 1: Gaussian sketch
    CK((sketch<W>(st, P->seed, 0, m, l, Lam, m)));
    const double sw = sizeof(W);
    const double pass_bytes = sw * ((double)n * m + (double)n * l + (double)m * l);
    const double pass_flops = 2.0 * n * m * l;
    P->prof_n = 0; P->prof_bytes = 0; P->prof_flops = 0;
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
        W* Zo = nullptr;
        if (int rc = orth(Z, Zq, m, 1, &Zo)) return rc;
        prof_begin(P, st);
        CK((gemm<W, W, W, W>(st, false, n, l, m, 1, S, lds, Zo, m, Y, 1, n, 0, status, false)));
        prof_end(P, st, pass_bytes, pass_flops);
      }
      // Alg. 1 QR of the sampled matrix (CholeskyQR2 for the final basis)
      W* Qo = nullptr;
      if (int rc = orth(Y, Qb, n, it == q ? 2 : 1, &Qo)) return rc;
      Q = Qo;  // Y's buffer is free again once Z = S^T Q is formed
    }
    // Alg. 1: T = Q^T S, stored transposed (m x l)
    const W* ST = Sref ? Sref : S;
    const int64_t ldt = Sref ? ldr : lds;
    prof_begin(P, st);
    CK((gemm<W, W, W, W>(st, true, m, l, n, P->nsplit_z, ST, ldt, Q, n, part, 1, m, m * l, status,
                         false)));
    prof_end(P, st, pass_bytes, pass_flops);
    CK((reduce_splits<W, W>(st, m, l, P->nsplit_z, part, Tt, 1, m)));
    // Alg. 1: SVD of T via the eigenpairs of T T^T (FP64 Gram)
    double* GT = dbuf(P->off_g);
    {
      const int ns = P->nsplit_t;
      CK((gemm<W, W, W, double>(st, true, l, l, m, ns, Tt, m, Tt, m, dbuf(P->off_gpart), 1, l,
                                (int64_t)l * l, status, false)));
      CK((reduce_splits<double, double>(st, l, l, ns, dbuf(P->off_gpart), GT, 1, l)));
    }
    double* Uhat = dbuf(P->off_uhat);
    CK((sym_eig(st, l, GT, sigma, Uhat, dbuf(P->off_eig), status, 3)));
    // Alg. 1: lift U = Q Uhat (first k or all l columns), then the sign rule
    const int ku = (P->flags & RPOD_FLAG_RETURN_ALL_L) ? l : k;
    CK((gemm<W, double, W, W>(st, false, n, ku, l, 1, Q, n, Uhat, l, U, 1, ldu, 0, status, false)));
    CK((sign_fix<W>(st, n, ku, U, ldu, Uhat, l, ws + P->off_sign, P->sign_bytes)));
    // Sec. 4.3 coefficients C = U_k^T S = Uhat_k^T T (k x m)
    CK((gemm<W, double, W, W>(st, false, m, k, l, 1, Tt, m, Uhat, l, C, ldc, 1, 0, status, false)));
    return 0;
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
    return 0;
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
    default: return "unknown status";
  }
}

int rpod_plan_create(rpod_plan** out, int64_t n, int64_t m, int32_t k, int32_t p, int32_t q,
                     uint64_t seed, int32_t compute, uint32_t flags) {
  if (!out) return RPOD_ERR_INVALID_ARG;
  *out = nullptr;
  const int64_t l = (int64_t)k + p;
  if (n < 1 || m < 1 || k < 1 || p < 0 || q < 0 || l > n || l > m || l > kMaxL)
    return RPOD_ERR_INVALID_ARG;
  if (compute < RPOD_F64 || compute > RPOD_F16) return RPOD_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(RPOD_FLAG_REFINE_FP32 | RPOD_FLAG_RETURN_ALL_L)) return RPOD_ERR_INVALID_ARG;
  rpod_plan* P = new (std::nothrow) rpod_plan();
  if (!P) return RPOD_ERR_INVALID_ARG;
  P->n = n; P->m = m; P->k = k; P->p = p; P->q = q; P->l = (int)l;
  P->seed = seed; P->compute = compute; P->flags = flags;
  const size_t w = (compute == RPOD_F64) ? 8 : 4;
  const size_t L = (size_t)l;
  P->nsplit_z = splits_for(n, compute == RPOD_F64 ? 4096 : 8192, 64);
  P->nsplit_t = splits_for(m, 256, 512);
  const int nsg = 256;
  P->part_elems = std::max((size_t)P->nsplit_z * m * L, (size_t)1);
  P->gpart_elems = std::max((size_t)nsg, (size_t)P->nsplit_t) * L * L;
  P->sign_bytes = sign_fix_scratch_bytes(n, (int)L);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  P->off_status = take(256);
  P->off_lam = take(w * m * L);
  P->off_y = take(w * n * L);
  P->off_q = take(w * n * L);
  P->off_z = take(w * m * L);
  P->off_zq = take(w * m * L);
  P->off_tt = take(w * m * L);
  P->off_part = take(w * P->part_elems);
  P->off_gpart = take(8 * P->gpart_elems);
  P->off_g = take(8 * L * L);
  P->off_x = take(8 * L * L);
  P->off_xw = take(w * L * L);
  P->off_eig = take(8 * sym_eig_work_doubles((int)L));
  P->off_sigma = take(8 * L);
  P->off_uhat = take(8 * L * L);
  P->off_sign = take(P->sign_bytes);
  P->off_lowp = 0;
  if (is16(compute)) {
    if (int rc = tc_plan_extend(P->n, P->m, P->l, compute, &off, &P->off_lowp)) {
      delete P;
      return rc;
    }
  }
  P->total = off;
  P->last_launches = 0;
  *out = P;
  return RPOD_OK;
}

int rpod_workspace_bytes(const rpod_plan* P, size_t* bytes) {
  if (!P || !bytes) return RPOD_ERR_INVALID_ARG;
  *bytes = P->total;
  return RPOD_OK;
}

void rpod_plan_destroy(rpod_plan* P) {
  if (P && P->prof_on) rpod_profile_enable(P, 0);
  delete P;
}

int rpod_last_launch_count(const rpod_plan* P) { return P ? P->last_launches : -1; }

static int check_ws(const rpod_plan* P, void* ws, size_t bytes) {
  if (!ws || bytes < P->total || ((uintptr_t)ws & 255)) return RPOD_ERR_WORKSPACE;
  return RPOD_OK;
}

int rpod_basis(rpod_plan* P, const void* S, int64_t lds, int32_t s_dtype, const float* S_refine,
               int64_t ldr, void* U, int64_t ldu, double* sigma, void* C, int64_t ldc,
               void* workspace, size_t workspace_bytes, void* stream) {
  if (!P || !S || !U || !sigma || !C) return RPOD_ERR_INVALID_ARG;
  if (lds < P->n || ldc < P->k || ldu < P->n) return RPOD_ERR_INVALID_ARG;
  if (int rc = check_ws(P, workspace, workspace_bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int c = P->compute;
  g_launches = 0;
  if (c == RPOD_F64 || c == RPOD_F32) {
    if (s_dtype != c) return RPOD_ERR_INVALID_ARG;
    if (c == RPOD_F64) {
      SimtRun<double> R{P, ws, st, (unsigned*)(ws + P->off_status)};
      const int rc = R.run((const double*)S, lds, nullptr, 0, (double*)U, ldu, sigma, (double*)C, ldc);
      P->last_launches = g_launches;
      return rc;
    }
    SimtRun<float> R{P, ws, st, (unsigned*)(ws + P->off_status)};
    const int rc = R.run((const float*)S, lds, nullptr, 0, (float*)U, ldu, sigma, (float*)C, ldc);
    P->last_launches = g_launches;
    return rc;
  }
  // 16-bit tensor-core forms
  if (!(s_dtype == c || s_dtype == RPOD_F32)) return RPOD_ERR_INVALID_ARG;
  if ((P->flags & RPOD_FLAG_REFINE_FP32) && s_dtype != RPOD_F32 && (!S_refine || ldr < P->n))
    return RPOD_ERR_INVALID_ARG;
  TcArgs a;
  a.n = P->n; a.m = P->m; a.k = P->k; a.l = P->l; a.q = P->q; a.seed = P->seed;
  a.compute = c; a.flags = P->flags;
  a.S = S; a.lds = lds; a.s_dtype = s_dtype; a.Sref = S_refine; a.ldr = ldr;
  a.U = (float*)U; a.ldu = ldu; a.sigma = sigma; a.C = (float*)C; a.ldc = ldc;
  a.ws = ws; a.stream = st;
  a.off_status = P->off_status; a.off_lam = P->off_lam; a.off_y = P->off_y; a.off_q = P->off_q;
  a.off_z = P->off_z; a.off_zq = P->off_zq; a.off_tt = P->off_tt; a.off_part = P->off_part;
  a.off_gpart = P->off_gpart; a.off_g = P->off_g; a.off_x = P->off_x; a.off_xw = P->off_xw;
  a.off_eig = P->off_eig; a.off_uhat = P->off_uhat; a.off_sign = P->off_sign;
  a.off_lowp = P->off_lowp; a.sign_bytes = P->sign_bytes;
  a.nsplit_z = P->nsplit_z; a.nsplit_t = P->nsplit_t;
  const int rc = tc_basis(a);
  P->last_launches = g_launches;
  return rc;
}

int rpod_project(const rpod_plan* P, const void* U, int64_t ldu, int32_t kc, const void* S_new,
                 int64_t lds, int64_t m_new, int32_t s_dtype, void* C, int64_t ldc, void* workspace,
                 size_t workspace_bytes, void* stream) {
  if (!P || !U || !S_new || !C || kc < 1 || kc > P->l || m_new < 1) return RPOD_ERR_INVALID_ARG;
  if (ldu < P->n || lds < P->n || ldc < kc) return RPOD_ERR_INVALID_ARG;
  if (int rc = check_ws(P, workspace, workspace_bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  rpod_plan* Pm = const_cast<rpod_plan*>(P);
  g_launches = 0;
  if (P->compute == RPOD_F64) {
    if (s_dtype != RPOD_F64) return RPOD_ERR_INVALID_ARG;
    SimtRun<double> R{Pm, ws, st, (unsigned*)(ws + P->off_status)};
    const int rc = R.project((const double*)U, ldu, kc, (const double*)S_new, lds, m_new, (double*)C, ldc);
    Pm->last_launches = g_launches;
    return rc;
  }
  if (s_dtype == RPOD_F32) {
    SimtRun<float> R{Pm, ws, st, (unsigned*)(ws + P->off_status)};
    const int rc = R.project((const float*)U, ldu, kc, (const float*)S_new, lds, m_new, (float*)C, ldc);
    Pm->last_launches = g_launches;
    return rc;
  }
  if (is16(P->compute) && s_dtype == P->compute) {
    const int rc = tc_project(P->n, (const float*)U, ldu, kc, S_new, lds, m_new, s_dtype, (float*)C, ldc,
                              ws, P->off_part, P->part_elems, P->nsplit_z, P->off_status, st);
    Pm->last_launches = g_launches;
    return rc;
  }
  return RPOD_ERR_INVALID_ARG;
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

int rpod_profile_enable(rpod_plan* P, int enable) {
  if (!P) return RPOD_ERR_INVALID_ARG;
  if (enable && !P->prof_on) {
    for (int i = 0; i < 2 * 64; ++i)
      if (cudaEventCreate(&P->prof_ev[i]) != cudaSuccess) return RPOD_ERR_CUDA;
    P->prof_on = 1;
  } else if (!enable && P->prof_on) {
    for (int i = 0; i < 2 * 64; ++i) cudaEventDestroy(P->prof_ev[i]);
    P->prof_on = 0;
  }
  P->prof_n = 0;
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
