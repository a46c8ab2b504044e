// Starting eigenvectors of the small SVD (Alg. 1, SVD of T = Q^T S): the
// left singular vectors of T are the eigenvectors of its l x l Gram matrix
// G = T T^T, and the eigensolver refines a starting basis X in FP64
// (Ogita-Aishima passes, rpod_simt.cu).  This file computes that start in
// FP32 with one CTA:
//
//   1. G / max_i G_ii in FP32; Householder reduction to tridiagonal form
//      A = H T H^T (lower variant: column 0 first, so a matrix whose large
//      entries sit at the top left -- the Gram of a power-iterated basis --
//      keeps its small eigenvalues' relative accuracy).
//   2. Eigenvalues of the tridiagonal T by multisection on Sturm counts
//      (the number of negative pivots of the LDL^T factorization of T - x I
//      is the number of eigenvalues below x), 8 points per step and per
//      eigenvalue, stopped at a relative width of two ulps.
//   3. Eigenvectors of T from twisted factorizations (Dhillon and Parlett,
//      "Multiple representations to compute orthogonal eigenvectors of
//      symmetric tridiagonal matrices", Lin. Alg. Appl. 387, 2004): with the
//      forward pivots D+ and backward pivots D- of T - lambda I, the twist
//      index r minimising |gamma_r|, gamma_r = D+_r - e_r^2 / D-_{r+1},
//      gives the vector with x_r = 1 by two one-term recurrences; one
//      Rayleigh-quotient correction lambda += gamma_r / ||x||^2 and a second
//      factorization follow.
//   4. Vectors of eigenvalues closer than 1e-4 ||T|| are orthogonalised
//      against each other (modified Gram-Schmidt in ascending order); a
//      vector that loses more than half its norm there (a multiple
//      eigenvalue) is replaced by a pseudo-random vector orthogonalised
//      against all others.
//   5. Back-transformation X = H Z, column by column, each column held in
//      the registers of 8 threads.
//
// The FP64 refinement that follows squares the error of this start per
// pass; its accuracy, not this one's, sets the final result.
#include <float.h>
#include <math.h>

#include "rpod_internal.cuh"

namespace rpod {
namespace {

constexpr int kEigThreads = 1024;
constexpr int kGrp = 8;                    // threads per eigenvalue / per column
constexpr int kRowsPerThread = kMaxL / kGrp;

__host__ __device__ inline int eig_lda(int l) { return (l & 1) ? l : l + 1; }
// Smallest leading dimension >= l that is 4 mod 32: the back-transform's
// 8 rows x 4 columns per warp then fall in 32 distinct banks.
__host__ __device__ inline int eig_ldx(int l) { return ((l + 27) / 32) * 32 + 4; }

size_t eig_smem_bytes(int l) {
  return sizeof(float) * ((size_t)l * eig_lda(l) + 2 * (size_t)l * eig_ldx(l) + 8 * (size_t)kMaxL);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
  return x;
}

__global__ void __launch_bounds__(kEigThreads)
k_tridiag_eig32(int l, const double* __restrict__ G, double* __restrict__ Xout,
                unsigned* __restrict__ status) {
  extern __shared__ float4 sm4[];
  float* const A = reinterpret_cast<float*>(sm4);
  const int lda = eig_lda(l), ldx = eig_ldx(l);
  float* const Xs = A + (size_t)l * lda;   // eigenvectors of T, row r at r*ldx
  float* const Ws = Xs + (size_t)l * ldx;  // per-eigenvalue forward pivots
  float* const vs = Ws + (size_t)l * ldx;  // Householder vector, double-buffered
  float* const ps = vs + 2 * kMaxL;
  float* const dd = ps + kMaxL;            // diagonal of T
  float* const ee = dd + kMaxL;            // off-diagonal of T
  float* const e2 = ee + kMaxL;
  float* const tau = e2 + kMaxL;
  float* const lam = tau + kMaxL;
  __shared__ double s_red[32];
  __shared__ float s_bnd[3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  const float pivmin = 1e-30f;

  // ---- 1. A = G / max_i G_ii (FP32, both triangles from G's lower one)
  double dm = 0.0;
  for (int i = tid; i < l; i += nt) dm = fmax(dm, fabs(G[i + (size_t)i * l]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if (lane == 0) s_red[warp] = dm;
  __syncthreads();
  if (warp == 0) {
    dm = lane < (nt >> 5) ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) s_red[0] = dm;
  }
  __syncthreads();
  dm = s_red[0];
  const double sc = dm > 0.0 ? 1.0 / dm : 1.0;
  for (int e = tid; e < l * l; e += nt) {
    const int i = e / l, j = e - i * l;
    const int a = max(i, j), b = min(i, j);
    A[i * lda + j] = (float)(G[a + (size_t)b * l] * sc);
  }
  __syncthreads();

  // ---- 2. Householder tridiagonalization.  Row r of the trailing matrix
  // belongs to warp r % 32 (matrix-vector product and rank-2 update);
  // step j's reflector comes from row j (= column j) and is kept in row j,
  // columns j+2..l-1 (v_j(j+1) = 1 is implicit).
  for (int j = 0; j + 1 < l; ++j) {
    const int m = l - 1 - j;
    float* const v = vs + (j & 1) * kMaxL;
    float* const Aj = A + j * lda + j + 1;
    if (warp == (j & 31)) {
      float s2 = 0.f;
      for (int k = 1 + lane; k < m; k += 32) s2 = fmaf(Aj[k], Aj[k], s2);
      s2 = warp_sum(s2);
      const float alpha = Aj[0];
      float t = 0.f, scv = 0.f, beta = alpha;
      if (s2 > 0.f) {
        beta = -copysignf(sqrtf(fmaf(alpha, alpha, s2)), alpha);
        t = (beta - alpha) / beta;
        scv = 1.f / (alpha - beta);
      }
      for (int k = lane; k < m; k += 32) {
        const float vk = k == 0 ? 1.f : Aj[k] * scv;
        v[k] = vk;
        if (k) Aj[k] = vk;
      }
      if (lane == 0) {
        tau[j] = t;
        dd[j] = A[j * lda + j];
        ee[j] = beta;
      }
    }
    __syncthreads();
    const float t = tau[j];
    if (t == 0.f) continue;
    const int r0 = j + 1 + ((warp - (j + 1)) & 31);  // first row of this warp
    float s[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 32 * u;
      s[u] = 0.f;
      if (r < l) {
        const float* Ar = A + r * lda + j + 1;
        for (int k = lane; k < m; k += 32) s[u] = fmaf(Ar[k], v[k], s[u]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + 32 * u < l) ps[r0 + 32 * u - j - 1] = t * s[u];
    }
    __syncthreads();
    // w = p - (t/2)(p.v) v; A22 -= v w^T + w v^T on this warp's rows
    float pv = 0.f;
    for (int k = lane; k < m; k += 32) pv = fmaf(ps[k], v[k], pv);
    const float K = -0.5f * t * warp_sum(pv);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 32 * u;
      if (r >= l) break;
      const int i = r - j - 1;
      const float vi = v[i], wi = fmaf(K, vi, ps[i]);
      float* Ar = A + r * lda + j + 1;
      for (int k = lane; k < m; k += 32) {
        const float vk = v[k];
        const float wk = fmaf(K, vk, ps[k]);
        Ar[k] = fmaf(-wi, vk, fmaf(-vi, wk, Ar[k]));
      }
    }
  }
  if (tid == 0) dd[l - 1] = A[(l - 1) * lda + l - 1];
  __syncthreads();

  // ---- 3. eigenvalues of T (ascending) by multisection
  for (int k = tid; k + 1 < l; k += nt) e2[k] = ee[k] * ee[k];
  if (warp == 0) {
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int k = lane; k < l; k += 32) {
      const float r = (k > 0 ? fabsf(ee[k - 1]) : 0.f) + (k + 1 < l ? fabsf(ee[k]) : 0.f);
      lo = fminf(lo, dd[k] - r);
      hi = fmaxf(hi, dd[k] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const float bn = fmaxf(fabsf(lo), fabsf(hi));
    const float pad = 4.f * FLT_EPSILON * bn * (float)l + pivmin;
    if (lane == 0) { s_bnd[0] = lo - pad; s_bnd[1] = hi + pad; s_bnd[2] = bn; }
  }
  __syncthreads();
  {
    const int g = tid / kGrp, t8 = tid % kGrp;
    const unsigned gmask = 0xFFu << (lane & 24);
    if (g < l) {
      float lo = s_bnd[0], hi = s_bnd[1];
      const float atol = 1e-14f * s_bnd[2];
      for (int it = 0; it < 20; ++it) {
        if (hi - lo <= fmaf(2.4e-7f, fmaxf(fabsf(lo), fabsf(hi)), atol)) break;
        const float h = (hi - lo) * (1.f / 9.f);
        const float x = fmaf(h, (float)(t8 + 1), lo);
        float q = dd[0] - x;
        if (fabsf(q) < pivmin) q = -pivmin;
        int c = q < 0.f;
        for (int k = 1; k < l; ++k) {
          q = (dd[k] - x) - __fdividef(e2[k - 1], q);
          if (fabsf(q) < pivmin) q = -pivmin;
          c += q < 0.f;
        }
        const unsigned bits = (__ballot_sync(gmask, c > g) >> (lane & 24)) & 0xFFu;
        const int tt = bits ? __ffs(bits) - 1 : kGrp;
        const float nlo = tt == 0 ? lo : fmaf(h, (float)tt, lo);
        const float nhi = tt == kGrp ? hi : fmaf(h, (float)(tt + 1), lo);
        lo = nlo;
        hi = nhi;
      }
      if (t8 == 0) lam[g] = 0.5f * (lo + hi);
    }
  }
  __syncthreads();

  // ---- 4. eigenvectors of T by twisted factorizations (thread i: lambda_i)
  if (tid < l) {
    float lm = lam[tid];
    float* const Dp = Ws + tid;
    float* const Xc = Xs + tid;
    for (int pass = 0; pass < 2; ++pass) {
      float q = dd[0] - lm;
      if (fabsf(q) < pivmin) q = -pivmin;
      Dp[0] = q;
      for (int k = 1; k < l; ++k) {
        q = (dd[k] - lm) - __fdividef(e2[k - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        Dp[k * ldx] = q;
      }
      // backward pivots D-_k (kept in the vector's column until overwritten)
      float qm = dd[l - 1] - lm;
      if (fabsf(qm) < pivmin) qm = -pivmin;
      Xc[(l - 1) * ldx] = qm;
      float gb = q;  // gamma_{l-1} = D+_{l-1}
      int r = l - 1;
      for (int k = l - 2; k >= 0; --k) {
        const float bm = __fdividef(e2[k], qm);
        const float gk = Dp[k * ldx] - bm;
        if (fabsf(gk) <= fabsf(gb)) { gb = gk; r = k; }
        qm = (dd[k] - lm) - bm;
        if (fabsf(qm) < pivmin) qm = -pivmin;
        Xc[k * ldx] = qm;
      }
      float xv = 1.f, n2 = 1.f;
      Xc[r * ldx] = 1.f;
      for (int k = r - 1; k >= 0; --k) {
        xv = -__fdividef(ee[k], Dp[k * ldx]) * xv;
        Xc[k * ldx] = xv;
        n2 = fmaf(xv, xv, n2);
      }
      xv = 1.f;
      for (int k = r; k + 1 < l; ++k) {
        xv = -__fdividef(ee[k], Xc[(k + 1) * ldx]) * xv;
        Xc[(k + 1) * ldx] = xv;
        n2 = fmaf(xv, xv, n2);
      }
      if (!(n2 <= FLT_MAX)) {  // overflow: fall back to e_r (the cluster pass may replace it)
        for (int k = 0; k < l; ++k) Xc[k * ldx] = k == r ? 1.f : 0.f;
        n2 = 1.f;
      }
      if (pass == 0) {
        lm += gb / n2;
      } else {
        const float s = rsqrtf(n2);
        for (int k = 0; k < l; ++k) Xc[k * ldx] *= s;
      }
    }
  }
  __syncthreads();

  // ---- 5. orthogonalise vectors of close eigenvalues (warp 0)
  if (warp == 0) {
    const float ctol = 1e-4f * fmaxf(fabsf(lam[0]), fabsf(lam[l - 1]));
    int start = 0, nrep = 0;
    for (int i = 1; i <= l; ++i) {
      if (i < l && lam[i] - lam[i - 1] <= ctol) continue;
      for (int a = start + 1; a < i; ++a) {
        float xa[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = lane + 32 * u;
          xa[u] = r < l ? Xs[r * ldx + a] : 0.f;
        }
        for (int b = start; b < a; ++b) {
          float xb[4], dt = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = lane + 32 * u;
            xb[u] = r < l ? Xs[r * ldx + b] : 0.f;
            dt = fmaf(xa[u], xb[u], dt);
          }
          dt = warp_sum(dt);
#pragma unroll
          for (int u = 0; u < 4; ++u) xa[u] = fmaf(-dt, xb[u], xa[u]);
        }
        float n2 = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) n2 = fmaf(xa[u], xa[u], n2);
        n2 = warp_sum(n2);
        if (n2 < 0.25f) {
          // a multiple eigenvalue: a pseudo-random vector orthogonal to all others
          ++nrep;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = lane + 32 * u;
            const uint32_t h = mix32((uint32_t)(a * 131 + r) * 2654435761u + 12345u);
            xa[u] = r < l ? (float)(h >> 8) * (1.f / 8388608.f) - 1.f : 0.f;
          }
          for (int rep = 0; rep < 2; ++rep)
            for (int b = 0; b < l; ++b) {
              if (b == a) continue;
              float xb[4], dt = 0.f;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int r = lane + 32 * u;
                xb[u] = r < l ? Xs[r * ldx + b] : 0.f;
                dt = fmaf(xa[u], xb[u], dt);
              }
              dt = warp_sum(dt);
#pragma unroll
              for (int u = 0; u < 4; ++u) xa[u] = fmaf(-dt, xb[u], xa[u]);
            }
          n2 = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) n2 = fmaf(xa[u], xa[u], n2);
          n2 = warp_sum(n2);
        }
        const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = lane + 32 * u;
          if (r < l) Xs[r * ldx + a] = xa[u] * s;
        }
        __syncwarp();
      }
      start = i;
    }
    // diagnostic word at byte 16 of the status block: replaced vectors
    if (lane == 0) status[4] = (unsigned)nrep;
  }
  __syncthreads();

  // ---- 6. back-transformation X = H_0 ... H_{l-2} Z (8 threads per column)
  {
    const int c = tid / kGrp, t8 = tid % kGrp;
    const unsigned gmask = 0xFFu << (lane & 24);
    if (c < l) {
      float xr[kRowsPerThread], vr[kRowsPerThread];
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        const int r = t8 + kGrp * u;
        xr[u] = r < l ? Xs[r * ldx + c] : 0.f;
      }
      for (int j = l - 2; j >= 0; --j) {
        const float t = tau[j];
        if (t == 0.f) continue;
        const float* vj = A + j * lda;
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < kRowsPerThread; ++u) {
          const int r = t8 + kGrp * u;
          vr[u] = (r > j + 1 && r < l) ? vj[r] : (r == j + 1 ? 1.f : 0.f);
          s = fmaf(vr[u], xr[u], s);
        }
        s += __shfl_xor_sync(gmask, s, 1);
        s += __shfl_xor_sync(gmask, s, 2);
        s += __shfl_xor_sync(gmask, s, 4);
        const float f = t * s;
#pragma unroll
        for (int u = 0; u < kRowsPerThread; ++u) xr[u] = fmaf(-f, vr[u], xr[u]);
      }
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        const int r = t8 + kGrp * u;
        if (r < l) Xout[r + (size_t)c * l] = (double)xr[u];
      }
    }
  }
}

}  // namespace

cudaError_t tridiag_eig32(cudaStream_t st, int l, const double* G, double* X, unsigned* status) {
  if (l < 1 || l > kMaxL) return cudaErrorInvalidValue;
  k_tridiag_eig32<<<1, kEigThreads, eig_smem_bytes(l), st>>>(l, G, X, status);
  note_launch();
  return cudaGetLastError();
}

void prepare_eig_kernels() {
  cudaFuncSetAttribute(k_tridiag_eig32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)eig_smem_bytes(kMaxL));
}

}  // namespace rpod
