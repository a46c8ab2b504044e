// Starting eigenvectors of the small SVD (Alg. 1, SVD of T = Q^T S): the
// left singular vectors of T are the eigenvectors of its l x l Gram matrix
// G = T T^T, and the eigensolver refines a starting basis X in FP64
// (Ogita-Aishima passes, rpod_simt.cu).  This file computes that start in
// FP32 in four launches:
//
//   1. (one CTA) G / max_i G_ii in FP32; Householder reduction to
//      tridiagonal form A = H T H^T (lower variant: column 0 first, so a
//      matrix whose large entries sit at the top left -- the Gram of a
//      power-iterated basis -- keeps its small eigenvalues' relative
//      accuracy).  The diagonal and off-diagonal of T, the reflector
//      vectors and their factors go to a scratch buffer.
//   2. (one CTA per eight eigenvalues) Eigenvalues of T by multisection on
//      Sturm counts (the number of negative pivots of the LDL^T
//      factorization of T - x I is the number of eigenvalues below x): one
//      pass of 256 counts at geometrically spaced points brackets every
//      eigenvalue, then a warp per eigenvalue narrows its bracket with 32
//      points per step to a relative width of two ulps.  The counts use IEEE
//      infinities in place of a pivot threshold (a zero pivot gives an
//      infinite next pivot, counted by its sign bit), with e_k^2 kept at or
//      above the smallest normal number so that no 0/0 arises.
//      Eigenvectors of T from twisted factorizations (Dhillon and Parlett,
//      "Multiple representations to compute orthogonal eigenvectors of
//      symmetric tridiagonal matrices", Lin. Alg. Appl. 387, 2004): with the
//      forward pivots D+ and backward pivots D- of T - lambda I, the twist
//      index r minimising |gamma_r|, gamma_r = D+_r - e_r^2 / D-_{r+1},
//      gives the vector with x_r = 1 by two one-term recurrences.  Two
//      threads per eigenvalue, in different warps: one runs the forward
//      recurrences, one the backward ones.
//   3. (one CTA) Vectors of eigenvalues closer than 1e-5 ||T|| are
//      orthogonalised against each other (Gram-Schmidt in ascending order);
//      a vector that loses more than half its norm there (a multiple
//      eigenvalue) is replaced by inverse iteration with T - lambda I from
//      a pseudo-random vector, orthogonalised against the cluster's other
//      vectors.  Vectors of eigenvalues further apart come out of step 2
//      orthogonal to a few 1e-5 at most, which the refinement removes;
//      without a cluster this launch ends after the gap test.
//   4. (one CTA per 32 columns) Back-transformation X = H Z, each pair of
//      columns held in the registers of 16 threads.
//
// Step 1 keeps the rows of A as float4 (four consecutive rows per warp, the
// reduced rows replaced by the full reflector vectors, zeros included), so
// that the matrix-vector product, the rank-2 update and the
// back-transformation run on 16-byte shared-memory accesses without
// per-element bounds tests.  Steps 2 and 4 spread the independent
// per-eigenvalue and per-column work over many SMs.
//
// The FP64 refinement that follows squares the error of this start per
// pass; its accuracy, not this one's, sets the final result.
#include <float.h>
#include <math.h>

#include "rpod_internal.cuh"

namespace rpod {
namespace {

constexpr int kEigThreads = 1024;  // tridiagonalization and cluster kernels
constexpr int kVecThreads = 256;   // eigenvalue / eigenvector kernel
constexpr int kEpb = 8;            // eigenvalues per CTA of that kernel
constexpr int kBackThreads = 256;  // back-transformation: 16 column pairs per CTA
constexpr int kBackCols = 32;

// Rows of A start on 16-byte boundaries; the cluster pass's Z uses a leading
// dimension of 1 mod 32, so that a column and a row each fall in distinct
// banks.
__host__ __device__ inline int eig_lda(int l) { return (l + 3) & ~3; }
__host__ __device__ inline int eig_ldx(int l) { return ((l + 31) & ~31) + 1; }

// Shared memory of the tridiagonalization (A, reflector and p buffers, d, e,
// tau), the cluster pass (Z and the dot-product buffer) and the
// back-transformation (the reflector rows).
size_t tri_smem_bytes(int l) { return sizeof(float) * ((size_t)l * eig_lda(l) + 7 * (size_t)kMaxL); }
size_t clu_smem_bytes(int l) { return sizeof(float) * ((size_t)l * eig_ldx(l) + (size_t)kMaxL); }
size_t back_smem_bytes(int l) { return sizeof(float) * (size_t)l * eig_lda(l); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float pick(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// Number of eigenvalues of the tridiagonal T below x: the negative pivots
// of the LDL^T factorization of T - x I (de[k] = (d_k, e_{k-1}^2)).
__device__ __forceinline__ unsigned sturm_count(const float2* de, int l, float x) {
  float q = de[0].x - x;
  unsigned c = __float_as_uint(q) >> 31;
#pragma unroll 4
  for (int k = 1; k < l; ++k) {
    const float2 p = de[k];
    q = fmaf(-p.y, __fdividef(1.f, q), p.x - x);
    c += __float_as_uint(q) >> 31;
  }
  return c;
}

constexpr int kBrk = 256;  // bracketing points (one per thread)
constexpr int kMs = 32;    // points per eigenvalue and multisection step (a warp)
static_assert(kBrk == kVecThreads, "one bracketing point per thread");
static_assert(kEpb * kMs <= kVecThreads, "multisection threads");
static_assert(kEpb <= 32, "one lane per eigenvalue in the vector recurrences");

__device__ __forceinline__ float brk_point(float bn, int i) {
  return bn * exp2f(40.f * ((float)i * (1.f / (kBrk - 1)) - 1.f));
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
  return x;
}

// Householder reflector of step j from row j (x: this lane's columns
// 4 lane .. 4 lane + 3), called by all 32 lanes of one warp.  Writes the full
// vector v (zeros up to column j, 1 at j + 1) to row j of A and to vbuf,
// tau_j, d_j and e_j, and clears the two entries of the step's p buffer
// that the step before last left behind.
__device__ __forceinline__ void reflector(int j, int lda, const float4& x, int lane, float* rowj,
                                          float* vbuf, float* pbuf, float* tau, float* dd,
                                          float* ee) {
  const int c0 = 4 * lane;
  float s2 = 0.f;
  s2 = c0 + 0 > j + 1 ? fmaf(x.x, x.x, s2) : s2;
  s2 = c0 + 1 > j + 1 ? fmaf(x.y, x.y, s2) : s2;
  s2 = c0 + 2 > j + 1 ? fmaf(x.z, x.z, s2) : s2;
  s2 = c0 + 3 > j + 1 ? fmaf(x.w, x.w, s2) : s2;
  s2 = warp_sum(s2);
  const float alpha = __shfl_sync(0xffffffffu, pick(x, (j + 1) & 3), (j + 1) >> 2);
  const float djj = __shfl_sync(0xffffffffu, pick(x, j & 3), j >> 2);
  float t = 0.f, scv = 0.f, beta = alpha;
  if (s2 > 0.f) {
    beta = -copysignf(sqrtf(fmaf(alpha, alpha, s2)), alpha);
    t = (beta - alpha) / beta;
    scv = 1.f / (alpha - beta);
  }
  float4 v;
  v.x = c0 + 0 == j + 1 ? 1.f : (c0 + 0 > j + 1 ? x.x * scv : 0.f);
  v.y = c0 + 1 == j + 1 ? 1.f : (c0 + 1 > j + 1 ? x.y * scv : 0.f);
  v.z = c0 + 2 == j + 1 ? 1.f : (c0 + 2 > j + 1 ? x.z * scv : 0.f);
  v.w = c0 + 3 == j + 1 ? 1.f : (c0 + 3 > j + 1 ? x.w * scv : 0.f);
  if (c0 < lda) {
    *reinterpret_cast<float4*>(rowj + c0) = v;
    *reinterpret_cast<float4*>(vbuf + c0) = v;
  }
  if (lane == 0) {
    tau[j] = t;
    dd[j] = djj;
    ee[j] = beta;
    pbuf[j] = 0.f;
    if (j > 0) pbuf[j - 1] = 0.f;
  }
}

// Step 1: G scaled to FP32, Householder tridiagonalization; T's diagonal
// and off-diagonal, the reflector rows (row j = v_j) and their factors tau_j
// are written to the scratch buffer.
__global__ void __launch_bounds__(kEigThreads)
k_eig_tri(int l, const double* __restrict__ G, float* __restrict__ sA, float* __restrict__ sd,
          float* __restrict__ se, float* __restrict__ stau) {
  extern __shared__ float4 sm4[];
  const int lda = eig_lda(l);
  float* const A = reinterpret_cast<float*>(sm4);  // l x lda
  float* const vs = A + (size_t)l * lda;           // [2][kMaxL] reflector vectors
  float* const psb = vs + 2 * kMaxL;               // [2][kMaxL] p = tau A22 v
  float* const dd = psb + 2 * kMaxL;               // diagonal of T
  float* const ee = dd + kMaxL;                    // off-diagonal of T
  float* const tau = ee + kMaxL;
  __shared__ double s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

  // ---- 1. A = G / max_i G_ii (FP32, zero padding columns); p buffers
  // cleared
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
  // entries of a Gram matrix are bounded by its largest diagonal entry;
  // when that is above 1e-30 the FP32 conversion before scaling loses nothing
  const bool f32scale = dm > 1e-30;
  const double scd = dm > 0.0 ? 1.0 / dm : 1.0;
  const float scf = (float)scd;
  // row i of A from column i of the symmetric G (coalesced); warp w holds
  // rows w + 32u, eight loads of a thread in flight before their stores
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    double g[8];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = warp + 32 * (2 * h + u), j = lane + 32 * q;
        g[4 * u + q] = (i < l && j < l) ? G[j + (size_t)i * l] : 0.0;
      }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = warp + 32 * (2 * h + u), j = lane + 32 * q;
        if (i < l && j < lda)
          A[i * lda + j] = f32scale ? (float)g[4 * u + q] * scf : (float)(g[4 * u + q] * scd);
      }
  }
  for (int e = tid; e < 2 * kMaxL; e += nt) psb[e] = 0.f;
  __syncthreads();

  // ---- 2. Householder tridiagonalization.  Warp w owns rows 4w..4w+3 of
  // the trailing matrix and keeps them in registers for the whole
  // reduction (lane q holds columns 4q..4q+3 of a row).  Step j:
  // p = tau A22 v on the owned rows, then A22 -= v w^T + w v^T with
  // w = p - (tau/2)(p.v) v; the owner of row j+1 forms the next reflector
  // from the updated row while it is still in registers and stores it (the
  // full vector, zeros included) as row j+1 of A for the back-transformation.
  // Columns up to j of v and p are zero, so whole rows are processed; the
  // register copies of rows already reduced are no longer read.
  const int c0 = 4 * lane;
  const bool lact = c0 < lda;
  const int rb = 4 * warp;
  float4 rw[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = rb + u;
    rw[u] = (r < l && lact) ? *reinterpret_cast<const float4*>(A + r * lda + c0) : z4;
  }
  if (l >= 2 && warp == 0) reflector(0, lda, rw[0], lane, A, vs, psb, tau, dd, ee);
  for (int j = 0; j + 1 < l; ++j) {
    __syncthreads();
    const float t = tau[j];
    const int nxt = j + 1;
    const bool mk_next = nxt + 1 < l && warp == (nxt >> 2);
    if (t == 0.f) {
      if (mk_next) {
        const int u = nxt & 3;
        const float4 x = u == 0 ? rw[0] : (u == 1 ? rw[1] : (u == 2 ? rw[2] : rw[3]));
        reflector(nxt, lda, x, lane, A + nxt * lda, vs + (nxt & 1) * kMaxL,
                  psb + (nxt & 1) * kMaxL, tau, dd, ee);
      }
      continue;
    }
    const float* const v = vs + (j & 1) * kMaxL;
    float* const ps = psb + (j & 1) * kMaxL;
    const bool owns = rb + 3 >= j + 1 && rb < l;
    float4 v4 = z4;
    if (owns) {
      v4 = lact ? *reinterpret_cast<const float4*>(v + c0) : z4;
      float s[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] = dot4(rw[u], v4);
      // four row sums at once: lanes 8u..8u+7 end with the sum of row rb+u
      const bool hi16 = lane & 16, hi8 = lane & 8;
      float k0 = hi16 ? s[2] : s[0], k1 = hi16 ? s[3] : s[1];
      k0 += __shfl_xor_sync(0xffffffffu, hi16 ? s[0] : s[2], 16);
      k1 += __shfl_xor_sync(0xffffffffu, hi16 ? s[1] : s[3], 16);
      float k = hi8 ? k1 : k0;
      k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
      k += __shfl_xor_sync(0xffffffffu, k, 4);
      k += __shfl_xor_sync(0xffffffffu, k, 2);
      k += __shfl_xor_sync(0xffffffffu, k, 1);
      const int r = rb + (lane >> 3);
      if ((lane & 7) == 0 && r >= j + 1 && r < l) ps[r] = t * k;
    }
    __syncthreads();
    if (owns) {
      const float4 p4 = lact ? *reinterpret_cast<const float4*>(ps + c0) : z4;
      const float K = -0.5f * t * warp_sum(dot4(p4, v4));
      float4 w4;
      w4.x = fmaf(K, v4.x, p4.x); w4.y = fmaf(K, v4.y, p4.y);
      w4.z = fmaf(K, v4.z, p4.z); w4.w = fmaf(K, v4.w, p4.w);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = rb + u;
        if (r < j + 1 || r >= l) continue;
        const float vr = v[r], wr = fmaf(K, vr, ps[r]);
        float4 a = rw[u];
        a.x = fmaf(-wr, v4.x, fmaf(-vr, w4.x, a.x));
        a.y = fmaf(-wr, v4.y, fmaf(-vr, w4.y, a.y));
        a.z = fmaf(-wr, v4.z, fmaf(-vr, w4.z, a.z));
        a.w = fmaf(-wr, v4.w, fmaf(-vr, w4.w, a.w));
        rw[u] = a;
        if (r == nxt && mk_next)
          reflector(nxt, lda, a, lane, A + nxt * lda, vs + (nxt & 1) * kMaxL,
                    psb + (nxt & 1) * kMaxL, tau, dd, ee);
      }
    }
  }
  // the last diagonal entry, from the registers of its row's owner
  if (warp == ((l - 1) >> 2) && lane == ((l - 1) >> 2)) {
    const int u = (l - 1) & 3;
    const float4 x = u == 0 ? rw[0] : (u == 1 ? rw[1] : (u == 2 ? rw[2] : rw[3]));
    dd[l - 1] = pick(x, (l - 1) & 3);
  }
  __syncthreads();

  // T and the reflectors to the scratch buffer
  for (int e = tid; e < l * lda / 4; e += nt)
    reinterpret_cast<float4*>(sA)[e] = reinterpret_cast<const float4*>(A)[e];
  for (int k = tid; k < l; k += nt) {
    sd[k] = dd[k];
    se[k] = k + 1 < l ? ee[k] : 0.f;
    stau[k] = k + 1 < l ? tau[k] : 0.f;
  }
}

// Step 2: eigenvalues g0 .. g0 + kEpb - 1 of T (g0 = kEpb blockIdx.x) and
// their eigenvectors, written as columns of Z (ld l) and to lam.
__global__ void __launch_bounds__(kVecThreads)
k_eig_vec(int l, const float* __restrict__ sd, const float* __restrict__ se, float* __restrict__ Z,
          float* __restrict__ slam) {
  __shared__ float dd[kMaxL], ee[kMaxL];
  __shared__ float2 de[kMaxL];
  __shared__ float lam[kEpb];
  __shared__ float s_bnd[3];
  __shared__ unsigned s_cnt[kBrk];
  constexpr int ldx = kEpb + 1;  // pivots and vectors of the CTA's eigenvalues: row k at k * ldx
  __shared__ float Ws[kMaxL * ldx], Xs[kMaxL * ldx];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  const int g0 = kEpb * blockIdx.x;
  const float pivmin = 1e-30f;
  for (int k = tid; k < l; k += blockDim.x) {
    dd[k] = sd[k];
    ee[k] = se[k];
  }
  __syncthreads();
  for (int k = tid; k < l; k += nt)
    de[k] = make_float2(dd[k], k > 0 ? fmaxf(ee[k - 1] * ee[k - 1], FLT_MIN) : 0.f);
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
    // (the e_k^2 floor moves eigenvalues by less than 1e-18)
    const float pad = 4.f * FLT_EPSILON * bn * (float)l + 1e-18f;
    if (lane == 0) { s_bnd[0] = lo - pad; s_bnd[1] = hi + pad; s_bnd[2] = bn; }
  }
  __syncthreads();
  // bracketing pass: every thread counts the eigenvalues below one of
  // kBrk points spaced geometrically over 2^-40 bn .. bn (the eigenvalues of
  // a power-iterated Gram spread over decades; ratio 1.115 between points)
  {
    const float bn = s_bnd[2];
    s_cnt[tid] = tid < kBrk ? sturm_count(de, l, brk_point(bn, tid)) : 0u;
  }
  __syncthreads();
  {
    // one warp per eigenvalue: kMs = 32 points per step (5 bits)
    const int gl = warp, g = g0 + gl;
    if (gl < kEpb && g < l) {
      // first point whose count exceeds g (binary search: the points on
      // either side of the result were both probed, so lambda_g lies
      // between them even where rounding makes the counts non-monotone)
      int bl = 0, bh = kBrk;
      while (bl < bh) {
        const int md = (bl + bh) >> 1;
        if (s_cnt[md] > (unsigned)g) bh = md; else bl = md + 1;
      }
      const float bn = s_bnd[2];
      float lo = bl == 0 ? s_bnd[0] : brk_point(bn, bl - 1);
      float hi = bl == kBrk ? s_bnd[1] : brk_point(bn, bl);
      const float atol = 1e-14f * bn;
      for (int it = 0; it < 40; ++it) {
        if (hi - lo <= fmaf(2.4e-7f, fmaxf(fabsf(lo), fabsf(hi)), atol)) break;
        const float h = (hi - lo) * (1.f / (kMs + 1));
        const unsigned c = sturm_count(de, l, fmaf(h, (float)(lane + 1), lo));
        const unsigned bits = __ballot_sync(0xffffffffu, c > (unsigned)g);
        const int tt = bits ? __ffs(bits) - 1 : kMs;
        const float nlo = tt == 0 ? lo : fmaf(h, (float)tt, lo);
        const float nhi = tt == kMs ? hi : fmaf(h, (float)(tt + 1), lo);
        lo = nlo;
        hi = nhi;
      }
      if (lane == 0) lam[gl] = 0.5f * (lo + hi);
    }
  }
  __syncthreads();

  // eigenvectors of T by twisted factorizations: lane il of warp 0 runs the
  // forward pivots D+ (into Ws) and the vector above the twist index, lane
  // il of warp 1 the backward pivots D- (into Xs) and the vector below it,
  // for lambda_il (two warps, so the two recurrences run side by side)
  {
    __shared__ float s_gb[2][kEpb], s_n2[2][kEpb];
    __shared__ int s_r[2][kEpb];
    const bool fwd = warp == 0;
    const int il = lane;
    const bool act = warp < 2 && il < kEpb && g0 + il < l;
    float* const Dp = Ws + il;
    float* const Xc = Xs + il;
    const float lm = act ? lam[il] : 0.f;
    if (act) {
      if (fwd) {
        float q = dd[0] - lm;
        if (fabsf(q) < pivmin) q = -pivmin;
        Dp[0] = q;
#pragma unroll 4
        for (int k = 1; k < l; ++k) {
          q = (dd[k] - lm) - __fdividef(de[k].y, q);
          if (fabsf(q) < pivmin) q = -pivmin;
          Dp[k * ldx] = q;
        }
      } else {
        float q = dd[l - 1] - lm;
        if (fabsf(q) < pivmin) q = -pivmin;
        Xc[(l - 1) * ldx] = q;
#pragma unroll 4
        for (int k = l - 2; k >= 0; --k) {
          q = (dd[k] - lm) - __fdividef(de[k + 1].y, q);
          if (fabsf(q) < pivmin) q = -pivmin;
          Xc[k * ldx] = q;
        }
      }
    }
    __syncthreads();
    // twist index: gamma_k = D+_k - e_k^2 / D-_{k+1} (gamma_{l-1} = D+_{l-1});
    // the forward lane scans k < l/2, the backward one the rest
    if (act) {
      const int h = l >> 1;
      float gb = FLT_MAX;
      int r = l;
#pragma unroll 4
      for (int k = fwd ? 0 : h; k < (fwd ? h : l); ++k) {
        const float gk = k + 1 < l ? Dp[k * ldx] - __fdividef(de[k + 1].y, Xc[(k + 1) * ldx])
                                   : Dp[k * ldx];
        if (fabsf(gk) < gb) { gb = fabsf(gk); r = k; }
      }
      s_gb[warp][il] = gb;
      s_r[warp][il] = r;
    }
    __syncthreads();
    int r = l;
    if (act) {
      const float g0v = s_gb[0][il], g1v = s_gb[1][il];
      const int r0 = s_r[0][il], r1 = s_r[1][il];
      r = (g1v < g0v || (g1v == g0v && r1 < r0)) ? r1 : r0;
      if (r >= l) r = 0;  // every gamma non-finite: any twist index will do
    }
    __syncthreads();  // the pivots read by the twist scan are overwritten below
    float n2 = 0.f;
    if (act) {
      float xv = 1.f;
      if (fwd) {
        Xc[r * ldx] = 1.f;
        n2 = 1.f;
        for (int k = r - 1; k >= 0; --k) {
          xv = -__fdividef(ee[k], Dp[k * ldx]) * xv;
          Xc[k * ldx] = xv;
          n2 = fmaf(xv, xv, n2);
        }
      } else {
        for (int k = r; k + 1 < l; ++k) {
          xv = -__fdividef(ee[k], Xc[(k + 1) * ldx]) * xv;
          Xc[(k + 1) * ldx] = xv;
          n2 = fmaf(xv, xv, n2);
        }
      }
      s_n2[warp][il] = n2;
    }
    __syncthreads();
    if (act) {
      n2 = s_n2[0][il] + s_n2[1][il];
      if (!(n2 <= FLT_MAX)) {  // overflow: e_r instead (the cluster pass may replace it)
        for (int k = fwd ? 0 : 1; k < l; k += 2) Xc[k * ldx] = k == r ? 1.f : 0.f;
      } else {
        const float sc = rsqrtf(n2);
        if (fwd) {
          for (int k = 0; k <= r; ++k) Xc[k * ldx] *= sc;
        } else {
          for (int k = r + 1; k < l; ++k) Xc[k * ldx] *= sc;
        }
      }
    }
  }
  __syncthreads();

  // the CTA's vectors to Z and its eigenvalues to lam
  for (int e = tid; e < kEpb * l; e += blockDim.x) {
    const int el = e / l, r = e - el * l;
    if (g0 + el < l) Z[r + (size_t)(g0 + el) * l] = Xs[r * ldx + el];
  }
  if (tid < kEpb && g0 + tid < l) slam[g0 + tid] = lam[tid];
}

// Step 3: vectors of clustered eigenvalues (Z in place); without a cluster
// the kernel ends after the gap test.
__global__ void __launch_bounds__(kEigThreads)
k_eig_cluster(int l, const float* __restrict__ sd, const float* __restrict__ se,
              const float* __restrict__ slam, float* __restrict__ Z, unsigned* __restrict__ status) {
  extern __shared__ float4 sm4[];
  const int ldx = eig_ldx(l);
  float* const Xs = reinterpret_cast<float*>(sm4);  // Z: row r at r * ldx
  float* const Ws = Xs + (size_t)l * ldx;           // dot products
  __shared__ float lam[kMaxL], dd[kMaxL], ee[kMaxL];
  __shared__ int s_any;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  if (tid == 0) s_any = 0;
  for (int k = tid; k < l; k += nt) {
    lam[k] = slam[k];
    dd[k] = sd[k];
    ee[k] = se[k];
  }
  __syncthreads();
  {
    const float ctol = fmaxf(1e-5f * fmaxf(fabsf(lam[0]), fabsf(lam[l - 1])), 1e-15f);
    for (int i = tid + 1; i < l; i += nt)
      if (lam[i] - lam[i - 1] <= ctol) s_any = 1;
  }
  __syncthreads();
  if (!s_any) {
    if (tid == 0) status[4] = 0u;
    return;
  }
  for (int e = tid; e < l * l; e += nt) {
    const int g = e / l, r = e - g * l;
    Xs[r * ldx + g] = Z[e];
  }
  __syncthreads();
  // orthogonalise vectors of close eigenvalues.  Per vector a of a
  // cluster, two classical Gram-Schmidt passes against the cluster's
  // earlier (already orthonormal) vectors: the dots by one warp each, the
  // update by 16 threads per row.  A vector that loses more than half its
  // norm (a multiple eigenvalue) is replaced by warp 0: inverse iteration
  // with T - lambda I from a pseudo-random vector, which keeps the
  // replacement in its own cluster's invariant subspace (orthogonalising a
  // random vector against all other vectors does not: while another
  // cluster still holds a duplicate, that complement mixes both clusters'
  // missing directions), then modified Gram-Schmidt against the cluster's
  // processed vectors.  The forward-pivot array is free again and holds the
  // dot products.
  {
    float* const dts = Ws;
    __shared__ float s_n2;
    // inverse iteration of a replaced vector: LU of T - lambda I and the vector
    __shared__ float s_d[kMaxL], s_du[kMaxL], s_dl[kMaxL], s_du2[kMaxL], s_iv[kMaxL];
    __shared__ int s_piv[kMaxL];
    // eigenvalues closer than 1e-15 are one cluster even in a (near) zero matrix
    const float ctol = fmaxf(1e-5f * fmaxf(fabsf(lam[0]), fabsf(lam[l - 1])), 1e-15f);
    const int part = tid & 15, rsub = tid >> 4;
    const unsigned hmask = 0xFFFFu << (lane & 16);
    int start = 0, nrep = 0;
    for (int i = 1; i <= l; ++i) {
      if (i < l && lam[i] - lam[i - 1] <= ctol) continue;
      for (int a = start + 1; a < i; ++a) {
        for (int pass = 0; pass < 2; ++pass) {
          for (int b = start + warp; b < a; b += nt >> 5) {
            float dt = 0.f;
            for (int r = lane; r < l; r += 32) dt = fmaf(Xs[r * ldx + b], Xs[r * ldx + a], dt);
            dt = warp_sum(dt);
            if (lane == 0) dts[b] = dt;
          }
          __syncthreads();
          for (int r0 = 0; r0 < l; r0 += nt >> 4) {
            const int r = r0 + rsub;
            float acc = 0.f;
            if (r < l)
              for (int b = start + part; b < a; b += 16) acc = fmaf(dts[b], Xs[r * ldx + b], acc);
            acc += __shfl_xor_sync(hmask, acc, 1);
            acc += __shfl_xor_sync(hmask, acc, 2);
            acc += __shfl_xor_sync(hmask, acc, 4);
            acc += __shfl_xor_sync(hmask, acc, 8);
            if (r < l && part == 0) Xs[r * ldx + a] -= acc;
          }
          __syncthreads();
        }
        if (warp == 0) {
          float n2 = 0.f;
          for (int r = lane; r < l; r += 32) n2 = fmaf(Xs[r * ldx + a], Xs[r * ldx + a], n2);
          n2 = warp_sum(n2);
          if (n2 < 0.25f) {
            // a multiple eigenvalue: two steps of inverse iteration with
            // T - lambda_a I from a pseudo-random vector (the cluster's own
            // invariant subspace grows by about 1/eps against every other
            // eigenvector), then Gram-Schmidt against the cluster's
            // processed vectors
            ++nrep;
            const float lm = lam[a];
            for (int r = lane; r < l; r += 32) {
              const uint32_t hsh = mix32((uint32_t)(a * 131 + r) * 2654435761u + 12345u);
              s_iv[r] = (float)(hsh >> 8) * (1.f / 8388608.f) - 1.f;
            }
            __syncwarp();
            if (lane == 0) {
              // LU with partial pivoting of the tridiagonal T - lm I
              const float tn = fmaxf(fmaxf(fabsf(lam[0]), fabsf(lam[l - 1])), 1e-30f);
              const float tiny = FLT_EPSILON * tn;
              for (int k = 0; k < l; ++k) {
                s_d[k] = dd[k] - lm;
                s_du[k] = k + 1 < l ? ee[k] : 0.f;
                s_dl[k] = k + 1 < l ? ee[k] : 0.f;
                s_du2[k] = 0.f;
                s_piv[k] = 0;
              }
              for (int k = 0; k + 1 < l; ++k) {
                if (fabsf(s_d[k]) >= fabsf(s_dl[k])) {
                  if (!(fabsf(s_d[k]) >= tiny)) s_d[k] = s_d[k] < 0.f ? -tiny : tiny;
                  const float f = s_dl[k] / s_d[k];
                  s_dl[k] = f;
                  s_d[k + 1] -= f * s_du[k];
                } else {
                  const float f = s_d[k] / s_dl[k];
                  s_d[k] = s_dl[k];
                  s_dl[k] = f;
                  const float t = s_du[k];
                  s_du[k] = s_d[k + 1];
                  s_d[k + 1] = t - f * s_d[k + 1];
                  if (k + 2 < l) {
                    s_du2[k] = s_du[k + 1];
                    s_du[k + 1] = -f * s_du[k + 1];
                  }
                  s_piv[k] = 1;
                }
              }
              // pivots below eps ||T|| are raised to it (a perturbation of
              // T at rounding level) so the solves cannot overflow
              for (int k = 0; k < l; ++k)
                if (!(fabsf(s_d[k]) >= tiny)) s_d[k] = s_d[k] < 0.f ? -tiny : tiny;
              for (int step = 0; step < 2; ++step) {
                for (int k = 0; k + 1 < l; ++k) {
                  if (s_piv[k]) {
                    const float t = s_iv[k];
                    s_iv[k] = s_iv[k + 1];
                    s_iv[k + 1] = t - s_dl[k] * s_iv[k + 1];
                  } else {
                    s_iv[k + 1] -= s_dl[k] * s_iv[k];
                  }
                }
                float mx = 0.f;
                for (int k = l - 1; k >= 0; --k) {
                  float v = s_iv[k];
                  if (k + 1 < l) v -= s_du[k] * s_iv[k + 1];
                  if (k + 2 < l) v -= s_du2[k] * s_iv[k + 2];
                  v /= s_d[k];
                  s_iv[k] = v;
                  mx = fmaxf(mx, fabsf(v));
                }
                const float sc = mx > 0.f && mx <= FLT_MAX ? 1.f / mx : 0.f;
                for (int k = 0; k < l; ++k) s_iv[k] = sc > 0.f ? s_iv[k] * sc : (k == a ? 1.f : 0.f);
              }
            }
            __syncwarp();
            float xa[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;
              xa[u] = r < l ? s_iv[r] : 0.f;
            }
            for (int rep = 0; rep < 2; ++rep)
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
            n2 = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) n2 = fmaf(xa[u], xa[u], n2);
            n2 = warp_sum(n2);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;
              if (r < l) Xs[r * ldx + a] = xa[u];
            }
          }
          if (lane == 0) s_n2 = n2;
        }
        __syncthreads();
        const float n2 = s_n2;
        const float sc = n2 > 0.f ? rsqrtf(n2) : 0.f;
        for (int r = tid; r < l; r += nt) Xs[r * ldx + a] *= sc;
        __syncthreads();
      }
      start = i;
    }
    // diagnostic word at byte 16 of the status block: replaced vectors
    if (tid == 0) status[4] = (unsigned)nrep;
  }

  __syncthreads();
  for (int e = tid; e < l * l; e += nt) {
    const int g = e / l, r = e - g * l;
    Z[e] = Xs[r * ldx + g];
  }
}

// Step 4: X = H_0 ... H_{l-2} Z for columns kBackCols blockIdx.x .. + 31,
// with the reflector rows in shared memory.
__global__ void __launch_bounds__(kBackThreads)
k_eig_back(int l, const float* __restrict__ sA, const float* __restrict__ stau,
           const float* __restrict__ Z, double* __restrict__ Xout) {
  extern __shared__ float4 sm4[];
  const int lda = eig_lda(l);
  float* const A = reinterpret_cast<float*>(sm4);  // reflector rows, row j at j * lda
  __shared__ float tau[kMaxL];
  const int tid = threadIdx.x, lane = tid & 31;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = tid; e < l * lda / 4; e += blockDim.x)
    reinterpret_cast<float4*>(A)[e] = reinterpret_cast<const float4*>(sA)[e];
  for (int k = tid; k < l; k += blockDim.x) tau[k] = stau[k];
  __syncthreads();
  // back-transformation X = H_0 ... H_{l-2} Z: 16 threads per pair
  // of columns, thread t16 holding rows 64u + 4 t16 + i (u < 2, i < 4) of
  // both in registers, so that each reflector row read from shared memory
  // serves two columns; row j of A is the full vector v_j.  The two dot
  // products are summed over the 16 threads with one transposed exchange
  // (lanes with bit 3 set carry column 1 on, the others column 0) and two
  // broadcasts.
  {
    const int cp = tid >> 4, t16 = tid & 15;
    const int c = kBackCols * blockIdx.x + 2 * cp;
    const unsigned gmask = 0xFFFFu << (lane & 16);
    if (c < l) {
      const bool two = c + 1 < l;
      float xa[8], xb[8];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 64 * u + 4 * t16 + i;
          xa[4 * u + i] = r < l ? Z[r + (size_t)c * l] : 0.f;
          xb[4 * u + i] = (r < l && two) ? Z[r + (size_t)(c + 1) * l] : 0.f;
        }
      const bool hi8 = lane & 8;
      const int base = lane & 16;
      for (int j = l - 2; j >= 0; --j) {
        const float t = tau[j];
        if (t == 0.f) continue;
        const float* vj = A + j * lda;
        float4 vv[2];
        float sa = 0.f, sb = 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int cc = 64 * u + 4 * t16;
          vv[u] = cc < lda ? *reinterpret_cast<const float4*>(vj + cc) : z4;
          sa = fmaf(vv[u].x, xa[4 * u + 0], fmaf(vv[u].y, xa[4 * u + 1],
                    fmaf(vv[u].z, xa[4 * u + 2], fmaf(vv[u].w, xa[4 * u + 3], sa))));
          sb = fmaf(vv[u].x, xb[4 * u + 0], fmaf(vv[u].y, xb[4 * u + 1],
                    fmaf(vv[u].z, xb[4 * u + 2], fmaf(vv[u].w, xb[4 * u + 3], sb))));
        }
        float k = hi8 ? sb : sa;
        k += __shfl_xor_sync(gmask, hi8 ? sa : sb, 8);
        k += __shfl_xor_sync(gmask, k, 4);
        k += __shfl_xor_sync(gmask, k, 2);
        k += __shfl_xor_sync(gmask, k, 1);
        const float fa = -t * __shfl_sync(gmask, k, base);
        const float fb = -t * __shfl_sync(gmask, k, base + 8);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          xa[4 * u + 0] = fmaf(fa, vv[u].x, xa[4 * u + 0]);
          xa[4 * u + 1] = fmaf(fa, vv[u].y, xa[4 * u + 1]);
          xa[4 * u + 2] = fmaf(fa, vv[u].z, xa[4 * u + 2]);
          xa[4 * u + 3] = fmaf(fa, vv[u].w, xa[4 * u + 3]);
          xb[4 * u + 0] = fmaf(fb, vv[u].x, xb[4 * u + 0]);
          xb[4 * u + 1] = fmaf(fb, vv[u].y, xb[4 * u + 1]);
          xb[4 * u + 2] = fmaf(fb, vv[u].z, xb[4 * u + 2]);
          xb[4 * u + 3] = fmaf(fb, vv[u].w, xb[4 * u + 3]);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 64 * u + 4 * t16 + i;
          if (r < l) {
            Xout[r + (size_t)c * l] = (double)xa[4 * u + i];
            if (two) Xout[r + (size_t)(c + 1) * l] = (double)xb[4 * u + i];
          }
        }
    }
  }
}

}  // namespace

size_t eig_scratch_floats(int l) {
  return (size_t)l * eig_lda(l) + (size_t)l * l + 4 * (size_t)kMaxL;
}

cudaError_t tridiag_eig32(cudaStream_t st, int l, const double* G, double* X, float* scratch,
                          unsigned* status) {
  if (l < 1 || l > kMaxL) return cudaErrorInvalidValue;
  float* const sA = scratch;                        // l x lda reflector rows
  float* const sZ = sA + (size_t)l * eig_lda(l);    // l x l eigenvectors of T
  float* const sd = sZ + (size_t)l * l;
  float* const se = sd + kMaxL;
  float* const stau = se + kMaxL;
  float* const slam = stau + kMaxL;
  k_eig_tri<<<1, kEigThreads, tri_smem_bytes(l), st>>>(l, G, sA, sd, se, stau);
  note_launch();
  k_eig_vec<<<(l + kEpb - 1) / kEpb, kVecThreads, 0, st>>>(l, sd, se, sZ, slam);
  note_launch();
  k_eig_cluster<<<1, kEigThreads, clu_smem_bytes(l), st>>>(l, sd, se, slam, sZ, status);
  note_launch();
  k_eig_back<<<(l + kBackCols - 1) / kBackCols, kBackThreads, back_smem_bytes(l), st>>>(l, sA, stau,
                                                                                      sZ, X);
  note_launch();
  return cudaGetLastError();
}

void prepare_eig_kernels() {
  cudaFuncSetAttribute(k_eig_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tri_smem_bytes(kMaxL));
  cudaFuncSetAttribute(k_eig_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)clu_smem_bytes(kMaxL));
  cudaFuncSetAttribute(k_eig_back, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)back_smem_bytes(kMaxL));
}

}  // namespace rpod
