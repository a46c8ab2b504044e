// SIMT kernels of librpod (Alg. 1, Sec. 4.2): the Philox sketch Lambda
// (first step); the tall-skinny GEMMs of the FP64 and FP32 passes over S --
// P = S Lambda (second step), the subspace iterations S (S^T Q) (third) and
// T = Q^T S (fifth) -- and of the small dense steps; split-K reductions; the
// Cholesky factors of CholeskyQR (the QR of the fourth step); the symmetric
// eigensolver of the small SVD (sixth step); and the column sign convention
// of the lift (last step).
#include <float.h>
#include <type_traits>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "rpod_internal.cuh"

namespace rpod {

// ------------------------------------------------------------------------
// conversions
template <typename T> __device__ __forceinline__ T cvt(float x) { return T(x); }
template <typename T> __device__ __forceinline__ T cvt(double x) { return T(x); }
template <typename T> __device__ __forceinline__ T cvt(__nv_bfloat16 x) { return T(__bfloat162float(x)); }
template <typename T> __device__ __forceinline__ T cvt(__half x) { return T(__half2float(x)); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half cvt<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <> __device__ __forceinline__ __half cvt<__half>(double x) { return __double2half(x); }

// ------------------------------------------------------------------------
// The Box-Muller sketch entries (Philox4x64-10 in rpod_internal.cuh).

// Entry e = i + j m of Lambda is z0 (e even) or z1 (e odd) of the
// Box-Muller pair of Philox block e / 2: u1 = (w0 >> 11 + 1) 2^-53,
// u2 = (w1 >> 11) 2^-53, z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = ... sin.
// FP64 and FP32 sketches evaluate it in FP64.  A sketch stored in a 16-bit
// type keeps 8 or 11 mantissa bits, so it is evaluated in FP32 (GB300's FP64
// transcendental throughput made the FP64 form of this kernel 90 us for
// m l = 1.2e6): the integer words and uniforms are the same, ln u1 is taken
// as log1p(-(1 - u1)) for u1 >= 1/2 so that u1 near 1 keeps its relative
// accuracy, and the result differs from the FP64 value by a few FP32 ulps,
// which changes the 16-bit rounding only for values within that distance
// of a rounding boundary (the angle is reduced to within a quarter turn in
// integer arithmetic, so values near the zeros of sin and cos keep their
// relative accuracy).
template <typename T>
__device__ __forceinline__ void box_muller_store(uint64_t w0, uint64_t w1, T* a, T* b) {
  const uint64_t x0 = w0 >> 11, x1 = w1 >> 11;
  if constexpr (sizeof(T) == 2) {
    float lnu;
    if (x0 >= (1ull << 52)) {
      // 1 - u1 = (2^53 - 1 - x0) 2^-53, exact in FP64, accurate in FP32
      const float d = (float)((double)((1ull << 53) - 1ull - x0) * 0x1p-53);
      lnu = log1pf(-d);
    } else {
      lnu = logf((float)(((double)x0 + 1.0) * 0x1p-53));
    }
    const float r = sqrtf(-2.f * lnu);
    // angle pi t with t = x1 2^-52 in [0, 2): split t = q/2 + f exactly in
    // integers (|f| <= 1/4) so that sin and cos keep their relative accuracy
    // near their zeros, then rotate by the quarter turns q
    const int64_t q = (int64_t)((x1 + (1ull << 50)) >> 51);
    const float f = (float)((double)((int64_t)x1 - q * (int64_t)(1ull << 51)) * 0x1p-52);
    float s0, c0;
    sincospif(f, &s0, &c0);
    float sn, cs;
    switch (q & 3) {
      case 0: sn = s0; cs = c0; break;
      case 1: sn = c0; cs = -s0; break;
      case 2: sn = -s0; cs = -c0; break;
      default: sn = -c0; cs = s0; break;
    }
    *a = cvt<T>(r * cs);
    if (b) *b = cvt<T>(r * sn);
  } else {
    const double u1 = ((double)x0 + 1.0) * 0x1p-53;
    const double u2 = (double)x1 * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    *a = cvt<T>(r * cs);
    if (b) *b = cvt<T>(r * sn);
  }
}

template <typename T>
__global__ void k_sketch(uint64_t seed, uint64_t sid, int64_t m, int64_t total, T* Lam, int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t e0 = 2 * t;
  if (e0 >= total) return;
  uint64_t c[4] = {(uint64_t)t, sid, 0ull, 0ull};
  philox4x64_10(c, seed, 0ull);
  const int64_t j0 = e0 / m, i0 = e0 - j0 * m;
  const int64_t i1 = (i0 + 1 == m) ? 0 : i0 + 1, j1 = (i0 + 1 == m) ? j0 + 1 : j0;
  box_muller_store<T>(c[0], c[1], Lam + i0 + j0 * ld, e0 + 1 < total ? Lam + i1 + j1 * ld : nullptr);
}

template <typename T>
cudaError_t sketch(cudaStream_t st, uint64_t seed, uint64_t sid, int64_t m, int l, T* Lam, int64_t ld) {
  const int64_t total = m * (int64_t)l;
  const int64_t pairs = (total + 1) / 2;
  k_sketch<T><<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(seed, sid, m, total, Lam, ld); note_launch();
  return cudaGetLastError();
}
template cudaError_t sketch<double>(cudaStream_t, uint64_t, uint64_t, int64_t, int, double*, int64_t);
template cudaError_t sketch<float>(cudaStream_t, uint64_t, uint64_t, int64_t, int, float*, int64_t);
template cudaError_t sketch<__nv_bfloat16>(cudaStream_t, uint64_t, uint64_t, int64_t, int, __nv_bfloat16*, int64_t);
template cudaError_t sketch<__half>(cudaStream_t, uint64_t, uint64_t, int64_t, int, __half*, int64_t);

// ------------------------------------------------------------------------
// Generic SIMT GEMM.  16 x 16 threads; thread (ty, tx) owns rows ty + 16 r
// and columns tx + 16 c of the BM x BN tile (ty varies fastest so that a
// warp stores 16 consecutive rows of a column-major output).  The shared
// tiles hold each thread's TM rows (TN columns) contiguously, so the inner
// product step reads them with 16-byte loads: the unpermuted layout needed
// one shared-memory wavefront per FMA pair and capped the kernel near half
// the FP32 rate.
__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

template <int NV>
__device__ __forceinline__ void lds_vec(const float* p, float* v) {
  if constexpr (NV % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NV / 4; ++i) {
      const float4 q = reinterpret_cast<const float4*>(p)[i];
      v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = p[i];
  }
}
template <int NV>
__device__ __forceinline__ void lds_vec(const double* p, double* v) {
  if constexpr (NV % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
      const double2 q = reinterpret_cast<const double2*>(p)[i];
      v[2 * i] = q.x; v[2 * i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = p[i];
  }
}

template <typename TA, typename TB, typename TC, typename TO, int BM, int BN, int BK, bool AKC>
__global__ void __launch_bounds__(256, (sizeof(TC) == 4 && BM * BN >= 32 * 128) ? 2 : 1)
k_gemm(int64_t M, int64_t N, int64_t K, int64_t kchunk, const TA* __restrict__ A, int64_t lda,
       const TB* __restrict__ B, int64_t ldb, TO* __restrict__ C, int64_t ci, int64_t cj,
       int64_t csplit, unsigned* status, int check, int bkc) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int NA = BM * BK / 256, NB = BN * BK / 256;
  constexpr int PAD = 16 / (int)sizeof(TC);  // keeps every row 16-byte aligned
  __shared__ __align__(16) TC As[BK][BM + PAD];
  __shared__ __align__(16) TC Bs[BK][BN + PAD];
  const int tid = threadIdx.x, ty = tid & 15, tx = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = (K < kb + kchunk) ? K : kb + kchunk;
  TC acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = TC(0);
  bool bad = false;
  // The next k-tile is loaded into registers while the current one is
  // multiplied, so each tile costs one global-load latency, not one per
  // element.
  TC ra[NA], rb[NB];
  auto load_tiles = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int idx = tid + u * 256;
      int kk, ii;
      if (AKC) { kk = idx % BK; ii = idx / BK; } else { ii = idx % BM; kk = idx / BM; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      ra[u] = (gi < M && gk < ke) ? cvt<TC>(AKC ? A[gk + gi * lda] : A[gi + gk * lda]) : TC(0);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      // B(k, j) = B[k + j*ldb] (K-contiguous) or B[k*ldb + j] (N-contiguous)
      const int idx = tid + u * 256;
      const int kk = bkc ? idx % BK : idx / BN, jj = bkc ? idx / BK : idx % BN;
      const int64_t gj = j0 + jj, gk = k0 + kk;
      rb[u] = (gj < N && gk < ke) ? cvt<TC>(bkc ? B[gk + gj * ldb] : B[gk * ldb + gj]) : TC(0);
    }
  };
  if (kb < ke) load_tiles(kb);
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int idx = tid + u * 256;
      int kk, ii;
      if (AKC) { kk = idx % BK; ii = idx / BK; } else { ii = idx % BM; kk = idx / BM; }
      if (check && !finite_val(ra[u])) bad = true;
      As[kk][(ii & 15) * TM + (ii >> 4)] = ra[u];  // row ty + 16 r at ty * TM + r
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = tid + u * 256;
      const int kk = bkc ? idx % BK : idx / BN, jj = bkc ? idx / BK : idx % BN;
      Bs[kk][(jj & 15) * TN + (jj >> 4)] = rb[u];
    }
    __syncthreads();
    if (k0 + BK < ke) load_tiles(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TC a[TM], b[TN];
      lds_vec<TM>(&As[kk][ty * TM], a);
      lds_vec<TN>(&Bs[kk][tx * TN], b);
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  if (check && bad) atomicOr(status, ST_NONFINITE);
  TO* Cz = C + (int64_t)blockIdx.z * csplit;
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int64_t gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < M && gj < N) Cz[gi * ci + gj * cj] = cvt<TO>(acc[r][c]);
    }
}

// FP32 pass GEMM for the plain FP32 form's passes over S of Alg. 1
// (P = S Lambda and S Z: AKC false; S^T Q and T = Q^T S: AKC true; M or K in the
// hundreds of thousands, N = l > 64): C_z = sum_{k in split z} A(i, k) B(k, j)
// with B(k, j) = B[k + j*ldb] and A(i, k) = A[i + k*lda] (AKC false) or
// A[k + i*lda] (AKC true).  128 x 128 x 16 tiles, 256 threads; thread
// (tx, ty) = (tid % 16, tid / 16) owns rows {4 ty .. 4 ty + 3} and
// {64 + 4 ty ..} and the same pattern of columns, so each inner step reads
// its eight A and eight B values with four 16-byte shared loads and global
// tiles move as float4 (16-byte aligned operands, leading dimensions
// multiples of four).  The shared tiles are double-buffered: the next
// tile's global loads are in flight during the current tile's 1024 FMAs per
// thread and one barrier per tile separates the buffers.  `check` flags
// non-finite A entries in *status.
namespace {
constexpr int kSgBM = 128, kSgBN = 128, kSgBK = 16, kSgLd = 132;

template <bool AKC>
__global__ void __launch_bounds__(256, 2)
k_sgemm(int64_t M, int64_t N, int64_t K, int64_t kchunk, const float* __restrict__ A, int64_t lda,
        const float* __restrict__ B, int64_t ldb, float* __restrict__ C, int64_t ci, int64_t cj,
        int64_t csplit, unsigned* status, int check) {
  __shared__ __align__(16) float As[2][kSgBK][kSgLd];
  __shared__ __align__(16) float Bs[2][kSgBK][kSgLd];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * kSgBM, j0 = (int64_t)blockIdx.y * kSgBN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = (K < kb + kchunk) ? K : kb + kchunk;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  bool bad = false;
  float4 ra[2], rb[2];
  // A tile: AKC false -- float4 along i (32 per k row), AKC true -- float4
  // along k (4 per row i); B tile: float4 along k (4 per column j)
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u;
      float v[4];
      if (!AKC) {
        const int kk = idx >> 5, i4 = idx & 31;
        const int64_t gi = i0 + 4 * i4, gk = k0 + kk;
        const float* p = A + gi + gk * lda;
        if (gk < ke && gi + 3 < M) {
          const float4 q = *reinterpret_cast<const float4*>(p);
          v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) v[e] = (gk < ke && gi + e < M) ? p[e] : 0.f;
        }
      } else {
        const int k4 = idx & 3, ii = idx >> 2;
        const int64_t gi = i0 + ii, gk = k0 + 4 * k4;
        const float* p = A + gk + gi * lda;
        if (gi < M && gk + 3 < ke) {
          const float4 q = *reinterpret_cast<const float4*>(p);
          v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) v[e] = (gi < M && gk + e < ke) ? p[e] : 0.f;
        }
      }
      ra[u] = make_float4(v[0], v[1], v[2], v[3]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u;
      const int k4 = idx & 3, jj = idx >> 2;
      const int64_t gj = j0 + jj, gk = k0 + 4 * k4;
      const float* p = B + gk + gj * ldb;
      float v[4];
      if (gj < N && gk + 3 < ke) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (gj < N && gk + e < ke) ? p[e] : 0.f;
      }
      rb[u] = make_float4(v[0], v[1], v[2], v[3]);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u;
      if (check && !(isfinite(ra[u].x) && isfinite(ra[u].y) && isfinite(ra[u].z) && isfinite(ra[u].w)))
        bad = true;
      if (!AKC) {
        *reinterpret_cast<float4*>(&As[buf][idx >> 5][4 * (idx & 31)]) = ra[u];
      } else {
        const int k4 = idx & 3, ii = idx >> 2;
        As[buf][4 * k4 + 0][ii] = ra[u].x;
        As[buf][4 * k4 + 1][ii] = ra[u].y;
        As[buf][4 * k4 + 2][ii] = ra[u].z;
        As[buf][4 * k4 + 3][ii] = ra[u].w;
      }
      const int k4 = idx & 3, jj = idx >> 2;
      Bs[buf][4 * k4 + 0][jj] = rb[u].x;
      Bs[buf][4 * k4 + 1][jj] = rb[u].y;
      Bs[buf][4 * k4 + 2][jj] = rb[u].z;
      Bs[buf][4 * k4 + 3][jj] = rb[u].w;
    }
  };
  const int64_t ntiles = kb < ke ? (ke - kb + kSgBK - 1) / kSgBK : 0;
  if (ntiles > 0) {
    load(kb);
    store(0);
  }
  __syncthreads();
  for (int64_t t = 0; t < ntiles; ++t) {
    const int cur = (int)(t & 1);
    if (t + 1 < ntiles) load(kb + (t + 1) * kSgBK);
#pragma unroll
    for (int kk = 0; kk < kSgBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + 4 * tx]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    if (t + 1 < ntiles) store(cur ^ 1);
    __syncthreads();
  }
  if (check && bad) atomicOr(status, ST_NONFINITE);
  float* Cz = C + (int64_t)blockIdx.z * csplit;
  const bool vec = ci == 1 && (cj & 3) == 0 && ((uintptr_t)Cz & 15) == 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t gj = j0 + (c < 4 ? 4 * tx + c : 64 + 4 * tx + c - 4);
    if (gj >= N) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gi = i0 + 64 * h + 4 * ty;
      float* p = Cz + gi * ci + gj * cj;
      if (vec && gi + 3 < M) {
        *reinterpret_cast<float4*>(p) =
            make_float4(acc[4 * h][c], acc[4 * h + 1][c], acc[4 * h + 2][c], acc[4 * h + 3][c]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (gi + e < M) p[e * ci] = acc[4 * h + e][c];
      }
    }
  }
}
}  // namespace

// The FP32 pass GEMM when it applies (FP32 operands and output, a product
// over S, 16-byte aligned operands): returns false to leave the product to
// the generic kernel.
static bool launch_sgemm(cudaStream_t st, bool akc, int64_t M, int64_t N, int64_t K, int nsplit,
                         const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                         int64_t ci, int64_t cj, int64_t csplit, unsigned* status, bool check,
                         cudaError_t* err) {
  if (N <= 64 || M < 128 || K < 128 || M * K < ((int64_t)1 << 22)) return false;
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda & 3) || (ldb & 3)) return false;
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + kSgBK - 1) / kSgBK) * kSgBK;
  dim3 grid((unsigned)((M + kSgBM - 1) / kSgBM), (unsigned)((N + kSgBN - 1) / kSgBN),
            (unsigned)nsplit);
  if (akc)
    k_sgemm<true><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, C, ci, cj, csplit, status,
                                        check ? 1 : 0);
  else
    k_sgemm<false><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, C, ci, cj, csplit, status,
                                         check ? 1 : 0);
  note_launch();
  *err = cudaGetLastError();
  return true;
}

template <typename TA, typename TB, typename TC, typename TO, int BM, int BN, int BK>
static cudaError_t launch_gemm(cudaStream_t st, bool akc, bool bkc, int64_t M, int64_t N,
                               int64_t K, int nsplit, const TA* A, int64_t lda, const TB* B,
                               int64_t ldb, TO* C, int64_t ci, int64_t cj, int64_t csplit,
                               unsigned* status, bool check) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk <= 0) kchunk = BK;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)nsplit);
  if (akc)
    k_gemm<TA, TB, TC, TO, BM, BN, BK, true><<<grid, 256, 0, st>>>(
        M, N, K, kchunk, A, lda, B, ldb, C, ci, cj, csplit, status, check ? 1 : 0, bkc ? 1 : 0);
  else
    k_gemm<TA, TB, TC, TO, BM, BN, BK, false><<<grid, 256, 0, st>>>(
        M, N, K, kchunk, A, lda, B, ldb, C, ci, cj, csplit, status, check ? 1 : 0, bkc ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

template <typename TA, typename TB, typename TC, typename TO>
cudaError_t gemm_ex(cudaStream_t st, bool akc, bool bkc, int64_t M, int64_t N, int64_t K,
                    int nsplit, const TA* A, int64_t lda, const TB* B, int64_t ldb, TO* C,
                    int64_t ci, int64_t cj, int64_t csplit, unsigned* status, bool check) {
  if (nsplit < 1) nsplit = 1;
  if constexpr (std::is_same<TA, float>::value && std::is_same<TB, float>::value &&
                std::is_same<TC, float>::value && std::is_same<TO, float>::value) {
    cudaError_t e = cudaSuccess;
    if (bkc && launch_sgemm(st, akc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status,
                            check, &e))
      return e;
  }
  if (sizeof(TC) == 4) {
    if (N <= 32) return launch_gemm<TA, TB, TC, TO, 128, 32, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
    if (N <= 64) return launch_gemm<TA, TB, TC, TO, 128, 64, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
    // products with few 128 x 128 tiles (the m x l by l x l steps: 79 tiles
    // at m = 10000) on 64 x 128 tiles when that fills every SM once, else
    // 32 x 128 (one wave either way, two CTAs per SM allowed)
    const int64_t ny = (N + 127) / 128;
    if (((M + 127) / 128) * ny * nsplit < 2 * 152) {
      if (((M + 63) / 64) * ny * nsplit >= 152)
        return launch_gemm<TA, TB, TC, TO, 64, 128, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
      return launch_gemm<TA, TB, TC, TO, 32, 128, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
    }
    return launch_gemm<TA, TB, TC, TO, 128, 128, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
  } else {
    // small FP64 products (the l x l steps of the eigensolver) on 32 x 32
    // tiles: GB300 issues about two FP64 FMAs per clock per SM, so the tile
    // count, not the tile efficiency, sets their time
    if ((M <= 32 && N <= 32) || (M <= 128 && N <= 256))
      return launch_gemm<TA, TB, TC, TO, 32, 32, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
    if (N <= 32) return launch_gemm<TA, TB, TC, TO, 64, 32, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
    return launch_gemm<TA, TB, TC, TO, 64, 64, 16>(st, akc, bkc, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit, status, check);
  }
}

template <typename TA, typename TB, typename TC, typename TO>
cudaError_t gemm(cudaStream_t st, bool akc, int64_t M, int64_t N, int64_t K, int nsplit,
                 const TA* A, int64_t lda, const TB* B, int64_t ldb, TO* C, int64_t ci,
                 int64_t cj, int64_t csplit, unsigned* status, bool check) {
  return gemm_ex<TA, TB, TC, TO>(st, akc, true, M, N, K, nsplit, A, lda, B, ldb, C, ci, cj, csplit,
                                 status, check);
}

#define INST_GEMM(TA, TB, TC, TO)                                                          \
  template cudaError_t gemm<TA, TB, TC, TO>(cudaStream_t, bool, int64_t, int64_t, int64_t, \
                                            int, const TA*, int64_t, const TB*, int64_t,  \
                                            TO*, int64_t, int64_t, int64_t, unsigned*, bool); \
  template cudaError_t gemm_ex<TA, TB, TC, TO>(cudaStream_t, bool, bool, int64_t, int64_t,   \
                                               int64_t, int, const TA*, int64_t, const TB*, \
                                               int64_t, TO*, int64_t, int64_t, int64_t,      \
                                               unsigned*, bool);
INST_GEMM(double, double, double, double)
INST_GEMM(float, float, float, float)
INST_GEMM(float, float, float, double)
INST_GEMM(float, double, float, float)
INST_GEMM(double, double, double, float)
INST_GEMM(float, __nv_bfloat16, float, float)
#undef INST_GEMM

// ------------------------------------------------------------------------
// Deterministic split-K reduction out(i, j) = sum_z part[z][i + j M]: a
// block covers 32 consecutive elements with 8 z-slices (32 x 8 threads), each
// slice summed in z order with four accumulators, the slices combined in a
// fixed order.
// Partials are summed in their own precision: FP64 partials (Grams, the
// FP64 form) in FP64, FP32 partials in FP32 (GB300 issues FP64 adds at
// 1/64 of the FP32 rate, which made an FP64-accumulating FP32 reduction
// arithmetic-bound).
// Knuth's TwoSum: s + x = t + err exactly; used to carry the rounding error
// of FP32 sums in a second word (FP64 sums of many FP32 values would run at
// GB300's narrow FP64 rate, and so would the conversions to FP64).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

template <typename TP, typename TO>
__global__ void __launch_bounds__(256)
k_reduce(int64_t M, int64_t N, int nsplit, const TP* __restrict__ part, TO* __restrict__ out,
         int64_t oi, int64_t oj) {
  // FP64 partials: FP64 sums; FP32 partials: compensated FP32 sums (about
  // as accurate as FP64 ones for these counts), combined in FP64
  __shared__ double acc[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t idx = (int64_t)blockIdx.x * 32 + tx;
  const int64_t MN = M * N;
  double tot = 0.0;
  if (idx < MN) {
    if (sizeof(TP) == 8) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int z = ty;
      for (; z + 24 < nsplit; z += 32) {
        s0 += (double)part[(int64_t)z * MN + idx];
        s1 += (double)part[(int64_t)(z + 8) * MN + idx];
        s2 += (double)part[(int64_t)(z + 16) * MN + idx];
        s3 += (double)part[(int64_t)(z + 24) * MN + idx];
      }
      for (; z < nsplit; z += 8) s0 += (double)part[(int64_t)z * MN + idx];
      tot = (s0 + s1) + (s2 + s3);
    } else {
      float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
      int z = ty;
      for (; z + 8 < nsplit; z += 16) {
        two_sum_acc(s0, c0, (float)part[(int64_t)z * MN + idx]);
        two_sum_acc(s1, c1, (float)part[(int64_t)(z + 8) * MN + idx]);
      }
      for (; z < nsplit; z += 8) two_sum_acc(s0, c0, (float)part[(int64_t)z * MN + idx]);
      tot = ((double)s0 + (double)s1) + ((double)c0 + (double)c1);
    }
  }
  acc[ty][tx] = tot;
  __syncthreads();
  if (ty == 0 && idx < MN) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += acc[k][tx];
    const int64_t j = idx / M, i = idx - j * M;
    out[i * oi + j * oj] = (TO)t;
  }
}

// Up to 32 splits (the W-pass partials): each thread sums four consecutive
// elements over z in order (16-byte loads of FP32 partials when aligned,
// compensated FP32 sums), with eight splits in flight.
template <typename TP, typename TO>
__global__ void __launch_bounds__(256)
k_reduce_flat(int64_t M, int64_t N, int nsplit, const TP* __restrict__ part, TO* __restrict__ out,
              int64_t oi, int64_t oj, int vec) {
  const int64_t idx0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const int64_t MN = M * N;
  if (idx0 >= MN) return;
  TP s[4] = {TP(0), TP(0), TP(0), TP(0)};
  if (vec && idx0 + 4 <= MN) {
    // FP32 partials: compensated FP32 sums (TwoSum), the error words added
    // at the end
    const float* pf = reinterpret_cast<const float*>(part);
    float f[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    int z = 0;
    for (; z + 8 <= nsplit; z += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = *(const float4*)(pf + (int64_t)(z + u) * MN + idx0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        two_sum_acc(f[0], c[0], v[u].x);
        two_sum_acc(f[1], c[1], v[u].y);
        two_sum_acc(f[2], c[2], v[u].z);
        two_sum_acc(f[3], c[3], v[u].w);
      }
    }
    for (; z < nsplit; ++z) {
      const float4 v = *(const float4*)(pf + (int64_t)z * MN + idx0);
      two_sum_acc(f[0], c[0], v.x);
      two_sum_acc(f[1], c[1], v.y);
      two_sum_acc(f[2], c[2], v.z);
      two_sum_acc(f[3], c[3], v.w);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) s[e] = (TP)(f[e] + c[e]);
  } else {
    for (int z = 0; z < nsplit; ++z)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (idx0 + e < MN) s[e] += part[(int64_t)z * MN + idx0 + e];
  }
  // one division per thread; the four elements advance (i, j) in order
  int64_t j = idx0 / M, i = idx0 - j * M;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (idx0 + e < MN) out[i * oi + j * oj] = (TO)s[e];
    if (++i == M) { i = 0; ++j; }
  }
}

template <typename TP, typename TO>
cudaError_t reduce_splits(cudaStream_t st, int64_t M, int64_t N, int nsplit, const TP* part,
                          TO* out, int64_t oi, int64_t oj) {
  const int64_t MN = M * N;
  if (nsplit <= 32) {
    const int vec = (sizeof(TP) == 4 && (MN & 3) == 0 && ((uintptr_t)part & 15) == 0) ? 1 : 0;
    k_reduce_flat<TP, TO><<<(unsigned)((MN + 1023) / 1024), 256, 0, st>>>(M, N, nsplit, part, out, oi,
                                                                          oj, vec);
  }
  else
    k_reduce<TP, TO><<<(unsigned)((MN + 31) / 32), 256, 0, st>>>(M, N, nsplit, part, out, oi, oj);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t reduce_splits<double, double>(cudaStream_t, int64_t, int64_t, int, const double*, double*, int64_t, int64_t);
template cudaError_t reduce_splits<float, float>(cudaStream_t, int64_t, int64_t, int, const float*, float*, int64_t, int64_t);
template cudaError_t reduce_splits<double, float>(cudaStream_t, int64_t, int64_t, int, const double*, float*, int64_t, int64_t);

// ------------------------------------------------------------------------
// One-block FP64 Cholesky G = R^T R (right-looking, upper factor kept in
// place), with a rank-revealing pivot test: column j is dropped when its
// remaining pivot is <= tol * G_jj (or G_jj is negligible against the
// largest diagonal), then the in-place inverse of the upper factor (column
// by column, using the columns already inverted).  Dropped directions get
// zero rows and columns in X, so Q = Y X has zero columns there.
__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : -DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// The factorization runs in TF and the inverse in TI: FP64 for the FP64
// form; for the FP32-working forms the first CholeskyQR round factors in
// FP64 (its Gram carries the squared condition number) and later rounds,
// whose Gram is near the identity, in FP32, while the inverse is formed in
// FP32 (its rounding is removed by the next CholeskyQR round).  Column j of
// the factor lives in column j of the shared array (stride l + 1) and is
// overwritten by column j of the inverse.
//
// shift_coef > 0 (round 0 of the FP64 form's shifted CholeskyQR3, Fukaya,
// Kannan, Nakatsukasa, Yamamoto & Yanagisawa, SIAM J. Sci. Comput. 42, 2020):
// factors G + s I with s = shift_coef * trace(G) (shift_coef = 11 (rows l +
// l (l + 1)) u; the trace bounds ||Y||_2^2), so the factorization cannot
// break down and Q = Y R^{-1} has a condition number of order u^{-1/2}
// whatever that of Y; only exactly vanishing columns are dropped.
// flag_tiny (the rounds after a shifted one): a column of the
// near-orthonormal basis with squared norm below 1e-16 -- a direction of the
// sampled matrix below about 1e-13 of its norm, i.e. rounding noise -- raises
// the rank-deficiency warning but is kept and normalised, which completes the
// basis with orthonormal directions as Householder QR would.
template <typename TF, typename TI, typename TW>
__global__ void __launch_bounds__(256)
k_cholesky(int l, const double* __restrict__ G, double tol, double* __restrict__ Xout,
           TW* __restrict__ Xw, int ldxw, unsigned* status, double shift_coef, int flag_tiny) {
  extern __shared__ double sm[];
  const int ld = l + 1;
  TF* A = (TF*)sm;                                        // l x l, column-major, stride ld
  // offsets in elements of the shared array (an integer round trip of the
  // pointer would turn its accesses into generic ones)
  double* d0 = sm + (((size_t)l * ld * sizeof(TF) + 15) / 16) * 2;  // original diagonal
  TI* tmp = (TI*)(d0 + l);                                // column buffer
  __shared__ double red[32];
  __shared__ TF s_rinv;
  __shared__ int s_keep[kMaxL];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e0 = 0; e0 < l * l; e0 += 8 * nt) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt + tid;
      v[u] = e < l * l ? G[e] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt + tid, i = e % l, j = e / l;
      if (e < l * l && i <= j) A[i + j * ld] = (TF)v[u];
    }
  }
  double dm = 0.0;
  for (int j = tid; j < l; j += nt) { d0[j] = G[j + j * l]; dm = fmax(dm, d0[j]); }
  const double gmax = block_max(dm, red);   // also orders the loads above
  if (shift_coef > 0.0) {
    double tr = 0.0;
    for (int j = tid; j < l; j += nt) tr += d0[j];
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    __shared__ double s_tr[8];
    if ((tid & 31) == 0) s_tr[tid >> 5] = tr;
    __syncthreads();
    tr = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) tr += s_tr[w];
    const double shift = shift_coef * tr;
    for (int j = tid; j < l; j += nt)
      if (d0[j] > 1e-300) A[j + j * ld] += (TF)shift;
    __syncthreads();
  }
  int ndropped = 0, ntiny = 0;
  const int cb = tid & 127, rg = tid >> 7, ng = nt >> 7;
  for (int j = 0; j < l; ++j) {
    if (tid == 0) {
      const double d = (double)A[j + j * ld];
      const bool keep = (d0[j] > 1e-300) && (d0[j] > 1e-30 * gmax) && (d > tol * d0[j]);
      s_keep[j] = keep ? 1 : 0;
      const TF r = keep ? (TF)sqrt(d) : (TF)0;
      s_rinv = keep ? (TF)1 / r : (TF)0;
      A[j + j * ld] = r;
    }
    __syncthreads();
    const TF rinv = s_rinv;
    if (!s_keep[j]) ++ndropped;
    else if (flag_tiny && d0[j] < 1e-16) ++ntiny;
    for (int c = j + 1 + tid; c < l; c += nt) A[j + c * ld] *= rinv;
    __syncthreads();
    // trailing update of the upper triangle: column b = j + 1 + cb, rows a <= b
    const int b = j + 1 + cb;
    if (b < l) {
      const TF rb = A[j + b * ld];
      for (int a = j + 1 + rg; a <= b; a += ng) A[a + b * ld] -= A[j + a * ld] * rb;
    }
    __syncthreads();
  }
  // inverse of the upper factor, column by column, in place
  for (int j = 0; j < l; ++j) {
    const bool keep = s_keep[j] != 0;
    for (int i = tid; i < j; i += nt) tmp[i] = keep ? (TI)A[i + j * ld] : (TI)0;
    __syncthreads();
    if (keep) {
      const TI ajj = (TI)1 / (TI)A[j + j * ld];
      for (int i = tid; i < j; i += nt) {
        TI s = 0;
        for (int t2 = i; t2 < j; ++t2) s += (TI)A[i + t2 * ld] * tmp[t2];
        A[i + j * ld] = (TF)(-ajj * s);
      }
      __syncthreads();
      if (tid == 0) A[j + j * ld] = (TF)ajj;
    } else {
      for (int i = tid; i <= j; i += nt) A[i + j * ld] = (TF)0;
    }
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += nt) {
    const int i = e % l, j = e / l;
    const double v = (i <= j) ? (double)A[i + j * ld] : 0.0;
    Xout[e] = v;
    Xw[i + (int64_t)j * ldxw] = (TW)v;
  }
  if (tid == 0 && ndropped > 0) atomicOr(status, ndropped == l ? (ST_RANK_DEF | ST_BREAKDOWN) : ST_RANK_DEF);
  if (tid == 0 && ntiny > 0) atomicOr(status, ST_RANK_DEF);
}

template <typename TF, typename TI, typename TW>
static cudaError_t launch_cholesky(cudaStream_t st, int l, const double* G, double tol, double* X,
                                   TW* Xw, int ldxw, unsigned* status, double shift_coef,
                                   int flag_tiny) {
  const size_t sm = (size_t)l * (l + 1) * sizeof(TF) + 16 + (size_t)l * (sizeof(double) + sizeof(TI));
  prepare_kernels();
  k_cholesky<TF, TI, TW><<<1, 256, sm, st>>>(l, G, tol, X, Xw, ldxw, status, shift_coef, flag_tiny);
  note_launch();
  return cudaGetLastError();
}

// Blocked FP32 CholeskyQR step (l <= 128): A = R^T R with R upper, in 8 x 8
// blocks.  The 256 threads form a 16 x 16 grid; thread (ty, tx) holds block
// (ty, tx) of the zero-padded Gram matrix in registers.  Block step k: the
// owner of diagonal block (k, k) factors it (pivot test per column), the
// owners of row block k solve R_kj = R_kk^{-T} A_kj, and the owners of the
// upper trailing blocks apply A_ij -= R_ki^T R_kj: two barriers per block step
// instead of per column.  The inverse X = R^{-1} comes from the blocked
// column sweep X(:, k) = W(:, k) R_kk^{-1}, W(:, c) -= X(:, k) R_kc, W = I,
// run one block step behind the factorization in the same barrier
// intervals (15 block steps in all for l = 120, not 30).  Pivot
// semantics as k_cholesky: a column whose pivot falls to tol times its
// original diagonal is dropped (zero row of R, zero column of X); with a
// gate word, a pivot below ill_tol of it raises the FP64 gate.
// Eight consecutive values to a 16-byte aligned address as 16-byte stores.
__device__ __forceinline__ void store8(float* p, const float* v) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void store8(double* p, const float* v) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    reinterpret_cast<double2*>(p)[i] = make_double2((double)v[2 * i], (double)v[2 * i + 1]);
}

constexpr int kBlkLd = 132;  // row stride of the shared R (16-byte aligned rows)
constexpr size_t kBlkSmem = (size_t)(128 * kBlkLd + 128 * 8) * sizeof(float);

template <typename TW>
__global__ void __launch_bounds__(256)
k_cholesky_blk(int l, const float* __restrict__ G, float tol, int* gate, float ill_tol,
               double* __restrict__ Xout,
               TW* __restrict__ Xw, int ldxw, unsigned* status) {
  extern __shared__ __align__(16) float s_R[];  // [128][kBlkLd]: G, then R rows, then X
  float* s_X = s_R + 128 * kBlkLd;              // [128][8]: one block column of X
  __shared__ float s_d0[128];
  __shared__ float s_rd[128];
  __shared__ float s_ri[128];  // 1 / R_jj (0 for a dropped column)
  __shared__ int s_keep[128];
  __shared__ int s_ill;
  __shared__ double red[32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = ty * 8, c0 = tx * 8;
  const int nb = (l + 7) >> 3;
  for (int e0 = 0; e0 < 128 * 128; e0 += 256 * 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + u * 256 + tid, i = e & 127, j = e >> 7;
      // upper triangle of G only (the exact-product Gram leaves the lower one unset)
      v[u] = (i < l && j < l) ? G[min(i, j) + max(i, j) * l] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + u * 256 + tid, i = e & 127, j = e >> 7;
      s_R[j * kBlkLd + i] = v[u];  // G is symmetric: row j = column j
    }
  }
  double dm = 0.0;
  if (tid < 128) {
    const float g = tid < l ? G[tid + tid * l] : 0.f;
    s_d0[tid] = g;
    s_rd[tid] = 0.f;
    s_ri[tid] = 0.f;
    s_keep[tid] = 0;
    dm = g;
  }
  if (tid == 0) s_ill = 0;
  const float gmax = (float)block_max(dm, red);  // barrier: s_R, s_d0 visible
  float A[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) A[a][b] = s_R[(r0 + a) * kBlkLd + c0 + b];
  __syncthreads();
  // One register block per thread: thread (ty, tx) holds block (ty, tx) of
  // A until block step ty forms row block ty of R, then block (ty, tx) of W
  // (zero; the identity for ty = tx), which becomes block (ty, tx) of
  // X = R^{-1} at block step tx.  The inverse runs one block step behind the
  // factorization in the same barrier intervals: step k of X needs R_kk and
  // R_kc (c > k), both known after factorization step k.
  for (int k = 0; k < nb; ++k) {
    const int k0 = 8 * k;
    if (ty == k && tx == k) {
      // diagonal block: unblocked right-looking factorization in registers
      int ill = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = k0 + t;
        const float d = A[t][t], d0 = s_d0[j];
        const bool keep = (j < l) && (d0 > 1e-30f) && (d0 > 1e-30f * gmax) && (d > tol * d0);
        if (j < l && d < ill_tol * d0) ill = 1;
        const float rinv = keep ? rsqrtf(d) : 0.f;
        const float rd = d * rinv;
#pragma unroll
        for (int b = 0; b < 8; ++b) A[t][b] = (b > t) ? A[t][b] * rinv : (b == t ? rd : 0.f);
#pragma unroll
        for (int a = t + 1; a < 8; ++a)
#pragma unroll
          for (int b = t + 1; b < 8; ++b) A[a][b] -= A[t][a] * A[t][b];
        s_keep[j] = keep ? 1 : 0;
        s_rd[j] = rd;
        s_ri[j] = rinv;
      }
      if (ill) s_ill = 1;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) s_R[(k0 + a) * kBlkLd + k0 + b] = (b >= a) ? A[a][b] : 0.f;
    } else if (k > 0 && ty < k && tx >= k && tx < nb) {
      // inverse, second half of step k - 1: W(:, c) -= X(:, k-1) R_{k-1,c}
      const int j0 = k0 - 8;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float4* rk4 = (const float4*)&s_R[(j0 + s) * kBlkLd + c0];
        const float4 q0 = rk4[0], q1 = rk4[1];
        const float rk[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        float xs[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) xs[a] = s_X[(r0 + a) * 8 + s];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) A[a][b] -= xs[a] * rk[b];
      }
    }
    __syncthreads();
    if (ty == k && tx > k && tx < nb) {
      // row block k: R_kj = R_kk^{-T} A_kj, forward substitution over rows t
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float rinv = s_ri[k0 + t];
#pragma unroll
        for (int s = 0; s < t; ++s) {
          const float rst = s_R[(k0 + s) * kBlkLd + k0 + t];
#pragma unroll
          for (int b = 0; b < 8; ++b) A[t][b] -= rst * A[s][b];
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) A[t][b] *= rinv;
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float4* dst = (float4*)&s_R[(k0 + a) * kBlkLd + c0];
        dst[0] = make_float4(A[a][0], A[a][1], A[a][2], A[a][3]);
        dst[1] = make_float4(A[a][4], A[a][5], A[a][6], A[a][7]);
      }
      // this block of R is in shared memory: the registers become W (zero
      // off the diagonal)
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) A[a][b] = 0.f;
    } else if (tx == k && ty <= k) {
      // inverse, first half of step k: X(:, k) = W(:, k) R_kk^{-1} (rows of
      // block column k above the diagonal and the diagonal block, whose W
      // is the identity)
      if (ty == k) {
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) A[a][b] = (a == b) ? 1.f : 0.f;
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float rinv = s_ri[k0 + b];
#pragma unroll
        for (int s = 0; s < b; ++s) {
          const float rsb = s_R[(k0 + s) * kBlkLd + k0 + b];
#pragma unroll
          for (int a = 0; a < 8; ++a) A[a][b] -= A[a][s] * rsb;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) A[a][b] *= rinv;
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float4* dst = (float4*)&s_X[(r0 + a) * 8];
        dst[0] = make_float4(A[a][0], A[a][1], A[a][2], A[a][3]);
        dst[1] = make_float4(A[a][4], A[a][5], A[a][6], A[a][7]);
      }
    }
    __syncthreads();
    if (ty > k && tx >= ty && tx < nb) {
      // upper trailing blocks: A_ij -= R_ki^T R_kj
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float4* ri4 = (const float4*)&s_R[(k0 + s) * kBlkLd + r0];
        const float4* rj4 = (const float4*)&s_R[(k0 + s) * kBlkLd + c0];
        const float4 i0 = ri4[0], i1 = ri4[1], j0 = rj4[0], j1 = rj4[1];
        const float ri[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
        const float rj[8] = {j0.x, j0.y, j0.z, j0.w, j1.x, j1.y, j1.z, j1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) A[a][b] -= ri[a] * rj[b];
      }
    }
    // block step k + 1 writes rows k0 + 8.. of s_R and reads s_X after its
    // first barrier only; no barrier needed here
  }
  __syncthreads();
  float (&W)[8][8] = A;
  // X straight from the register blocks: column c0 + b, rows r0 .. r0 + 7,
  // as 16-byte stores (zero below the diagonal); few wide store requests
  // instead of one request per 32 elements
  const bool vec = ((uintptr_t)Xw & 15) == 0 && ((size_t)ldxw * sizeof(TW)) % 16 == 0 &&
                   (!Xout || ((l & 1) == 0 && ((uintptr_t)Xout & 15) == 0));
  if (r0 < l && c0 < l) {
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int j = c0 + b;
      if (j < l) {
        float col[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) col[a] = (r0 + a <= j) ? W[a][b] : 0.f;
        if (vec && r0 + 8 <= l) {
          store8(Xw + r0 + (int64_t)j * ldxw, col);
          if (Xout) store8(Xout + r0 + (int64_t)j * l, col);
        } else {
#pragma unroll
          for (int a = 0; a < 8; ++a)
            if (r0 + a < l) {
              Xw[r0 + a + (int64_t)j * ldxw] = (TW)col[a];
              if (Xout) Xout[r0 + a + (int64_t)j * l] = (double)col[a];
            }
        }
      }
    }
  }
  if (tid == 0) {
    int ndropped = 0;
    for (int j = 0; j < l; ++j) ndropped += s_keep[j] ? 0 : 1;
    if (gate && s_ill) *gate = 1;
    if (ndropped > 0 && !(gate && s_ill))
      atomicOr(status, ndropped == l ? (ST_RANK_DEF | ST_BREAKDOWN) : ST_RANK_DEF);
  }
}

// CholeskyQR factor (the QR of Alg. 1's fourth step) in FP64, run only when
// the FP32 attempt raised the gate; its dynamic shared memory for an l x l
// Gram matrix.
constexpr size_t gated_smem_bytes(int l) {
  return (size_t)l * (l + 1) * (sizeof(double) + sizeof(float)) + (size_t)l * (sizeof(double) + sizeof(float));
}
template <typename TW>
__global__ void __launch_bounds__(256)
k_cholesky64_gated(int l, const double* __restrict__ G, double tol, int* gate,
                   double* __restrict__ Xout, TW* __restrict__ Xw, int ldxw, unsigned* status,
                   double* __restrict__ part, int nsplit, unsigned* ticket);

// Gram partials of an FP32 matrix with exact products, run only when the
// gate is raised (an FP32 Gram cannot resolve pivots below about 1e-9 of the
// column norms).  GB300 issues FP64 arithmetic at 1/64 of the FP32 rate, so
// the exact sums are kept as unevaluated FP32 pairs (double-float): each
// product a*b is split exactly into p = fl(a*b) and e = fma(a, b, -p), p is
// added to the high word with Knuth's TwoSum and the rounding error plus e
// go to the low word (Dekker, Numer. Math. 18, 1971), relative error of
// order rows * 2^-46.  Only blocks on or above the diagonal are formed (the
// factorization reads the upper triangle): thread t < 136 owns upper block
// (bi, bj) of a 16 x 16 grid of B x B blocks, 16 B >= l.
template <int B>
__global__ void __launch_bounds__(256)
k_gram_df_gated(int64_t rows, int l, const float* __restrict__ Y, int64_t ldy, int64_t chunk,
                double* __restrict__ part, const int* gate) {
  __shared__ int s_go;
  if (threadIdx.x == 0) s_go = *gate;
  __syncthreads();
  if (!s_go) return;
  constexpr int BR = 32, W = 16 * B;
  __shared__ __align__(16) float Ys[BR][W + 4];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = (r0 + chunk < rows) ? r0 + chunk : rows;
  int bi = 0, bj = 0;
  const bool active = tid < 136;
  if (active) {
    int rem = tid;
    while (rem >= 16 - bi) { rem -= 16 - bi; ++bi; }
    bj = bi + rem;
  }
  const bool work = active && bi * B < l && bj * B < l;
  float sh[B][B], sl[B][B];
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int b = 0; b < B; ++b) { sh[a][b] = 0.f; sl[a][b] = 0.f; }
  for (int64_t rb = r0; rb < r1; rb += BR) {
    constexpr int NL = BR * W / 256;  // loads per thread, in batches of 8 in flight
#pragma unroll
    for (int u0 = 0; u0 < NL; u0 += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + (u0 + u) * 256, rr = e % BR, c = e / BR;
        const int64_t r = rb + rr;
        v[u] = (u0 + u < NL && c < l && r < r1) ? Y[r + (int64_t)c * ldy] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + (u0 + u) * 256;
        if (u0 + u < NL) Ys[e % BR][e / BR] = v[u];
      }
    }
    __syncthreads();
    if (work) {
      for (int rr = 0; rr < BR; ++rr) {
        float av[B], bv[B];
#pragma unroll
        for (int a = 0; a < B; ++a) av[a] = Ys[rr][bi * B + a];
#pragma unroll
        for (int b = 0; b < B; ++b) bv[b] = Ys[rr][bj * B + b];
#pragma unroll
        for (int a = 0; a < B; ++a)
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const float p = av[a] * bv[b];
            const float e = fmaf(av[a], bv[b], -p);
            const float t = sh[a][b] + p;
            const float bp = t - sh[a][b];
            const float err = (sh[a][b] - (t - bp)) + (p - bp);
            sh[a][b] = t;
            sl[a][b] += err + e;
          }
      }
    }
    __syncthreads();
  }
  if (!work) return;
  double* pz = part + (int64_t)blockIdx.x * l * l;
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = bi * B + a, j = bj * B + b;
      if (i < l && j < l) pz[i + j * l] = (double)sh[a][b] + (double)sl[a][b];
    }
}

template <typename TW>
cudaError_t cholesky(cudaStream_t st, int l, const void* Gv, double tol, int round, double* X,
                     TW* Xw, int ldxw, unsigned* status, const float* Y, int64_t rows,
                     double* part, int nsplit, int64_t ldy, double shift_coef, bool flag_tiny,
                     bool gate_second) {
  if (ldy == 0) ldy = rows;
  if (sizeof(TW) == 8)
    return launch_cholesky<double, double, TW>(st, l, (const double*)Gv, tol, X, Xw, ldxw, status,
                                               shift_coef, flag_tiny ? 1 : 0);
  const float* G = (const float*)Gv;
  // the gate word sits next to the status word (same 256-byte status block)
  int* gate = (int*)(status + 2);
  prepare_kernels();
  // round 0: the gate rises where a pivot shows a condition number beyond
  // FP32 reach; second round (gate_second): where the first round's basis
  // Q1 has kappa(Q1)^2 > 2 (a pivot below half its column's norm) -- the
  // FP32 Gram and factorization of Q1 leave an orthogonality error of about
  // sqrt(rows) * u * kappa(Q1)^2, the FP64 ones about u * kappa(Q1) (the
  // rounding of the apply).  Only a first round that took the FP64 path
  // on a sampled matrix near FP32's noise level leaves such a Q1.
  const bool gated = round == 0 || (round == 1 && gate_second);
  k_cholesky_blk<TW><<<1, 256, kBlkSmem, st>>>(l, G, (float)tol, gated ? gate : nullptr,
                                               round == 0 ? 1e-4f : 0.5f, X, Xw, ldxw, status);
  note_launch();
  if (!gated) return cudaGetLastError();
  // the FP64 refactorization needs the exact-product Gram of Y
  if (!(Y && part && nsplit > 0)) return cudaGetLastError();
  double* gp = nullptr;
  if (Y && part && nsplit > 0) {
    int64_t chunk = (rows + nsplit - 1) / nsplit;
    chunk = (chunk + 31) / 32 * 32;
    if (l <= 64)
      k_gram_df_gated<4><<<nsplit, 256, 0, st>>>(rows, l, Y, ldy, chunk, part, gate);
    else
      k_gram_df_gated<8><<<nsplit, 256, 0, st>>>(rows, l, Y, ldy, chunk, part, gate);
    note_launch();
    gp = part;
  }
  const size_t sm64 = gated_smem_bytes(l);
  const unsigned grid = gp && nsplit > 1 ? (unsigned)(((int64_t)l * l + 63) / 64) : 1u;
  k_cholesky64_gated<TW><<<grid, 256, sm64, st>>>(l, nullptr, 1e-13, gate, X, Xw, ldxw, status, gp,
                                                  nsplit, status + 9);
  note_launch();
  return cudaGetLastError();
}

template <typename TW>
__global__ void __launch_bounds__(256)
k_cholesky64_gated(int l, const double* __restrict__ G, double tol, int* gate,
                   double* __restrict__ Xout, TW* __restrict__ Xw, int ldxw, unsigned* status,
                   double* __restrict__ part, int nsplit, unsigned* ticket) {
  __shared__ int s_go, s_last;
  __shared__ double s_zs[8][32];
  if (threadIdx.x == 0) s_go = *gate;
  __syncthreads();
  if (!s_go) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (part && nsplit > 1) {
    // The Gram matrix is the sum of the nsplit exact-product partials of
    // k_gram_df_gated (element e = i + j*l, i <= j, of split z at
    // part[z*l*l + e]).  GB300 adds about two FP64 numbers per clock per
    // SM, so the sums are spread over the grid: CTA b sums elements
    // [64 b, 64 b + 64) into split 0, warps w and w + 4k (k < 4) take the
    // splits z = k, k + 4, ... of one 32-element group, and their four sums
    // are added in warp order; the last CTA to finish (a ticket counter,
    // reset for the next call) factors.  The result does not depend on
    // the CTAs' timing.
    const int lane = tid & 31, w = tid >> 5, grp = w >> 2, wz = w & 3;
    const int64_t nel = (int64_t)l * l;
    const int64_t e = (int64_t)blockIdx.x * 64 + grp * 32 + lane;
    const bool up = e < nel && (e % l) <= (e / l);
    double zs = 0.0;
    if (up) {
#pragma unroll 4
      for (int z = wz; z < nsplit; z += 4) zs += part[(int64_t)z * nel + e];
    }
    s_zs[w][lane] = zs;
    __syncthreads();
    if (wz == 0 && up) {
      part[e] = ((s_zs[w][lane] + s_zs[w + 1][lane]) + s_zs[w + 2][lane]) + s_zs[w + 3][lane];
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid == 0) *ticket = 0u;
  }
  // FP64 factorization of the Gram matrix, then the FP32 inverse of the
  // factor.  Dynamic shared memory: A (l x ld doubles), d0 (l doubles), Rf
  // (l x ld floats), rf (l floats); Xf (l x ldx floats) reuses A once R is
  // in Rf.
  extern __shared__ double sm[];
  const int ld = l + 1, ldx = (l + 1) & ~1;
  double* A = sm;
  double* d0 = sm + (size_t)l * ld;
  float* Rf = (float*)(d0 + l);
  float* rf = Rf + (size_t)l * ld;
  float* Xf = (float*)sm;
  __shared__ double red[32];
  __shared__ double s_ri[kMaxL];
  __shared__ int s_keep[kMaxL];
  for (int e = tid; e < l * l; e += nt) {
    const int i = e % l, j = e / l;
    if (i > j) continue;
    // split 0 holds the sums (written by other CTAs: read through L2)
    const double g = part ? (nsplit > 1 ? __ldcg(part + e) : part[e]) : G[e];
    A[i + j * ld] = g;
    if (i == j) d0[j] = g;
  }
  __syncthreads();
  double dm = 0.0;
  for (int j = tid; j < l; j += nt) dm = fmax(dm, d0[j]);
  const double gmax = block_max(dm, red);
  // Right-looking factorization with unscaled rows: after step j, row j
  // holds r_jj times row j of R, the trailing block loses the outer product
  // of that row with itself times 1/r_jj^2, and the rows are scaled once at
  // the end.  Thread 0 makes the last update of the next diagonal entry in
  // each step and takes that pivot's decision and square root while the
  // other threads finish the step, so a column costs one barrier.
  const int cb = tid & 127, rg = tid >> 7, ng = nt >> 7;
  auto pivot = [&](int j, double d) {
    const bool keep = (d0[j] > 1e-300) && (d0[j] > 1e-30 * gmax) && (d > 1e-13 * d0[j]);
    const double ri = keep ? rsqrt(d) : 0.0;
    s_keep[j] = keep ? 1 : 0;
    s_ri[j] = ri;
    A[j + j * ld] = keep ? d * ri : 0.0;
  };
  if (tid == 0) pivot(0, A[0]);
  __syncthreads();
  for (int j = 0; j + 1 < l; ++j) {
    const double ri = s_ri[j];
    const int b = j + 1 + cb;
    if (b < l) {
      const double rb = A[j + b * ld] * (ri * ri);
      for (int a = j + 1 + rg; a <= b; a += ng) A[a + b * ld] -= A[j + a * ld] * rb;
    }
    // thread 0 (b = j + 1, a = j + 1) has just updated the next pivot
    if (tid == 0) pivot(j + 1, A[(j + 1) + (j + 1) * ld]);
    __syncthreads();
  }
  // R with scaled rows (a dropped row is zero), in FP32, and 1 / r_jj
  for (int e = tid; e < l * l; e += nt) {
    const int i = e % l, j = e / l;
    if (i > j) continue;
    const double v = (i == j) ? A[i + j * ld] : A[i + j * ld] * s_ri[i];
    Rf[i + j * ld] = (float)v;
  }
  for (int j = tid; j < l; j += nt) rf[j] = s_keep[j] ? 1.f / (float)A[j + j * ld] : 0.f;
  __syncthreads();
  // X = R^{-1} by rows, without barriers: thread i forms row i (stored
  // contiguously, Xf[i * ldx + j]), X_ii = 1 / r_ii and, for j > i,
  // X_ij = -(sum_{t=i}^{j-1} X_it R_tj) / r_jj.  A dropped direction j gives
  // a zero column j and, through X_jj = 0, a zero row j.
  if (tid < l) {
    const int i = tid;
    float* xr = Xf + (size_t)i * ldx;
    xr[i] = rf[i];
    for (int j = i + 1; j < l; ++j) {
      const float* rc = Rf + (size_t)j * ld;
      float s0 = 0.f, s1 = 0.f;
      int t = i;
      for (; t + 1 < j; t += 2) {
        s0 = fmaf(xr[t], rc[t], s0);
        s1 = fmaf(xr[t + 1], rc[t + 1], s1);
      }
      if (t < j) s0 = fmaf(xr[t], rc[t], s0);
      xr[j] = -rf[j] * (s0 + s1);
    }
  }
  __syncthreads();
  for (int e = tid; e < l * l; e += nt) {
    const int i = e % l, j = e / l;
    const float v = (i <= j) ? Xf[(size_t)i * ldx + j] : 0.f;
    if (Xout) Xout[e] = (double)v;
    Xw[i + (int64_t)j * ldxw] = (TW)v;
  }
  if (tid == 0) {
    int ndropped = 0;
    for (int j = 0; j < l; ++j) ndropped += s_keep[j] ? 0 : 1;
    *gate = 0;
    if (ndropped > 0) atomicOr(status, ndropped == l ? (ST_RANK_DEF | ST_BREAKDOWN) : ST_RANK_DEF);
  }
  (void)tol;
}
template cudaError_t cholesky<double>(cudaStream_t, int, const void*, double, int, double*, double*, int, unsigned*, const float*, int64_t, double*, int, int64_t, double, bool, bool);
template cudaError_t cholesky<float>(cudaStream_t, int, const void*, double, int, double*, float*, int, unsigned*, const float*, int64_t, double*, int, int64_t, double, bool, bool);

// ------------------------------------------------------------------------
// Symmetric eigensolver for the small SVD.  T T^T = Uhat Sigma^2 Uhat^T, so
// the left singular vectors and values of T come from the eigenpairs of its
// l x l Gram matrix.
//
// Stage 1: an FP32 starting basis from the tridiagonal reduction of the
// Gram matrix (tridiag_eig32, rpod_eig.cu).  Stage 2: FP64 iterative
// refinement of the eigenvectors (Ogita & Aishima, "Iterative refinement
// for symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math. 35,
// 2018): with R = I - X^T X and S = X^T A X, lambda_i = S_ii / (1 - R_ii),
// E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) when
// |lambda_i - lambda_j| > delta, else R_ij / 2, E_ii = R_ii / 2,
// X <- X + X E; each pass squares the error.

// Ogita-Aishima pass, part 1: per block, FP64 partial sums over its columns
// of ||I - X^T X||_F^2, ||X^T A X - diag(lambda)||_F^2 and ||A||_F^2
// (lambda_i = (X^T A X)_ii / (X^T X)_ii); the last block to finish (a ticket
// counter, reset for the next call) adds the partials in block order -- the
// result does not depend on the blocks' timing -- and writes the separation
// threshold delta and lambda.  XS = [X^T X | X^T A X] (l x 2l, ld l).
__global__ void __launch_bounds__(256)
k_oa_norm(int l, const double* __restrict__ XS, const double* __restrict__ A,
          double* __restrict__ part3, unsigned* __restrict__ ticket, double* __restrict__ lam,
          double* __restrict__ delta) {
  const double* XtX = XS;
  const double* S = XS + (size_t)l * l;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double sr = 0.0, so = 0.0, sa = 0.0;
  for (int j = blockIdx.x; j < l; j += gridDim.x) {
    const double lj = S[j + (size_t)j * l] / XtX[j + (size_t)j * l];
    for (int i = tid; i < l; i += blockDim.x) {
      const size_t e = i + (size_t)j * l;
      const double rij = (i == j ? 1.0 : 0.0) - XtX[e];
      const double sij = S[e] - (i == j ? lj : 0.0);
      sr = fma(rij, rij, sr);
      so = fma(sij, sij, so);
      sa = fma(A[e], A[e], sa);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    so += __shfl_xor_sync(0xffffffffu, so, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  __shared__ double rs[3][8];
  __shared__ bool s_last;
  if (lane == 0) { rs[0][w] = sr; rs[1][w] = so; rs[2][w] = sa; }
  __syncthreads();
  if (tid == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a0 += rs[0][k]; a1 += rs[1][k]; a2 += rs[2][k]; }
    part3[blockIdx.x] = a0;
    part3[gridDim.x + blockIdx.x] = a1;
    part3[2 * gridDim.x + blockIdx.x] = a2;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the partials in parallel (L2 loads: other blocks wrote them), then
  // added by one thread in block order
  __shared__ double s_p[3][64];
  for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
    s_p[0][b] = __ldcg(part3 + b);
    s_p[1][b] = __ldcg(part3 + gridDim.x + b);
    s_p[2][b] = __ldcg(part3 + 2 * gridDim.x + b);
  }
  __syncthreads();
  if (tid == 0) {
    double r = 0.0, o = 0.0, g = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      r += s_p[0][b];
      o += s_p[1][b];
      g += s_p[2][b];
    }
    const double normA = sqrt(g);
    // floor: once the passes have converged, delta falls to the rounding
    // level, where the Rayleigh quotients of a multiple eigenvalue differ by
    // rounding alone; without the floor such a pair counts as separated and
    // E divides by that difference.  The Gram comes from FP32 products of
    // the FP32 matrix T and the start from FP32 arithmetic: neither
    // determines the eigenvectors of a pair closer than about
    // 100 u_32 ||A|| (u_32 = 2^-24), whose start keeps an arbitrary rotation
    // within the pair -- a pass that took such a pair as separated would
    // apply an O(1) first-order rotation and lose orthogonality, so the pair
    // keeps the orthonormalizing update (its span is still refined)
    const double floor64 = 64.0 * DBL_EPSILON * (double)l * normA;
    const double floor32 = 100.0 * (double)(FLT_EPSILON / 2) * normA;
    *delta = fmax(2.0 * (sqrt(o) + normA * sqrt(r)), fmax(floor64, floor32));
    *ticket = 0u;
  }
  for (int i = tid; i < l; i += blockDim.x)
    lam[i] = S[i + (size_t)i * l] / XtX[i + (size_t)i * l];
}

// Ogita-Aishima pass, part 2: I + E from XS, lambda and delta, so that the
// next basis is X (I + E); the FP64 divisions spread over the grid.
__global__ void __launch_bounds__(256)
k_oa_e(int l, const double* __restrict__ XS, const double* __restrict__ lam,
       const double* __restrict__ delta, double* __restrict__ E) {
  extern __shared__ double lm[];
  const double* XtX = XS;
  const double* S = XS + (size_t)l * l;
  for (int i = threadIdx.x; i < l; i += blockDim.x) lm[i] = lam[i];
  __syncthreads();
  const double dl = *delta;
  for (int j = blockIdx.x; j < l; j += gridDim.x)
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
      const size_t e = i + (size_t)j * l;
      const double rij = (i == j ? 1.0 : 0.0) - XtX[e];
      double v;
      if (i == j) v = 1.0 + 0.5 * rij;
      else if (fabs(lm[i] - lm[j]) > dl) v = (S[e] + lm[j] * rij) / (lm[j] - lm[i]);
      else v = 0.5 * rij;
      E[e] = v;
    }
}

// Sort eigenpairs by descending eigenvalue (stable), sigma = sqrt(max(lambda,
// 0)): one CTA per eigenpair c finds its rank and copies its column.
__global__ void __launch_bounds__(128)
k_sort_eig(int l, const double* __restrict__ lam, const double* __restrict__ X,
           double* __restrict__ sigma, double* __restrict__ U) {
  __shared__ int s_rank;
  const int c = blockIdx.x, tid = threadIdx.x;
  const double lc = lam[c];
  if (tid < 32) {
    int r = 0;
    for (int j = tid; j < l; j += 32) {
      const double lj = lam[j];
      r += (lj > lc) || (lj == lc && j < c);
    }
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (tid == 0) {
      s_rank = r;
      sigma[r] = sqrt(fmax(lc, 0.0));
    }
  }
  __syncthreads();
  const int r = s_rank;
  for (int i = tid; i < l; i += blockDim.x) U[i + (size_t)r * l] = X[i + (size_t)c * l];
}


size_t sym_eig_work_doubles(int l) {
  // [X0 | AX0], [X1 | AX1], [X^T X | X^T A X], E, split partials (4 splits
  // of l x 2l), lambda, norm partials and delta, then the FP32 scratch of
  // the starting eigenvectors
  return (size_t)l * l * 15 + (size_t)l + 3 * 64 + 8 + (eig_scratch_floats(l) + 1) / 2 + 2;
}

cudaError_t sym_eig(cudaStream_t st, int l, const double* G, double* sigma, double* Uhat,
                    double* work, unsigned* status, int refine_iters) {
  const size_t ll = (size_t)l * l;
  double* XA[2] = {work, work + 2 * ll};  // [X | G X], ld l
  double* XS = work + 4 * ll;             // [X^T X | X^T G X]
  double* E = XS + 2 * ll;
  double* part = E + ll;                  // 4 * 2 ll
  double* lam = part + 8 * ll;
  double* part3 = lam + l;                // 3 x (at most 64) norm partials
  double* delta = part3 + 3 * 64;
  // 16-byte aligned FP32 scratch after delta (the work buffer is aligned)
  const size_t esc_off = (size_t)(delta + 8 - work + 1) & ~(size_t)1;
  float* esc = reinterpret_cast<float*>(work + esc_off);
  // the ticket of k_oa_norm sits in the status block (cleared at every basis
  // call; the kernel's last block resets it)
  unsigned* ticket = status + 8;
  prepare_kernels();
  cudaError_t e = tridiag_eig32(st, l, G, XA[0], esc, status);
  if (e != cudaSuccess) return e;
  const int nsp = l > 64 ? 8 : 4;
  const unsigned nb = (unsigned)std::min(64, l);
  int cur = 0;
  // lambda and E from the basis in XA[cur]: G X, then [X^T X | X^T G X] as
  // one product, then the two pass kernels
  auto oa_step = [&]() -> cudaError_t {
    double* X = XA[cur];
    double* AX = X + ll;
    cudaError_t r;
    if ((r = gemm<double, double, double, double>(st, false, l, l, l, nsp, G, l, X, l, part, 1, l, ll, status, false))) return r;
    if ((r = reduce_splits<double, double>(st, l, l, nsp, part, AX, 1, l))) return r;
    if ((r = gemm<double, double, double, double>(st, true, l, 2 * l, l, 4, X, l, X, l, part, 1, l, 2 * ll, status, false))) return r;
    if ((r = reduce_splits<double, double>(st, l, 2 * l, 4, part, XS, 1, l))) return r;
    k_oa_norm<<<nb, 256, 0, st>>>(l, XS, G, part3, ticket, lam, delta);
    note_launch();
    k_oa_e<<<nb, 256, l * sizeof(double), st>>>(l, XS, lam, delta, E);
    note_launch();
    return cudaGetLastError();
  };
  for (int it = 0; it < refine_iters; ++it) {
    if ((e = oa_step())) return e;
    // X <- X (I + E), into the other buffer
    if ((e = gemm<double, double, double, double>(st, false, l, l, l, nsp, XA[cur], l, E, l, part, 1, l, ll, status, false))) return e;
    if ((e = reduce_splits<double, double>(st, l, l, nsp, part, XA[cur ^ 1], 1, l))) return e;
    cur ^= 1;
  }
  // eigenvalues: Rayleigh quotients of the final basis (refine_iters = 0:
  // of the starting vectors)
  if (refine_iters == 0 && (e = oa_step())) return e;
  k_sort_eig<<<l, 128, 0, st>>>(l, lam, XA[cur], sigma, Uhat);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Column sign convention.
struct ArgMax { double v; long long i; };

// Per column and 8192-row block: the entry of largest magnitude (first row
// on ties).  Eight loads in flight per thread, then warp shuffles and one
// pass over the eight warp results.
template <typename T>
__device__ __forceinline__ void argmax_merge(T& ba, T& bv, long long& bi, T a, T v, long long i) {
  if (a > ba || (a == ba && i < bi)) { ba = a; bv = v; bi = i; }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_colmax_partial(int64_t n, int64_t rows_per_blk, const T* __restrict__ U, int64_t ldu,
                 ArgMax* __restrict__ out, int nblk) {
  const int c = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
  const int64_t r1 = (r0 + rows_per_blk < n) ? r0 + rows_per_blk : n;
  const T* u = U + (int64_t)c * ldu;
  // compared in the matrix's own type (FP64 compares of FP32 data would run
  // on GB300's narrow FP64 pipe)
  T bv = T(0), ba = T(-1);
  long long bi = LLONG_MAX;
  // rows visited in increasing order so the first of equal magnitudes wins
  const int64_t step = blockDim.x;
  for (int64_t rb = r0 + threadIdx.x; rb < r1; rb += 8 * step) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t r = rb + k * step;
      v[k] = r < r1 ? u[r] : T(0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t r = rb + k * step;
      const T a = fabs(v[k]);
      if (r < r1 && a > ba) { ba = a; bv = v[k]; bi = r; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T oa = __shfl_xor_sync(0xffffffffu, ba, o);
    const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
    argmax_merge(ba, bv, bi, oa, ov, oi);
  }
  __shared__ T sa[8], sv[8];
  __shared__ long long si[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sa[w] = ba; sv[w] = bv; si[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) argmax_merge(ba, bv, bi, sa[k], sv[k], si[k]);
    out[c * nblk + blockIdx.x] = ArgMax{ba < T(0) ? 0.0 : (double)bv, bi};
  }
}

__global__ void k_colsign(int ncols, int nblk, const ArgMax* __restrict__ part, double* __restrict__ sgn,
                          double* __restrict__ Uhat, int l) {
  const int c = blockIdx.x;
  __shared__ double s_s;
  if (threadIdx.x == 0) {
    double ba = -1.0, bv = 0.0;
    long long bi = LLONG_MAX;
    for (int b = 0; b < nblk; ++b) {
      const ArgMax p = part[c * nblk + b];
      const double a = fabs(p.v);
      if (p.i != LLONG_MAX && (a > ba || (a == ba && p.i < bi))) { ba = a; bv = p.v; bi = p.i; }
    }
    s_s = (bv < 0.0) ? -1.0 : 1.0;
    sgn[c] = s_s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < l; i += blockDim.x) Uhat[i + c * l] *= s_s;
}

// grid: x = column, y = chunks of 1024 rows (grid-stride); a column whose
// sign is + is left untouched.
template <typename T>
__global__ void __launch_bounds__(256)
k_scale_cols(int64_t n, int ncols, T* __restrict__ U, int64_t ldu, const double* __restrict__ sgn) {
  const int c = blockIdx.x;
  if (!(sgn[c] < 0.0)) return;
  T* u = U + (int64_t)c * ldu;
  for (int64_t r0 = (int64_t)blockIdx.y * 1024 + threadIdx.x; r0 < n; r0 += (int64_t)gridDim.y * 1024) {
    T v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (r0 + 256 * k < n) ? u[r0 + 256 * k] : T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (r0 + 256 * k < n) u[r0 + 256 * k] = -v[k];
  }
}

static dim3 col_grid(int64_t rows, int64_t cols) {
  const int64_t chunks = (rows + 1023) / 1024;
  return dim3((unsigned)cols, (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, 65535)));
}

size_t sign_fix_scratch_bytes(int64_t n, int ncols) {
  const int64_t nblk = (n + 8191) / 8192;
  return (size_t)ncols * nblk * sizeof(ArgMax) + (size_t)ncols * sizeof(double) + 256;
}

template <typename T>
cudaError_t sign_fix(cudaStream_t st, int64_t n, int ncols, T* U, int64_t ldu, double* Uhat, int l,
                     void* scratch, size_t) {
  const int64_t rpb = 8192;
  const int nblk = (int)((n + rpb - 1) / rpb);
  ArgMax* part = (ArgMax*)scratch;
  double* sgn = (double*)((char*)scratch + (((size_t)ncols * nblk * sizeof(ArgMax) + 255) / 256) * 256);
  k_colmax_partial<T><<<dim3(nblk, ncols), 256, 0, st>>>(n, rpb, U, ldu, part, nblk); note_launch();
  k_colsign<<<ncols, 128, 0, st>>>(ncols, nblk, part, sgn, Uhat, l); note_launch();
  k_scale_cols<T><<<col_grid(n, ncols), 256, 0, st>>>(n, ncols, U, ldu, sgn); note_launch();
  return cudaGetLastError();
}
template cudaError_t sign_fix<double>(cudaStream_t, int64_t, int, double*, int64_t, double*, int, void*, size_t);
template cudaError_t sign_fix<float>(cudaStream_t, int64_t, int, float*, int64_t, double*, int, void*, size_t);

// Sign rule over row blocks held by different calls.  xb (6 ncols doubles):
// [0, nc) the largest magnitude per column (exchanged, max), [nc, 2nc) the
// lowest global row holding it (exchanged, min), [2nc, 3nc) the sign of that
// entry (exchanged, sum: exactly one block contributes), [3nc, 6nc) this
// block's own candidate (magnitude, global row, sign).
constexpr double kNoRow = 1e300;

__global__ void k_sign_rows_local(int ncols, int nblk, const ArgMax* __restrict__ part, int64_t row0,
                                  double* __restrict__ xb) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double ba = -1.0, bv = 0.0;
  long long bi = LLONG_MAX;
  for (int b = 0; b < nblk; ++b) {
    const ArgMax p = part[c * nblk + b];
    const double a = fabs(p.v);
    if (p.i != LLONG_MAX && (a > ba || (a == ba && p.i < bi))) { ba = a; bv = p.v; bi = p.i; }
  }
  const bool any = bi != LLONG_MAX;
  xb[c] = any ? ba : -1.0;
  xb[3 * ncols + c] = any ? ba : -1.0;
  xb[4 * ncols + c] = any ? (double)(row0 + bi) : kNoRow;
  xb[5 * ncols + c] = bv < 0.0 ? -1.0 : 1.0;
}

// step 1 (after the max): offer this block's row if it holds the largest
// magnitude; step 2 (after the min): offer the sign if that row is ours.
__global__ void k_sign_rows_step(int ncols, double* __restrict__ xb, int step) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const bool holds = xb[3 * ncols + c] >= 0.0 && xb[3 * ncols + c] == xb[c];
  if (step == 1)
    xb[ncols + c] = holds ? xb[4 * ncols + c] : kNoRow;
  else
    xb[2 * ncols + c] = (holds && xb[4 * ncols + c] == xb[ncols + c]) ? xb[5 * ncols + c] : 0.0;
}

__global__ void k_sign_rows_uhat(int ncols, double* __restrict__ xb, double* __restrict__ Uhat, int l) {
  const int c = blockIdx.x;
  const double sg = xb[2 * ncols + c] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  if (threadIdx.x == 0) xb[2 * ncols + c] = sg;
  for (int i = threadIdx.x; i < l; i += blockDim.x) Uhat[i + c * l] *= sg;
}

template <typename T>
cudaError_t sign_rows_candidates(cudaStream_t st, int64_t n, int ncols, const T* U, int64_t ldu,
                                 int64_t row0, double* xb, void* scratch, size_t) {
  const int64_t rpb = 8192;
  const int nblk = (int)((n + rpb - 1) / rpb);
  ArgMax* part = (ArgMax*)scratch;
  k_colmax_partial<T><<<dim3(nblk, ncols), 256, 0, st>>>(n, rpb, U, ldu, part, nblk); note_launch();
  k_sign_rows_local<<<(ncols + 127) / 128, 128, 0, st>>>(ncols, nblk, part, row0, xb); note_launch();
  return cudaGetLastError();
}
template cudaError_t sign_rows_candidates<double>(cudaStream_t, int64_t, int, const double*, int64_t, int64_t, double*, void*, size_t);
template cudaError_t sign_rows_candidates<float>(cudaStream_t, int64_t, int, const float*, int64_t, int64_t, double*, void*, size_t);

cudaError_t sign_rows_step(cudaStream_t st, int ncols, double* xb, int step) {
  k_sign_rows_step<<<(ncols + 127) / 128, 128, 0, st>>>(ncols, xb, step); note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t sign_rows_apply(cudaStream_t st, int64_t n, int ncols, T* U, int64_t ldu, double* Uhat,
                            int l, double* xb) {
  k_sign_rows_uhat<<<ncols, 128, 0, st>>>(ncols, xb, Uhat, l); note_launch();
  k_scale_cols<T><<<col_grid(n, ncols), 256, 0, st>>>(n, ncols, U, ldu, xb + 2 * ncols); note_launch();
  return cudaGetLastError();
}
template cudaError_t sign_rows_apply<double>(cudaStream_t, int64_t, int, double*, int64_t, double*, int, double*);
template cudaError_t sign_rows_apply<float>(cudaStream_t, int64_t, int, float*, int64_t, double*, int, double*);

// ------------------------------------------------------------------------
// grid: x = column, y = chunks of 1024 rows (grid-stride), four loads in
// flight per thread.
template <typename TS, typename TD>
__global__ void __launch_bounds__(256)
k_convert(int64_t rows, int64_t cols, const TS* __restrict__ src, int64_t lds,
          TD* __restrict__ dst, int64_t ldd) {
  const int64_t c = blockIdx.x;
  const TS* sc = src + c * lds;
  TD* dc = dst + c * ldd;
  for (int64_t r0 = (int64_t)blockIdx.y * 1024 + threadIdx.x; r0 < rows; r0 += (int64_t)gridDim.y * 1024) {
    TS v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (r0 + 256 * k < rows) ? sc[r0 + 256 * k] : TS(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (r0 + 256 * k < rows) dc[r0 + 256 * k] = cvt<TD>(v[k]);
  }
}

template <typename TS, typename TD>
cudaError_t convert_matrix(cudaStream_t st, int64_t rows, int64_t cols, const TS* src, int64_t lds,
                           TD* dst, int64_t ldd) {
  if (rows < 1 || cols < 1) return cudaSuccess;
  k_convert<TS, TD><<<col_grid(rows, cols), 256, 0, st>>>(rows, cols, src, lds, dst, ldd); note_launch();
  return cudaGetLastError();
}
template cudaError_t convert_matrix<double, float>(cudaStream_t, int64_t, int64_t, const double*, int64_t, float*, int64_t);
template cudaError_t convert_matrix<double, double>(cudaStream_t, int64_t, int64_t, const double*, int64_t, double*, int64_t);

template <typename T>
__global__ void __launch_bounds__(256)
k_check_finite(int64_t rows, int64_t cols, const T* __restrict__ S, int64_t lds, unsigned* status) {
  const T* sc = S + (int64_t)blockIdx.x * lds;
  bool bad = false;
  for (int64_t r0 = (int64_t)blockIdx.y * 1024 + threadIdx.x; r0 < rows; r0 += (int64_t)gridDim.y * 1024) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (r0 + 256 * k < rows) ? cvt<float>(sc[r0 + 256 * k]) : 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) bad |= !isfinite(v[k]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

template <typename T>
cudaError_t check_finite(cudaStream_t st, int64_t rows, int64_t cols, const T* S, int64_t lds, unsigned* status) {
  if (rows < 1 || cols < 1) return cudaSuccess;
  k_check_finite<T><<<col_grid(rows, cols), 256, 0, st>>>(rows, cols, S, lds, status); note_launch();
  return cudaGetLastError();
}
template cudaError_t check_finite<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*, int64_t, unsigned*);
template cudaError_t check_finite<__half>(cudaStream_t, int64_t, int64_t, const __half*, int64_t, unsigned*);

}  // namespace rpod

namespace rpod {

// ------------------------------------------------------------------------
// FP32 -> 16-bit snapshot copy (the down-conversion of the 16-bit forms).
// Work is split into units of (column, 8192-row chunk) handed out grid-
// stride, so no per-element division; in the vector form each thread moves
// 8 consecutive rows per step (two 16-byte loads, one 16-byte store) with
// four steps in flight.
template <typename TD> __device__ __forceinline__ unsigned pack2(float a, float b);
template <> __device__ __forceinline__ unsigned pack2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  unsigned u;
  memcpy(&u, &h, 4);
  return u;
}
template <> __device__ __forceinline__ unsigned pack2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  unsigned u;
  memcpy(&u, &h, 4);
  return u;
}

__device__ __forceinline__ bool finite4(const float4& v) {
  return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

constexpr int kConvThreads = 256;
constexpr int kConvSteps = 4;
constexpr int kConvRows = kConvThreads * 8 * kConvSteps;  // rows per work unit

template <typename TD>
__global__ void __launch_bounds__(kConvThreads, 4)
k_convert_snapshots(int64_t rows, int64_t cols, const float* __restrict__ S, int64_t lds,
                    TD* __restrict__ D, int64_t ldd, unsigned* status, int vec) {
  bool bad = false;
  const int64_t per_col = (rows + kConvRows - 1) / kConvRows;
  const int64_t units = per_col * cols;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t c = u / per_col;
    const int64_t r0 = (u - c * per_col) * kConvRows;
    const float* s = S + c * lds;
    TD* d = D + c * ldd;
    if (vec) {  // rows % 8 == 0: every 8-row group is whole
      float4 v[2 * kConvSteps];
#pragma unroll
      for (int i = 0; i < kConvSteps; ++i) {
        const int64_t r = r0 + (int64_t)(i * kConvThreads + threadIdx.x) * 8;
        if (r < rows) {
          v[2 * i] = __ldcs(reinterpret_cast<const float4*>(s + r));
          v[2 * i + 1] = __ldcs(reinterpret_cast<const float4*>(s + r + 4));
        }
      }
#pragma unroll
      for (int i = 0; i < kConvSteps; ++i) {
        const int64_t r = r0 + (int64_t)(i * kConvThreads + threadIdx.x) * 8;
        if (r < rows) {
          const float4 a = v[2 * i], b = v[2 * i + 1];
          bad |= !(finite4(a) && finite4(b));
          uint4 o;
          o.x = pack2<TD>(a.x, a.y);
          o.y = pack2<TD>(a.z, a.w);
          o.z = pack2<TD>(b.x, b.y);
          o.w = pack2<TD>(b.z, b.w);
          *reinterpret_cast<uint4*>(d + r) = o;
        }
      }
    } else {
      const int64_t r1 = min(rows, r0 + (int64_t)kConvRows);
      for (int64_t r = r0 + threadIdx.x; r < r1; r += kConvThreads) {
        const float x = s[r];
        bad |= !isfinite(x);
        d[r] = cvt<TD>(x);
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

template <typename TD>
cudaError_t convert_snapshots(cudaStream_t st, int64_t rows, int64_t cols, const float* S,
                              int64_t lds, TD* D, int64_t ldd, unsigned* status) {
  const int vec = ((rows & 7) == 0 && (lds & 3) == 0 && (ldd & 7) == 0 &&
                   (((uintptr_t)S) & 15) == 0 && (((uintptr_t)D) & 15) == 0) ? 1 : 0;
  const int64_t units = (rows + kConvRows - 1) / kConvRows * cols;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(units, 152 * 4));
  k_convert_snapshots<TD><<<grid, kConvThreads, 0, st>>>(rows, cols, S, lds, D, ldd, status, vec);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t convert_snapshots<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const float*, int64_t, __nv_bfloat16*, int64_t, unsigned*);
template cudaError_t convert_snapshots<__half>(cudaStream_t, int64_t, int64_t, const float*, int64_t, __half*, int64_t, unsigned*);

// Round-to-nearest (ties away) of an FP32 matrix to TF32, same unit split.
__global__ void __launch_bounds__(kConvThreads)
k_round_tf32(int64_t rows, int64_t cols, const float* __restrict__ src, int64_t lds,
             float* __restrict__ dst, int64_t ldd) {
  const int64_t per_col = (rows + kConvRows - 1) / kConvRows;
  const int64_t units = per_col * cols;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t c = u / per_col;
    const int64_t r0 = (u - c * per_col) * kConvRows;
    const int64_t r1 = min(rows, r0 + (int64_t)kConvRows);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kConvThreads) {
      uint32_t v;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v) : "f"(src[r + c * lds]));
      dst[r + c * ldd] = __uint_as_float(v);
    }
  }
}

cudaError_t round_tf32(cudaStream_t st, int64_t rows, int64_t cols, const float* src, int64_t lds,
                       float* dst, int64_t ldd) {
  const int64_t units = (rows + kConvRows - 1) / kConvRows * cols;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(units, 152 * 8));
  k_round_tf32<<<grid, kConvThreads, 0, st>>>(rows, cols, src, lds, dst, ldd);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_check_finite_vec(int l, const double* __restrict__ v, unsigned* status) {
  for (int i = threadIdx.x; i < l; i += blockDim.x)
    if (!isfinite(v[i])) atomicOr(status, ST_NONFINITE);
}

cudaError_t check_finite_vec(cudaStream_t st, int l, const double* v, unsigned* status) {
  k_check_finite_vec<<<1, 128, 0, st>>>(l, v, status);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t convert_matrix<float, __nv_bfloat16>(cudaStream_t, int64_t, int64_t, const float*, int64_t, __nv_bfloat16*, int64_t);
template cudaError_t convert_matrix<float, __half>(cudaStream_t, int64_t, int64_t, const float*, int64_t, __half*, int64_t);

}  // namespace rpod

namespace rpod {

// ------------------------------------------------------------------------
// Gram partials of a tall FP32 matrix: part[z] = Y_z^T Y_z (l x l, FP64) for
// the z-th chunk of rows, Y column-major (rows x l, ld ldy, l <= 128).  The
// chunk is staged in shared memory once (both operands of the product are the
// same tile), each thread accumulates an 8 x 8 block in FP32 with float4
// shared loads, and the chunk's sum is written in FP64.
__global__ void __launch_bounds__(256)
k_gram_f32(int64_t rows, int l, const float* __restrict__ Y, int64_t ldy, int64_t chunk,
           double* __restrict__ part) {
  constexpr int BR = 32;
  __shared__ __align__(16) float Ys[BR][128 + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = (r0 + chunk < rows) ? r0 + chunk : rows;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int64_t rb = r0; rb < r1; rb += BR) {
    // column c, rows rb..rb+31: 32 consecutive floats per column
    for (int e = tid; e < BR * 128; e += 256) {
      const int rr = e & (BR - 1), c = e / BR;
      const int64_t r = rb + rr;
      Ys[rr][c] = (c < l && r < r1) ? Y[r + (int64_t)c * ldy] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < BR; ++rr) {
      const float4 a0 = *(const float4*)&Ys[rr][ty * 8];
      const float4 a1 = *(const float4*)&Ys[rr][ty * 8 + 4];
      const float4 b0 = *(const float4*)&Ys[rr][tx * 8];
      const float4 b1 = *(const float4*)&Ys[rr][tx * 8 + 4];
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  double* pz = part + (int64_t)blockIdx.x * l * l;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ty * 8 + a, j = tx * 8 + b;
      if (i < l && j < l) pz[i + j * l] = (double)acc[a][b];
    }
}

cudaError_t gram_f32(cudaStream_t st, int64_t rows, int l, const float* Y, int64_t ldy, int nsplit,
                     double* part) {
  int64_t chunk = (rows + nsplit - 1) / nsplit;
  chunk = (chunk + 31) / 32 * 32;
  k_gram_f32<<<nsplit, 256, 0, st>>>(rows, l, Y, ldy, chunk, part);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rpod

namespace rpod {

void prepare_kernels() {
  static std::once_flag once;
  std::call_once(once, [] {
    const int big = 160 * 1024;
    cudaFuncSetAttribute(k_cholesky<double, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_cholesky64_gated<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gated_smem_bytes(kMaxL));
    prepare_eig_kernels();
    prepare_jacobi_kernels();
    cudaFuncSetAttribute(k_cholesky_blk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlkSmem);
    cudaFuncSetAttribute(k_cholesky_blk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlkSmem);
  });
  prepare_kernels_tc();
}

}  // namespace rpod
