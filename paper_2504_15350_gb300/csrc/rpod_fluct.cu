// Per-sample time averages and fluctuation snapshots (Eqs. (time_av),
// (fluct_q), (fluct_psi)), and the energy-based rank of Eq. (energy).
//
// The snapshot matrix S (n x m, column-major) holds M = m / nt parameter
// samples of nt consecutive snapshots each.  For sample g the time average
// is Sbar(:, g) = (1/nt) sum_p S(:, g nt + p) and the fluctuation snapshots
// are F(:, g nt + p) = S(:, g nt + p) - Sbar(:, g).
//
// One CTA takes a tile of R rows of one sample: it stages the R x nt tile in
// shared memory with TMA boxes of about 8 KB (R rows x Bc columns, each
// completing on its own mbarrier; every byte of S is read from HBM once),
// sums every row while later boxes are still arriving (four independent
// compensated sums per thread, in FP64 for an FP64 S and in FP32
// otherwise), and writes the means and the centered tile, optionally
// twice (F in S's type or a 16-bit type, and a 16-bit copy H for the
// tensor-core forms of the rPOD).  The tile height R is chosen so that the
// tile fills about 52 KB (four CTAs per SM, loading, summing and writing
// out of step); when even a 128-byte-high tile of nt snapshots would not fit in
// shared memory, a streaming variant sums from global memory and reads S
// again for the write, and an S that tensor maps cannot describe (16-byte
// alignment) is staged with 16-byte asynchronous copies in eight commit
// groups instead.  The pass is bound by HBM bandwidth: it moves
// n m (sizeof(S) + sizeof(F) + sizeof(H)) bytes plus the n M means.
#include <cuda.h>

#include <cfloat>
#include <cstring>
#include <type_traits>

#include "rpod_internal.cuh"

namespace rpod {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxRows = 512;                 // tile height limit (s_mean)
constexpr size_t kTileBudget = 52u << 10;     // four CTAs per SM
constexpr size_t kTileMax = 200u << 10;       // one CTA per SM

constexpr int kStages = 8;                    // cp.async commit groups per tile
constexpr int kMaxBoxes = 32;                 // TMA boxes (mbarriers) per tile
constexpr int kBoxBytes = 8192;               // target bytes per TMA box
constexpr uint64_t kTimeoutNs = 4000000000ull; // 4 s per wait

struct NoOut {};  // a missing output

__device__ __forceinline__ uint32_t sh32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Waits until at most `pending` of this thread's cp.async groups are in
// flight (the count must be an immediate).
__device__ __forceinline__ void cp_async_wait(int pending) {
  switch (pending) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
  }
}

template <typename TA> __device__ __forceinline__ TA quiet_nan();
template <> __device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double quiet_nan<double>() {
  return __longlong_as_double(0x7ff8000000000000LL);
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool bar_ready(uint64_t* b) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(sh32(b))
      : "memory");
  return ok != 0;
}
// Bounded wait for the single phase of a box barrier: false after the
// deadline or once another thread of the CTA gave up.
__device__ __noinline__ bool bar_wait(uint64_t* b, volatile int* abort_flag,
                                      uint64_t limit_ns = kTimeoutNs) {
  if (bar_ready(b)) return true;
  const uint64_t t0 = now_ns();
  while (!bar_ready(b)) {
    if (*abort_flag) return false;
    if (now_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float widen(float x) { return x; }
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ float widen(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float widen(__half x) { return __half2float(x); }

template <typename TO, typename TA> __device__ __forceinline__ TO narrow(TA v);
template <> __device__ __forceinline__ double narrow<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float narrow<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half narrow<__half, float>(float v) {
  return __float2half_rn(v);
}

__device__ __forceinline__ float absval(float x) { return fabsf(x); }
__device__ __forceinline__ double absval(double x) { return fabs(x); }

// Neumaier's compensated summation: s + c carries the sum.
template <typename TA>
__device__ __forceinline__ void neumaier(TA& s, TA& c, TA x) {
  const TA t = s + x;
  c += (absval(s) >= absval(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// V consecutive outputs of one column to dst (vector store when `vec`, else
// the first `valid` elements one by one).
template <typename TO, int V>
__device__ __forceinline__ void store_run(TO* dst, const TO (&v)[V], bool vec, int valid) {
  constexpr int kBytes = V * (int)sizeof(TO);
  if (vec && valid == V) {
    if constexpr (kBytes == 16) {
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
    } else if constexpr (kBytes == 8) {
      *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(v);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) dst[e] = v[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e)
      if (e < valid) dst[e] = v[e];
  }
}

// Four independent compensated sums (the loop-carried chain of one
// Neumaier sum, not the memory, would otherwise bound the kernel).
template <typename TA>
struct Sum4 {
  TA s[4] = {TA(0), TA(0), TA(0), TA(0)};
  TA c[4] = {TA(0), TA(0), TA(0), TA(0)};
  __device__ __forceinline__ void add4(TA x0, TA x1, TA x2, TA x3) {
    neumaier(s[0], c[0], x0);
    neumaier(s[1], c[1], x1);
    neumaier(s[2], c[2], x2);
    neumaier(s[3], c[3], x3);
  }
  __device__ __forceinline__ void add1(TA x) { neumaier(s[0], c[0], x); }
  __device__ __forceinline__ void total(TA& so, TA& co) const {
    so = s[0];
    co = c[0] + c[1] + c[2] + c[3];
    neumaier(so, co, s[1]);
    neumaier(so, co, s[2]);
    neumaier(so, co, s[3]);
  }
};

// Grid: one CTA per (row tile, sample), the row tile fastest.
//   SMEM:    stage the tile in dynamic shared memory (R x nt elements,
//            column segments of R rows contiguous) in kStages commit groups
//            of columns, summing each group while later ones load; else
//            stream from global memory.
//   in_vec:  S and lds allow 16-byte copies of V = 16 / sizeof(T) rows.
//   f_vec, h_vec: F, H and their leading dimensions allow V-element stores.
template <typename T, typename TF, typename TH, bool SMEM>
__global__ void __launch_bounds__(kThreads)
k_fluct(const __grid_constant__ CUtensorMap tm_main, const __grid_constant__ CUtensorMap tm_tail,
        int Bc, bool use_tma, int64_t n, int64_t nt, int64_t tiles, int R, const T* S,
        int64_t lds, TF* F, int64_t ldf, TH* __restrict__ H, int64_t ldh,
        typename AccOf<T>::type* __restrict__ Sbar, int64_t ldb, bool in_vec, bool f_vec,
        bool h_vec) {
  using TA = typename AccOf<T>::type;
  constexpr int V = 16 / (int)sizeof(T);
  constexpr bool kF = !std::is_same<TF, NoOut>::value;
  constexpr bool kH = !std::is_same<TH, NoOut>::value;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ TA s_sum[kThreads], s_cmp[kThreads];
  __shared__ TA s_mean[kMaxRows];
  __shared__ __align__(8) uint64_t s_bar[kMaxBoxes];
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int64_t g = (int64_t)blockIdx.x / tiles;
  const int64_t r0 = ((int64_t)blockIdx.x - g * tiles) * R;
  const T* Sg = S + g * nt * lds;
  const int CH = R / V;  // 16-byte chunks per column segment (a power of two)
  const int lgCH = __ffs(CH) - 1;
  // row sums: Rm = min(R, 256) rows side by side, NP column phases
  const int Rm = R < kThreads ? R : kThreads;
  const int NP = kThreads / Rm;
  const int cp = tid / Rm;
  // rows per thread: 1 or 2 (R <= kMaxRows = 2 * kThreads); the loops over
  // them run a fixed two iterations so the sums stay in registers
  static_assert(kMaxRows <= 2 * kThreads, "two rows per thread at most");
  Sum4<TA> acc[2];
  if (tid == 0) s_abort = 0;

  // adds the staged columns [ja, jb) of this thread's rows and phase
  auto sum_cols = [&](int ja, int jb) {
    const int j = ja + (cp - ja % NP + NP) % NP;  // first column of this phase
    const int step = NP * R;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = tid % Rm + u * Rm;
      if (r >= R) break;
      const T* p = tile + j * R + r;
      const T* const end = tile + jb * R;
      for (; p + 3 * step < end; p += 4 * step)
        acc[u].add4((TA)widen(p[0]), (TA)widen(p[step]), (TA)widen(p[2 * step]),
                    (TA)widen(p[3 * step]));
      for (; p < end; p += step) acc[u].add1((TA)widen(p[0]));
    }
  };

  if constexpr (SMEM) {
    if (use_tma) {
      // one TMA box of R rows x Bc columns per barrier (the last box from
      // the tail map); rows beyond n arrive as zeros
      const int nbox = (int)((nt + Bc - 1) / Bc);
      const int nfull = (int)(nt / Bc);
      if (tid == 0) {
        for (int b = 0; b < nbox; ++b)
          asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh32(&s_bar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      __syncthreads();
      if (tid == 0)
        for (int b = 0; b < nbox; ++b) {
          const int cols = b < nfull ? Bc : (int)(nt - (int64_t)nfull * Bc);
          const CUtensorMap* map = b < nfull ? &tm_main : &tm_tail;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                           sh32(&s_bar[b])),
                       "r"((uint32_t)(cols * R * (int)sizeof(T)))
                       : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], "
              "[%1, {%3, %4}], [%2];" ::"r"(sh32(tile + b * Bc * R)),
              "l"((uint64_t)map), "r"(sh32(&s_bar[b])), "r"((int)r0),
              "r"((int)(g * nt + (int64_t)b * Bc))
              : "memory");
        }
      for (int b = 0; b < nbox; ++b) {
        if (!bar_wait(&s_bar[b], &s_abort)) break;
        const int jb = (b + 1) * Bc < nt ? (b + 1) * Bc : (int)nt;
        sum_cols(b * Bc, jb);
      }
    } else {
      // issue: stage st covers columns [j0(st), j0(st + 1))
      for (int st = 0; st < kStages; ++st) {
        const int ja = (int)(nt * st / kStages), jb = (int)(nt * (st + 1) / kStages);
        for (int c = ja * CH + tid; c < jb * CH; c += kThreads) {
          const int j = c >> lgCH, q = c & (CH - 1);
          const int64_t row = r0 + q * V;
          const T* src = Sg + (int64_t)j * lds + row;
          T* dst = tile + c * V;  // = tile + j * R + q * V
          const int64_t left = n - row;
          const int valid = left >= V ? V : (left > 0 ? (int)left : 0);
          if (in_vec) {
            // rows at or beyond n are zero-filled without reading them
            const void* gsrc = valid > 0 ? (const void*)src : (const void*)S;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sh32(dst)),
                         "l"(gsrc), "r"(valid * (int)sizeof(T))
                         : "memory");
          } else {
#pragma unroll
            for (int e = 0; e < V; ++e) dst[e] = e < valid ? src[e] : T(0.0f);
          }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
      // sum stage by stage as the groups land
      for (int st = 0; st < kStages; ++st) {
        cp_async_wait(kStages - 1 - st);
        __syncthreads();
        sum_cols((int)(nt * st / kStages), (int)(nt * (st + 1) / kStages));
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = tid % Rm + u * Rm;
      if (r >= R || r0 + r >= n) break;
      const int64_t step = (int64_t)NP * lds;
      const T* p = Sg + r0 + r + (int64_t)cp * lds;
      int64_t j = cp;
      for (; j + 3 * NP < nt; j += 4 * NP, p += 4 * step)
        acc[u].add4((TA)widen(p[0]), (TA)widen(p[step]), (TA)widen(p[2 * step]),
                    (TA)widen(p[3 * step]));
      for (; j < nt; j += NP, p += step) acc[u].add1((TA)widen(p[0]));
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int r = tid % Rm + u * Rm;
    if (r >= R) break;
    TA s, c;
    acc[u].total(s, c);
    if (NP == 1) {
      s_mean[r] = (s + c) / (TA)nt;
    } else {
      s_sum[cp * Rm + r] = s;
      s_cmp[cp * Rm + r] = c;
    }
  }
  __syncthreads();
  if (SMEM && s_abort) {
    // a box barrier never completed (4 s): let this CTA's copies land
    // (bounded), mark the tile's means NaN and write no fluctuations
    if (tid == 0)
      for (int b = 0; b < (int)((nt + Bc - 1) / Bc); ++b) {
        const uint64_t t0 = now_ns();
        while (!bar_ready(&s_bar[b]) && now_ns() - t0 < kTimeoutNs) {
        }
      }
    for (int r = tid; r < R; r += kThreads)
      if (r0 + r < n) Sbar[r0 + r + g * ldb] = quiet_nan<TA>();
    __syncthreads();
    return;
  }
  if (NP > 1 && tid < R) {
    TA s = TA(0), c = TA(0);
    for (int k = 0; k < NP; ++k) {
      neumaier(s, c, s_sum[k * Rm + tid]);
      c += s_cmp[k * Rm + tid];
    }
    s_mean[tid] = (s + c) / (TA)nt;
  }
  __syncthreads();
  for (int r = tid; r < R; r += kThreads)
    if (r0 + r < n) Sbar[r0 + r + g * ldb] = s_mean[r];

  // ---- centered snapshots
  if constexpr (kF || kH) {
    if constexpr (SMEM) {
      const int nchunks = CH * (int)nt;
      for (int c = tid; c < nchunks; c += kThreads) {
        const int j = c >> lgCH, q = c & (CH - 1);
        const int64_t row = r0 + q * V;
        const int64_t left = n - row;
        if (left <= 0) continue;
        const int valid = left >= V ? V : (int)left;
        T x[V];
        *reinterpret_cast<uint4*>(x) = *reinterpret_cast<const uint4*>(tile + c * V);
        TA d[V];
#pragma unroll
        for (int e = 0; e < V; ++e) d[e] = (TA)widen(x[e]) - s_mean[q * V + e];
        const int64_t col = g * nt + j;
        if constexpr (kF) {
          TF o[V];
#pragma unroll
          for (int e = 0; e < V; ++e) o[e] = narrow<TF, TA>(d[e]);
          store_run<TF, V>(F + col * ldf + row, o, f_vec, valid);
        }
        if constexpr (kH) {
          TH o[V];
#pragma unroll
          for (int e = 0; e < V; ++e) o[e] = narrow<TH, TA>((TA)d[e]);
          store_run<TH, V>(H + col * ldh + row, o, h_vec, valid);
        }
      }
    } else {
      // streaming: thread (r, cp) rewrites the elements it summed
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = tid % Rm + u * Rm;
        if (r >= R || r0 + r >= n) break;
        const int64_t row = r0 + r;
        const TA mu = s_mean[r];
        const T* p = Sg + row + (int64_t)cp * lds;
        TF* pf = nullptr;
        TH* ph = nullptr;
        if constexpr (kF) pf = F + (g * nt + cp) * ldf + row;
        if constexpr (kH) ph = H + (g * nt + cp) * ldh + row;
        for (int64_t j = cp; j < nt; j += NP) {
          const TA d = (TA)widen(p[0]) - mu;
          p += (int64_t)NP * lds;
          if constexpr (kF) {
            *pf = narrow<TF, TA>(d);
            pf += (int64_t)NP * ldf;
          }
          if constexpr (kH) {
            *ph = narrow<TH, TA>(d);
            ph += (int64_t)NP * ldh;
          }
        }
      }
    }
  }
}

// Self-test of the bounded waits: the CTA waits on an mbarrier that nothing
// arrives on (no copy is issued), through the same helper as the staged
// tiles, limited to limit_ns; the expected outcome is the timeout status.
__device__ unsigned g_selftest_status;

__global__ void k_wait_selftest(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    g_selftest_status = 0u;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = bar_wait(&bar, &abort_flag, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok || abort_flag) atomicOr(&g_selftest_status, ST_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(sh32(&bar)) : "memory");
  }
}

// Eq. (energy) on the device, one thread: the smallest N with
// c_N / c_count >= delta, c_N the sequential partial sums of sigma; 0 when
// c_count is not positive.
__global__ void k_energy_rank(const double* __restrict__ sigma, int count, double delta,
                              int* __restrict__ rank) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double total = 0.0;
  for (int i = 0; i < count; ++i) total += sigma[i];
  int r = count;
  if (!(total > 0.0)) {
    r = 0;
  } else {
    double c = 0.0;
    for (int i = 0; i < count; ++i) {
      c += sigma[i];
      if (c / total >= delta) {
        r = i + 1;
        break;
      }
    }
  }
  *rank = r;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

template <typename T> CUtensorMapDataType map_type();
template <> CUtensorMapDataType map_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <> CUtensorMapDataType map_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType map_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> CUtensorMapDataType map_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

// Tensor map of the column-major n x m matrix S (rows contiguous), box of
// br rows x bc columns, no swizzle (the box lands as bc column segments of
// br rows), out-of-range rows read as zeros.
template <typename T>
bool snapshot_map(CUtensorMap* map, const T* S, int64_t n, int64_t m, int64_t lds, int br,
                  int bc) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)(lds * (int64_t)sizeof(T))};
  cuuint32_t box[2] = {(cuuint32_t)br, (cuuint32_t)bc};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, map_type<T>(), 2, const_cast<T*>(S), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, typename TF, typename TH>
int launch_fluct(int64_t n, int64_t m, int64_t nt, const T* S, int64_t lds, TF* F, int64_t ldf,
                 TH* H, int64_t ldh, typename AccOf<T>::type* Sbar, int64_t ldb,
                 cudaStream_t st) {
  constexpr int V = 16 / (int)sizeof(T);
  const int64_t M = m / nt;
  // tile height: the largest column segment (128 B .. 2 KB) whose tile
  // fits the budget, no taller than n needs
  int R = 0;
  bool smem = true;
  for (int bytes = 2048; bytes >= 128; bytes /= 2) {
    const int rows = bytes / (int)sizeof(T);
    if ((size_t)bytes * (size_t)nt <= kTileBudget && rows <= kMaxRows) {
      R = rows;
      break;
    }
  }
  if (R == 0) {
    const int rows = 128 / (int)sizeof(T);
    if ((size_t)128 * (size_t)nt <= kTileMax) {
      R = rows;
    } else {
      R = 64;  // streaming: 64 rows x 4 column phases
      smem = false;
    }
  }
  int64_t need = 1;
  while (need < n) need *= 2;
  const int64_t rmin = smem ? V : 32;
  if (need < rmin) need = rmin;
  if (need < R) R = (int)need;
  const int64_t tiles = (n + R - 1) / R;
  const int64_t grid = tiles * M;
  if (grid > 0x7fffffffLL) return RPOD_ERR_UNSUPPORTED;
  const bool in_vec = aligned(S, 16) && (lds * (int64_t)sizeof(T)) % 16 == 0;
  bool f_vec = false, h_vec = false;
  if constexpr (!std::is_same<TF, NoOut>::value)
    f_vec = aligned(F, V * sizeof(TF)) && (ldf % V) == 0;
  if constexpr (!std::is_same<TH, NoOut>::value)
    h_vec = aligned(H, V * sizeof(TH)) && (ldh % V) == 0;
  const size_t dyn = smem ? (size_t)R * (size_t)nt * sizeof(T) : 0;
  // TMA boxes of about kBoxBytes (R rows x Bc columns, at most kMaxBoxes
  // per tile; the tail map covers the nt mod Bc last columns of a sample)
  // when S allows tensor maps and a column segment is a multiple of 128 B
  CUtensorMap tm_main, tm_tail;
  memset(&tm_main, 0, sizeof(tm_main));
  memset(&tm_tail, 0, sizeof(tm_tail));
  int Bc = 1;
  bool use_tma = smem && in_vec && (R * (int)sizeof(T)) % 128 == 0 && n < (1LL << 31) &&
                 m < (1LL << 31);
  if (use_tma) {
    Bc = kBoxBytes / (R * (int)sizeof(T));
    if (Bc < 1) Bc = 1;
    if (Bc > nt) Bc = (int)nt;
    if ((nt + Bc - 1) / Bc > kMaxBoxes) Bc = (int)((nt + kMaxBoxes - 1) / kMaxBoxes);
    if (Bc > 256) use_tma = false;
  }
  if (use_tma) {
    const int tail = (int)(nt % Bc);
    use_tma = snapshot_map(&tm_main, S, n, m, lds, R, Bc) &&
              (tail == 0 || snapshot_map(&tm_tail, S, n, m, lds, R, tail));
  }
  cudaError_t err;
  if (smem) {
    auto kern = k_fluct<T, TF, TH, true>;
    // the static arrays take up to 9 KB beside the tile: raise the limit
    // whenever the sum could pass the 48 KB default
    if (dyn > (32u << 10)) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTileMax);
      if (err != cudaSuccess) return RPOD_ERR_CUDA;
    }
    kern<<<(unsigned)grid, kThreads, dyn, st>>>(tm_main, tm_tail, Bc, use_tma, n, nt, tiles, R,
                                                 S, lds, F, ldf, H, ldh, Sbar, ldb, in_vec,
                                                 f_vec, h_vec);
  } else {
    k_fluct<T, TF, TH, false><<<(unsigned)grid, kThreads, 0, st>>>(
        tm_main, tm_tail, Bc, false, n, nt, tiles, R, S, lds, F, ldf, H, ldh, Sbar, ldb, in_vec,
        f_vec, h_vec);
  }
  note_launch();
  err = cudaGetLastError();
  return err == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}

// Output pointer of a given type or the missing output.
template <typename TF, typename TH, typename T>
int dispatch3(int64_t n, int64_t m, int64_t nt, const T* S, int64_t lds, void* F, int64_t ldf,
              void* H, int64_t ldh, void* Sbar, int64_t ldb, cudaStream_t st) {
  using TA = typename AccOf<T>::type;
  return launch_fluct<T, TF, TH>(n, m, nt, S, lds, (TF*)F, ldf, (TH*)H, ldh, (TA*)Sbar, ldb, st);
}

template <typename T, typename TF>
int dispatch_h(int64_t n, int64_t m, int64_t nt, const T* S, int64_t lds, void* F, int64_t ldf,
               void* H, int64_t ldh, int32_t h_dtype, void* Sbar, int64_t ldb, cudaStream_t st) {
  if (!H) return dispatch3<TF, NoOut>(n, m, nt, S, lds, F, ldf, nullptr, 0, Sbar, ldb, st);
  if (h_dtype == RPOD_BF16)
    return dispatch3<TF, __nv_bfloat16>(n, m, nt, S, lds, F, ldf, H, ldh, Sbar, ldb, st);
  if (h_dtype == RPOD_F16)
    return dispatch3<TF, __half>(n, m, nt, S, lds, F, ldf, H, ldh, Sbar, ldb, st);
  return RPOD_ERR_UNSUPPORTED;
}

}  // namespace
}  // namespace rpod

using namespace rpod;

extern "C" int rpod_fluctuations(int64_t n, int64_t m, int64_t nt, const void* S, int64_t lds,
                                 int32_t s_dtype, void* F, int64_t ldf, int32_t f_dtype,
                                 void* H, int64_t ldh, int32_t h_dtype, void* Sbar,
                                 int64_t ldb, void* stream) {
  if (n < 1 || m < 1 || nt < 1 || m % nt != 0 || !S || !Sbar || lds < n || ldb < n)
    return RPOD_ERR_INVALID_ARG;
  if (F && ldf < n) return RPOD_ERR_INVALID_ARG;
  if (H && ldh < n) return RPOD_ERR_INVALID_ARG;
  if (s_dtype < RPOD_F64 || s_dtype > RPOD_F16) return RPOD_ERR_INVALID_ARG;
  if (F && (f_dtype < RPOD_F64 || f_dtype > RPOD_F16)) return RPOD_ERR_INVALID_ARG;
  if (H && (h_dtype < RPOD_F64 || h_dtype > RPOD_F16)) return RPOD_ERR_INVALID_ARG;
  // F either is S (same type and leading dimension) or does not overlap it
  if (F == S && (f_dtype != s_dtype || ldf != lds)) return RPOD_ERR_INVALID_ARG;
  g_launches = 0;
  cudaStream_t st = (cudaStream_t)stream;
  switch (s_dtype) {
    case RPOD_F64: {
      if (H) return RPOD_ERR_UNSUPPORTED;
      const double* s = (const double*)S;
      if (!F) return dispatch3<NoOut, NoOut>(n, m, nt, s, lds, nullptr, 0, nullptr, 0, Sbar, ldb, st);
      if (f_dtype != RPOD_F64) return RPOD_ERR_UNSUPPORTED;
      return dispatch3<double, NoOut>(n, m, nt, s, lds, F, ldf, nullptr, 0, Sbar, ldb, st);
    }
    case RPOD_F32: {
      const float* s = (const float*)S;
      if (!F) return dispatch_h<float, NoOut>(n, m, nt, s, lds, nullptr, 0, H, ldh, h_dtype, Sbar, ldb, st);
      if (f_dtype == RPOD_F32)
        return dispatch_h<float, float>(n, m, nt, s, lds, F, ldf, H, ldh, h_dtype, Sbar, ldb, st);
      if (f_dtype == RPOD_BF16)
        return dispatch_h<float, __nv_bfloat16>(n, m, nt, s, lds, F, ldf, H, ldh, h_dtype, Sbar, ldb, st);
      if (f_dtype == RPOD_F16)
        return dispatch_h<float, __half>(n, m, nt, s, lds, F, ldf, H, ldh, h_dtype, Sbar, ldb, st);
      return RPOD_ERR_UNSUPPORTED;
    }
    case RPOD_BF16: {
      if (H || (F && f_dtype != RPOD_BF16)) return RPOD_ERR_UNSUPPORTED;
      const __nv_bfloat16* s = (const __nv_bfloat16*)S;
      if (!F) return dispatch3<NoOut, NoOut>(n, m, nt, s, lds, nullptr, 0, nullptr, 0, Sbar, ldb, st);
      return dispatch3<__nv_bfloat16, NoOut>(n, m, nt, s, lds, F, ldf, nullptr, 0, Sbar, ldb, st);
    }
    default: {
      if (H || (F && f_dtype != RPOD_F16)) return RPOD_ERR_UNSUPPORTED;
      const __half* s = (const __half*)S;
      if (!F) return dispatch3<NoOut, NoOut>(n, m, nt, s, lds, nullptr, 0, nullptr, 0, Sbar, ldb, st);
      return dispatch3<__half, NoOut>(n, m, nt, s, lds, F, ldf, nullptr, 0, Sbar, ldb, st);
    }
  }
}

extern "C" int rpod_selftest_wait_timeout(double seconds, void* stream) {
  if (!(seconds > 0.0) || !(seconds <= 2.0)) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)(seconds * 1e9));
  if (cudaGetLastError() != cudaSuccess) return RPOD_ERR_CUDA;
  unsigned h = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_selftest_status, sizeof(h), 0, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  return (h & ST_TIMEOUT) ? RPOD_ERR_TIMEOUT : RPOD_OK;
}

extern "C" int rpod_energy_rank(const double* sigma, int32_t count, double delta, int32_t* rank,
                                void* stream) {
  if (!sigma || !rank || count < 1 || !(delta > 0.0) || !(delta <= 1.0))
    return RPOD_ERR_INVALID_ARG;
  g_launches = 0;
  k_energy_rank<<<1, 32, 0, (cudaStream_t)stream>>>(sigma, count, delta, (int*)rank);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}
