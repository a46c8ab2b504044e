// Tensor-core passes over the snapshot matrix S for the 16-bit (and the TF32
// refinement) forms of Alg. 1 (Sec. 4.2), written for sm_103a:
// TMA (cp.async.bulk.tensor) stages 128-byte-swizzled tiles of S and of the
// skinny operand into shared memory through a STAGES-deep mbarrier ring, one
// elected thread issues tcgen05.mma into a TMEM accumulator, and all four
// warps drain TMEM with tcgen05.ld in the epilogue.
//
// Two pass shapes, both with the skinny l-wide operand as the MMA's M = 128
// side (l <= 128, rows >= l of the operand are TMA zero fill):
//   W-pass  W(c, j) = sum_i A(i, c) S(i, j)      (S^T Q and T = Q^T S)
//           K = n rows, K-major A and S tiles, split-K over n; partial
//           results part[z][c][j] are summed by a deterministic reduction.
//   Y-pass  Y(i, c) = sum_j S(i, j) A(j, c)      (S Lambda and S Z)
//           K = m snapshots, K-major A tile, MN-major S tile; each CTA owns
//           BN rows of Y and streams all of S's columns for them.
// The first Y-pass over an FP32 S can also write the 16-bit copy of S that
// the later passes read (one HBM read of S for both).
// A third kernel forms Gram matrices Y^T Y of FP32 tall-skinny matrices on
// the TF32 path with a hi/lo split (CholeskyQR's Gram, Alg. 1).
// Every mbarrier wait is bounded by a %globaltimer deadline; on expiry the
// kernel records ST_TIMEOUT, stops issuing work, frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "rpod_tc.cuh"

namespace rpod {
namespace tc {

constexpr uint64_t kTimeoutNs = 4000000000ull;  // 4 s per wait

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}
// 1024-byte aligned start within the dynamic shared memory.  Offset
// arithmetic on the shared array keeps every pointer derived from it in the
// shared address space, so that accesses through it compile to shared-memory
// loads and stores (a round trip of the address through an integer would
// leave the compiler generic accesses, which take the slower generic path).
__device__ __forceinline__ uint8_t* align_smem1024(uint8_t* base) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(base);
  return base + ((1024u - (a & 1023u)) & 1023u);
}
__device__ __forceinline__ float pick4(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on a phase; false when the deadline passed or another role
// already gave up (the shared abort flag).
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > kTimeoutNs) {
      *abort_flag = 1;
      return false;
    }
  }
}
// Bounded wait that ignores the abort flag: used after an abort to let this
// thread's own copies or MMAs finish before the shared memory and TMEM they
// target are released.
__device__ __noinline__ void mbar_wait_drain(uint64_t* b, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(b, parity))
    if (gtimer() - t0 > kTimeoutNs) return;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns of TMEM (one per thread and column).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05 format): start address, leading
// and stride byte offsets (>> 4), version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor: FP32 accumulate, A/B format (0 f16, 1 bf16, 2 tf32),
// A K-major, B K- or MN-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(int fmt, bool b_mn, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ constexpr int fmt_of(int kind) { return kind == 2 ? 2 : (kind == 1 ? 0 : 1); }

template <int BN, int STAGES>
struct Smem {
  static constexpr uint32_t A_BYTES = 128 * 128;
  static constexpr uint32_t B_BYTES = BN * 128;
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t BARS = STAGES * STAGE;
  static constexpr size_t TOTAL = 1024 + (size_t)STAGES * STAGE + 256;
};

// ---------------------------------------------------------------------------
// W-pass.  KIND 0 bf16, 1 fp16, 2 tf32 (32-bit containers, 32 per 128-B row).
template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(192, 1)
k_wpass(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmS, int64_t n,
        int64_t m, int l, int kchunk, float* __restrict__ part, unsigned* status) {
  using L = Smem<BN, STAGES>;
  constexpr int BKE = (KIND == 2) ? 32 : 64;
  extern __shared__ uint8_t smem_raw[];
  // TF32 form: the FP32 S tile is rounded to TF32 (round to nearest) in shared
  // memory by warps 2-5 before the MMA reads it, so that the tensor core's
  // truncation of the low mantissa bits adds no bias.  Warps 0-3 drain TMEM.
  constexpr bool RND = (KIND == 2);
  uint8_t* smem = align_smem1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + L::BARS);
  uint64_t* empty = full + STAGES;
  uint64_t* conv = empty + STAGES;
  uint64_t* done = conv + STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)blockIdx.x * BN;
  const int64_t ktiles = (n + BKE - 1) / BKE;
  const int64_t kt0 = (int64_t)blockIdx.y * kchunk;
  const int64_t kt1 = (kt0 + kchunk < ktiles) ? kt0 + kchunk : ktiles;
  const int nk = kt1 > kt0 ? (int)(kt1 - kt0) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, BN);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0 && nk > 0) {
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (it >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
      uint8_t* a = smem + s * L::STAGE;
      mbar_expect_tx(&full[s], L::STAGE);
      const int kc = (int)((kt0 + it) * BKE);
      tma_load_2d(a, &tmA, &full[s], kc, 0);
      tma_load_2d(a + L::A_BYTES, &tmS, &full[s], kc, (int)j0);
    }
  } else if (RND && warp >= 2 && nk > 0) {
    const int ct = threadIdx.x - 64;
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, abort_flag))) break;
      float4* b4 = (float4*)(smem + s * L::STAGE + L::A_BYTES);
      for (int e0 = ct; e0 < (int)(L::B_BYTES / 16); e0 += 4 * 128) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = b4[e0 + u * 128];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u].x = tf32_rna(v[u].x); v[u].y = tf32_rna(v[u].y);
          v[u].z = tf32_rna(v[u].z); v[u].w = tf32_rna(v[u].w);
          b4[e0 + u * 128] = v[u];
        }
      }
      // make the generic-proxy stores visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    constexpr uint32_t id = idesc(fmt_of(KIND), false, 128, BN);
    int it = 0;
    for (; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!mbar_wait(RND ? &conv[s] : &full[s], ph, abort_flag)) break;
      tc_after();
      const uint32_t a = su32(smem + s * L::STAGE), b = a + L::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma<KIND>(tmem, sdesc(a + 32 * kk, 16, 1024), sdesc(b + 32 * kk, 16, 1024), id,
                  (it > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  bool ok = true;
  if (nk > 0) ok = mbar_wait(done, 0, abort_flag);
  ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
  tc_after();
  if (warp < 4) {
    const int c = warp * 32 + lane;
    float* prow = part + (int64_t)blockIdx.y * (int64_t)l * m + (int64_t)c * m;
    for (int cc = 0; cc < BN; cc += 32) {
      float v[32];
      if (nk > 0 && ok) {
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
      } else {
  #pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      if (c < l) {
        const int64_t jb = j0 + cc;
        if (((m & 3) == 0) && jb + 32 <= m) {
          float4* d4 = (float4*)(prow + jb);
  #pragma unroll
          for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
          for (int i = 0; i < 32; ++i)
            if (jb + i < m) prow[jb + i] = v[i];
        }
      }
    }
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  tc_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------------------
// Y-pass (16-bit only): A^T tile K-major (128 x 64 snapshots), S tile MN-major
// (BN rows as BN/64 boxes of 64 rows x 64 snapshots).  blockIdx.y takes the
// 64-snapshot k-tiles kchunk * y .. kchunk * (y + 1) - 1 and writes its sum
// to Y + y * ysplit (a split over snapshots for matrices with few rows; the
// caller sums the slices).  Row tile blockIdx.x is tile tile0 + blockIdx.x of
// S; its rows i go to row i - yrow0 of Y (a launch over the last row tiles
// alone writes a compact slice).
template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(128, 1)
k_ypass(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmS, int64_t n,
        int64_t m, int l, float* __restrict__ Y, int64_t ldy, unsigned* status, int kchunk,
        int64_t ysplit, int64_t tile0, int64_t yrow0) {
  using L = Smem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align_smem1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + L::BARS);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (tile0 + (int64_t)blockIdx.x) * BN;
  // this CTA's k-tiles (the host sizes the chunks so that none is empty)
  const int nk_all = (int)((m + 63) / 64);
  const int kt0 = (int)blockIdx.y * kchunk;
  const int nk = min(nk_all, kt0 + kchunk) - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, BN);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    for (int j = 0; j < nk; ++j) {
      const int s = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (j >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
      const int it = kt0 + j;
      uint8_t* a = smem + s * L::STAGE;
      mbar_expect_tx(&full[s], L::STAGE);
      tma_load_2d(a, &tmA, &full[s], it * 64, 0);
#pragma unroll
      for (int b = 0; b < BN / 64; ++b)
        tma_load_2d(a + L::A_BYTES + b * 8192, &tmS, &full[s], (int)(i0 + 64 * b), it * 64);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc(fmt_of(KIND), true, 128, BN);
    for (int j = 0; j < nk; ++j) {
      const int s = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, abort_flag)) break;
      tc_after();
      const uint32_t a = su32(smem + s * L::STAGE), b = a + L::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma<KIND>(tmem, sdesc(a + 32 * kk, 16, 1024), sdesc(b + 2048 * kk, 8192, 1024), id,
                  (j > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  bool ok = mbar_wait(done, 0, abort_flag);
  ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
  tc_after();
  const int c = warp * 32 + lane;
  float* ycol = Y + (int64_t)blockIdx.y * ysplit + (int64_t)c * ldy;
  for (int cc = 0; cc < BN; cc += 32) {
    float v[32];
    if (ok) {
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
    }
    if (c < l) {
      const int64_t ib = i0 + cc;
      if (((ldy & 3) == 0) && ib + 32 <= n) {
        float4* d4 = (float4*)(ycol + (ib - yrow0));
#pragma unroll
        for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      } else {
        for (int i = 0; i < 32; ++i)
          if (ib + i < n) ycol[ib - yrow0 + i] = v[i];
      }
    }
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  tc_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------------------
// Gram matrix G = Y^T Y of an FP32 matrix on the TF32 tensor path with the
// three-term split y = hi + lo, hi = rn_tf32(y), lo = rn_tf32(y - hi):
// G ~ hi^T hi + hi^T lo + lo^T hi (the dropped lo^T lo term is below 2^-22 of
// each product).  One 32-row x 128-column K-major tile of Y serves as both
// MMA operands.  Warp 0 loads tiles by TMA, warps 2-5 split each tile into
// hi (in place) and lo (second buffer), warp 1 issues the MMAs; split-K over
// rows with FP64 partials part[z][c + j l], which the caller reduces.
template <int STAGES>
struct GramSmem {
  static constexpr uint32_t TILE = 128 * 128;  // 128 columns x 32 rows of FP32
  static constexpr uint32_t STAGE = 2 * TILE;
  static constexpr uint32_t BARS = STAGES * STAGE;
  static constexpr size_t TOTAL = 1024 + (size_t)STAGES * STAGE + 256;
};

template <int STAGES>
__global__ void __launch_bounds__(192, 1)
k_gram3(const __grid_constant__ CUtensorMap tmY, int64_t rows, int l, int kchunk,
        float* __restrict__ part, unsigned* status) {
  using L = GramSmem<STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align_smem1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + L::BARS);
  uint64_t* empty = full + STAGES;
  uint64_t* conv = empty + STAGES;
  uint64_t* done = conv + STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ktiles = (rows + 31) / 32;
  const int64_t kt0 = (int64_t)blockIdx.x * kchunk;
  const int64_t kt1 = (kt0 + kchunk < ktiles) ? kt0 + kchunk : ktiles;
  const int nk = kt1 > kt0 ? (int)(kt1 - kt0) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, 128);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0 && nk > 0) {
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (it >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
      mbar_expect_tx(&full[s], L::TILE);
      tma_load_2d(smem + s * L::STAGE, &tmY, &full[s], (int)((kt0 + it) * 32), 0);
    }
  } else if (warp >= 2 && nk > 0) {
    const int ct = threadIdx.x - 64;
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, abort_flag)) break;
      float4* h4 = (float4*)(smem + s * L::STAGE);
      float4* l4 = (float4*)(smem + s * L::STAGE + L::TILE);
#pragma unroll 4
      for (int e = ct; e < (int)(L::TILE / 16); e += 128) {
        const float4 v = h4[e];
        float4 h, o;
        h.x = tf32_rna(v.x); o.x = tf32_rna(v.x - h.x);
        h.y = tf32_rna(v.y); o.y = tf32_rna(v.y - h.y);
        h.z = tf32_rna(v.z); o.z = tf32_rna(v.z - h.z);
        h.w = tf32_rna(v.w); o.w = tf32_rna(v.w - h.w);
        h4[e] = h;
        l4[e] = o;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    constexpr uint32_t id = idesc(2, false, 128, 128);
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!mbar_wait(&conv[s], ph, abort_flag)) break;
      tc_after();
      const uint32_t h = su32(smem + s * L::STAGE), lo = h + L::TILE;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t dh = sdesc(h + 32 * kk, 16, 1024), dl = sdesc(lo + 32 * kk, 16, 1024);
        // smallest terms first
        mma<2>(tmem, dl, dh, id, (it > 0 || kk > 0) ? 1u : 0u);
        mma<2>(tmem, dh, dl, id, 1u);
        mma<2>(tmem, dh, dh, id, 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  if (warp >= 2) {
    bool ok = true;
    if (nk > 0) ok = mbar_wait(done, 0, abort_flag);
    ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
    tc_after();
    const int q = warp & 3;  // TMEM lane quarter this warp may read
    const int c = q * 32 + lane;
    float* pz = part + (int64_t)blockIdx.x * l * l;
    for (int cc = 0; cc < 128; cc += 32) {
      float v[32];
      if (nk > 0 && ok) {
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      if (c < l) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (cc + i < l) pz[c + (int64_t)(cc + i) * l] = v[i];
      }
    }
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  tc_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// Gram matrix with products as accurate as FP32 ones (the last CholeskyQR
// round, which fixes the orthogonality of the returned basis): every element
// of Y is split exactly into three TF32 parts h + m + r and the six products
// above 2^-33 (r h, h r, m m, m h, h m, h h) are accumulated.  The tensor
// core's FP32 accumulation drifts with the number of MMAs summed into one
// accumulator (its rounding does not average out), so the MMAs of each two
// 32-row tiles go into one of two TMEM accumulators, and warps 6-9 add every
// finished accumulator into FP32 sums in shared memory (round to nearest,
// upper triangle only) while the MMAs continue in the other one.
constexpr int kGxChain = 2;  // 32-row tiles per accumulator chain

template <int STAGES>
struct GramXSmem {
  static constexpr uint32_t TILE = 128 * 128;  // 128 columns x 32 rows of FP32
  static constexpr uint32_t STAGE = 3 * TILE;
  static constexpr uint32_t ACC = 4 * (128 * 129 / 2);  // one float per (c <= j)
  static constexpr uint32_t BARS = STAGES * STAGE + ACC;
  static constexpr size_t TOTAL = 1024 + (size_t)BARS + 256;
};

template <int STAGES>
__global__ void __launch_bounds__(320, 1)
k_gram_x(const __grid_constant__ CUtensorMap tmY, int64_t rows, int l, int kchunk,
         float* __restrict__ part, unsigned* status) {
  using L = GramXSmem<STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align_smem1024(smem_raw);
  float* acc = (float*)(smem + STAGES * L::STAGE);
  uint64_t* full = (uint64_t*)(smem + L::BARS);
  uint64_t* empty = full + STAGES;
  uint64_t* conv = empty + STAGES;
  uint64_t* tfull = conv + STAGES;  // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* mdone = tempty + 2;
  uint32_t* tslot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ktiles = (rows + 31) / 32;
  const int64_t kt0 = (int64_t)blockIdx.x * kchunk;
  const int64_t kt1 = (kt0 + kchunk < ktiles) ? kt0 + kchunk : ktiles;
  const int nk = kt1 > kt0 ? (int)(kt1 - kt0) : 0;
  const int nch = (nk + kGxChain - 1) / kGxChain;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp >= 6)
    for (int e = threadIdx.x - 192; e < 128 * 129 / 2; e += 128) acc[e] = 0.f;
  if (warp == 0) tmem_alloc(tslot, 256);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    int it = 0;
    for (; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (it >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
      mbar_expect_tx(&full[s], L::TILE);
      tma_load_2d(smem + s * L::STAGE, &tmY, &full[s], (int)((kt0 + it) * 32), 0);
    }
    if (*abort_flag)
      for (int i2 = it > STAGES ? it - STAGES : 0; i2 < it; ++i2)
        mbar_wait_drain(&full[i2 % STAGES], (uint32_t)(i2 / STAGES) & 1u);
  } else if (warp >= 2 && warp < 6) {
    const int ct = threadIdx.x - 64;
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, abort_flag))) break;
      float4* h4 = (float4*)(smem + s * L::STAGE);
      float4* m4 = (float4*)(smem + s * L::STAGE + L::TILE);
      float4* r4 = (float4*)(smem + s * L::STAGE + 2 * L::TILE);
#pragma unroll 4
      for (int e = ct; e < (int)(L::TILE / 16); e += 128) {
        const float4 v = h4[e];
        float4 h, m, r;
        h.x = tf32_rna(v.x); m.x = tf32_rna(v.x - h.x); r.x = tf32_rna((v.x - h.x) - m.x);
        h.y = tf32_rna(v.y); m.y = tf32_rna(v.y - h.y); r.y = tf32_rna((v.y - h.y) - m.y);
        h.z = tf32_rna(v.z); m.z = tf32_rna(v.z - h.z); r.z = tf32_rna((v.z - h.z) - m.z);
        h.w = tf32_rna(v.w); m.w = tf32_rna(v.w - h.w); r.w = tf32_rna((v.w - h.w) - m.w);
        h4[e] = h;
        m4[e] = m;
        r4[e] = r;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc(2, false, 128, 128);
    bool go = true, issued = false;
    for (int ch = 0, it = 0; ch < nch && go; ++ch) {
      const int buf = ch & 1;
      if (ch >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((ch >> 1) - 1) & 1u, abort_flag)) break;
      tc_after();
      const uint32_t d = tmem + (uint32_t)(buf * 128);
      for (int c2 = 0; c2 < kGxChain && it < nk; ++c2, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!mbar_wait(&conv[s], ph, abort_flag)) { go = false; break; }
        tc_after();
        const uint32_t h = su32(smem + s * L::STAGE), mm = h + L::TILE, r = h + 2 * L::TILE;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t dh = sdesc(h + 32 * kk, 16, 1024), dm = sdesc(mm + 32 * kk, 16, 1024),
                         dr = sdesc(r + 32 * kk, 16, 1024);
          mma<2>(d, dr, dh, id, (c2 > 0 || kk > 0) ? 1u : 0u);
          mma<2>(d, dh, dr, id, 1u);
          mma<2>(d, dm, dm, id, 1u);
          mma<2>(d, dm, dh, id, 1u);
          mma<2>(d, dh, dm, id, 1u);
          mma<2>(d, dh, dh, id, 1u);
        }
        mma_commit(&empty[s]);
        issued = true;
      }
      if (go) mma_commit(&tfull[buf]);
    }
    if (issued) {
      mma_commit(mdone);
      mbar_wait_drain(mdone, 0);
    }
  } else if (warp >= 6) {
    const int q = warp & 3;
    const int c = q * 32 + lane;
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull[buf], (uint32_t)(ch >> 1) & 1u, abort_flag))) break;
      tc_after();
      for (int cc = 0; cc < l; cc += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 128 + cc), v);
        if (c < l) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int j = cc + i;
            if (j >= c && j < l) acc[j * (j + 1) / 2 + c] += v[i];
          }
        }
      }
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
    // upper triangle only (coalesced); the lower one is left unset
    float* pz = part + (int64_t)blockIdx.x * l * l;
    if (c < l)
      for (int j = c; j < l; ++j)
        pz[c + (int64_t)j * l] = *abort_flag ? 0.f : acc[j * (j + 1) / 2 + c];
  }
  __syncwarp();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  tc_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// First Y-pass of the 16-bit forms fused with the down-conversion of an FP32
// S: TMA stages the FP32 tile (128 rows x 64 snapshots as four {32, 64} SW128
// boxes), warps 2-5 convert it into the MN-major 16-bit SW128 tile the MMA
// reads (two {64, 64} atoms) and store the same 16-bit values to the global
// copy Sh that the later passes read, warp 1 issues the MMAs.  S is read from
// HBM once for both the product and the copy.
template <int STAGES>
struct YcvtSmem {
  static constexpr uint32_t A_BYTES = 128 * 128;  // A^T tile, 128 x 64 16-bit
  static constexpr uint32_t F_BYTES = 128 * 256;  // FP32 S tile, 128 rows x 64
  static constexpr uint32_t H_BYTES = 128 * 128;  // 16-bit S tile
  static constexpr uint32_t STAGE = A_BYTES + F_BYTES + H_BYTES;
  static constexpr uint32_t BARS = STAGES * STAGE;
  static constexpr size_t TOTAL = 1024 + (size_t)STAGES * STAGE + 256;
};

template <typename TH> __device__ __forceinline__ uint32_t pack16x2(float a, float b);
template <> __device__ __forceinline__ uint32_t pack16x2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}
template <> __device__ __forceinline__ uint32_t pack16x2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// blockIdx.y: a chunk of kchunk 64-snapshot k-tiles, summed into
// Y + y * ysplit, as in k_ypass.
template <int KIND, int STAGES>
__global__ void __launch_bounds__(192, 1)
k_ypass_cvt(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmF,
            int64_t n, int64_t m, int l, float* __restrict__ Y, int64_t ldy, void* __restrict__ Sh,
            int64_t ldh, unsigned* status, int kchunk, int64_t ysplit, int64_t tile0,
            int64_t yrow0) {
  using L = YcvtSmem<STAGES>;
  using TH = typename std::conditional<KIND == 0, __nv_bfloat16, __half>::type;
  constexpr int BN = 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align_smem1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + L::BARS);
  uint64_t* empty = full + STAGES;
  uint64_t* conv = empty + STAGES;
  uint64_t* done = conv + STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (tile0 + (int64_t)blockIdx.x) * BN;
  const int nk_all = (int)((m + 63) / 64);
  const int kt0 = (int)blockIdx.y * kchunk;
  const int nk = min(nk_all, kt0 + kchunk) - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, BN);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    for (int j = 0; j < nk; ++j) {
      const int s = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (j >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
      const int it = kt0 + j;
      uint8_t* a = smem + s * L::STAGE;
      mbar_expect_tx(&full[s], L::A_BYTES + L::F_BYTES);
      tma_load_2d(a, &tmA, &full[s], it * 64, 0);
#pragma unroll
      for (int b = 0; b < 4; ++b)
        tma_load_2d(a + L::A_BYTES + b * 8192, &tmF, &full[s], (int)(i0 + 32 * b), it * 64);
    }
  } else if (warp >= 2) {
    // item = (row group rg of 8 rows, snapshot kk): 16 x 64 items per stage
    const int ct = threadIdx.x - 64;
    TH* shg = (TH*)Sh;
    bool bad = false;
    for (int j = 0; j < nk; ++j) {
      const int s = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, abort_flag)) break;
      const int it = kt0 + j;
      const uint8_t* f = smem + s * L::STAGE + L::A_BYTES;
      uint8_t* h = smem + s * L::STAGE + L::A_BYTES + L::F_BYTES;
#pragma unroll 2
      for (int i = 0; i < 8; ++i) {
        const int item = ct + 128 * i;
        const int rg = item & 15, kk = item >> 4;
        const int sw = kk & 7;
        const uint8_t* fb = f + (rg >> 2) * 8192 + kk * 128;
        const int c0 = (rg & 3) * 2;
        const float4 x = *(const float4*)(fb + ((c0 ^ sw) << 4));
        const float4 y = *(const float4*)(fb + (((c0 + 1) ^ sw) << 4));
        bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w) &&
                 isfinite(y.x) && isfinite(y.y) && isfinite(y.z) && isfinite(y.w));
        uint4 o;
        o.x = pack16x2<TH>(x.x, x.y);
        o.y = pack16x2<TH>(x.z, x.w);
        o.z = pack16x2<TH>(y.x, y.y);
        o.w = pack16x2<TH>(y.z, y.w);
        *(uint4*)(h + (rg >> 3) * 8192 + kk * 128 + (((rg & 7) ^ sw) << 4)) = o;
        const int64_t r = i0 + 8 * rg, c = (int64_t)it * 64 + kk;
        if (c < m) {
          TH* g = shg + r + c * ldh;
          if (r + 8 <= n) {
            *(uint4*)g = o;
          } else {
            const TH* ov = (const TH*)&o;
            for (int e = 0; e < 8; ++e)
              if (r + e < n) g[e] = ov[e];
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc(fmt_of(KIND), true, 128, BN);
    for (int j = 0; j < nk; ++j) {
      const int s = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (!mbar_wait(&conv[s], ph, abort_flag)) break;
      tc_after();
      const uint32_t a = su32(smem + s * L::STAGE), b = a + L::A_BYTES + L::F_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma<KIND>(tmem, sdesc(a + 32 * kk, 16, 1024), sdesc(b + 2048 * kk, 8192, 1024), id,
                  (j > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  if (warp >= 2) {
    bool ok = mbar_wait(done, 0, abort_flag);
    ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
    tc_after();
    const int q = warp & 3;
    const int c = q * 32 + lane;
    float* ycol = Y + (int64_t)blockIdx.y * ysplit + (int64_t)c * ldy;
    for (int cc = 0; cc < BN; cc += 32) {
      float v[32];
      if (ok) {
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      if (c < l) {
        const int64_t ib = i0 + cc;
        if (((ldy & 3) == 0) && ib + 32 <= n) {
          float4* d4 = (float4*)(ycol + (ib - yrow0));
#pragma unroll
          for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
          for (int i = 0; i < 32; ++i)
            if (ib + i < n) ycol[ib - yrow0 + i] = v[i];
        }
      }
    }
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  tc_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------------------
// CholeskyQR apply Q = Y X (Alg. 1, QR of the sampled matrix) for the
// 16-bit forms: Y n x l FP32 and X l x l FP32 (the inverse Cholesky factor),
// both rounded to TF32 (round to nearest), one kind::tf32 product with FP32
// accumulation.  The rounding of Y (2^-12 relative) is below the BF16
// error of the passes that produced Y, and the basis this apply returns is
// either rounded to BF16 for the next pass or re-orthonormalised by a
// CholeskyQR round on an exact FP32 Gram, so one TF32 product suffices.
// Persistent CTAs over 128-row tiles: warp 0 TMA-loads 128 x 32 column-major
// FP32 tiles of Y (one per 32-column k-block) into a ring of NR raw slots,
// warps 2-9 round them and transpose them into one of NC K-major SW128
// operand tiles (a raw slot is released once read, so up to NR k-blocks
// stay in flight from HBM), warp 1 issues the
// MMAs against X (resident in shared memory as the B operand) into one of two
// TMEM accumulators, and warps 10-17 drain the other accumulator (two warps
// per TMEM lane quarter, one per column half) through shared memory into
// 16-byte stores of any of: Q (FP32), Q rounded to the 16-bit type (the next
// W-pass operand), Q rounded to TF32 (the refinement pass operand).
// SPLIT = 2 (the lift U = Q1 (X2 Uhat) of the returned basis): both operands
// split into TF32 hi and lo parts and three products (lo hi, hi lo, hi hi),
// about 2^-21 relative error per entry.
template <int NR, int NC, int SPLIT>
struct ApplySmem {
  static constexpr uint32_t KB = 128 * 32 * 4;   // 128 rows x 32 columns of FP32
  static constexpr uint32_t RAW = NR * KB;       // TMA ring of raw Y tiles
  static constexpr uint32_t CONV = SPLIT * KB;   // one converted operand tile (all parts)
  static constexpr uint32_t XOP = SPLIT * 4 * KB;  // X parts: 4 k-blocks x 128 (j) x 32 (k)
  static constexpr uint32_t STG = 32 * 32 * 4;     // one epilogue warp's 32 x 32 staging block
  static constexpr uint32_t BARS = RAW + NC * CONV + XOP + 8 * STG;
  static constexpr size_t TOTAL = 1024 + (size_t)BARS + 256;
};

template <int KIND16, int NR, int NC, int SPLIT>
__global__ void __launch_bounds__(576, 1)
k_apply_tf32(const __grid_constant__ CUtensorMap tmY, const float* __restrict__ X, int64_t ldx,
             int64_t n, int l, int ncol, float* __restrict__ Q, int64_t ldq, void* __restrict__ Qh,
             int64_t ldh, float* __restrict__ Qt, int64_t ldt, unsigned* status) {
  using L = ApplySmem<NR, NC, SPLIT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align_smem1024(smem_raw);
  uint8_t* conv_buf = smem + L::RAW;
  uint8_t* xop = conv_buf + NC * L::CONV;
  uint8_t* stage = xop + L::XOP;
  uint64_t* rfull = (uint64_t*)(smem + L::BARS);
  uint64_t* rempty = rfull + NR;
  uint64_t* cfull = rempty + NR;
  uint64_t* cempty = cfull + NC;
  uint64_t* tfull = cempty + NC;    // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* mdone = tempty + 2;
  uint32_t* tslot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (l + 31) / 32;
  const int64_t ntiles = (n + 127) / 128;
  // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int nlt = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);

  if (threadIdx.x == 0) {
    // converter warps per k-block: four of two groups, or all eight
    constexpr uint32_t CW = NC >= 2 ? 4 : 8;
    for (int s = 0; s < NR; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], CW);
    }
    for (int c = 0; c < NC; ++c) {
      mbar_init(&cfull[c], CW);
      mbar_init(&cempty[c], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  // X as the B operand (N = j, K = k), K-major SW128, rounded to TF32, zero
  // outside l x l; eight loads per thread in flight before their stores
  if (warp >= 2 && warp < 10) {
    const int ct = threadIdx.x - 64;
    const bool vec = (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0;
#pragma unroll 1
    for (int e0 = 0; e0 < 4 * 128 * 8; e0 += 256 * 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * 256 + ct;
        const int j = (e >> 3) & 127, k = (e >> 10) * 32 + 4 * (e & 7);
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < ncol && k < l) {
          const float* xc = X + (int64_t)j * ldx + k;
          if (vec) {
            v[u] = *reinterpret_cast<const float4*>(xc);
          } else {
            v[u].x = xc[0];
            if (k + 1 < l) v[u].y = xc[1];
            if (k + 2 < l) v[u].z = xc[2];
            if (k + 3 < l) v[u].w = xc[3];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * 256 + ct;
        const int kb = e >> 10, j = (e >> 3) & 127, c4 = e & 7;
        const float4 r = make_float4(tf32_rna(v[u].x), tf32_rna(v[u].y), tf32_rna(v[u].z),
                                     tf32_rna(v[u].w));
        const uint32_t off = kb * L::KB + (j >> 3) * 1024 + (j & 7) * 128 + ((c4 ^ (j & 7)) << 4);
        *(float4*)(xop + off) = r;
        if (SPLIT == 2)
          *(float4*)(xop + 4 * L::KB + off) =
              make_float4(tf32_rna(v[u].x - r.x), tf32_rna(v[u].y - r.y), tf32_rna(v[u].z - r.z),
                          tf32_rna(v[u].w - r.w));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, 256);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    int it = 0;  // loads issued
    bool go = true;
    for (int lt = 0; lt < nlt && go; ++lt) {
      const int64_t t = blockIdx.x + (int64_t)lt * gridDim.x;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = it % NR;
        const uint32_t ph = (uint32_t)(it / NR) & 1u;
        if (it >= NR && !mbar_wait(&rempty[s], ph ^ 1u, abort_flag)) { go = false; break; }
        mbar_expect_tx(&rfull[s], L::KB);
        tma_load_2d(smem + s * L::KB, &tmY, &rfull[s], (int)(t * 128), kb * 32);
        ++it;
      }
    }
    // on an abort, wait (bounded) for the copies still in flight
    if (*abort_flag)
      for (int i2 = it > NR ? it - NR : 0; i2 < it; ++i2)
        mbar_wait_drain(&rfull[i2 % NR], (uint32_t)(i2 / NR) & 1u);
  } else if (warp >= 2 && warp < 10) {
    // converters (eight warps): raw tile s of the ring -> operand tile c;
    // the raw slot is released as soon as it is read, so the loads run NR
    // k-blocks ahead of the conversions and the MMAs.  Thread (c4, mq)
    // takes the 4 x 4 block of rows 4 mq .. + 3 and columns 4 c4 .. + 3:
    // four 16-byte loads down the columns, a transpose in registers, four
    // 16-byte stores along the rows of the K-major operand.  The rows are
    // stored in a lane-rotated order, so that the eight lanes of each store
    // phase cover all eight row residues mod 8 and hence eight distinct
    // swizzled 16-byte bank groups.
    // With two operand tiles (NC = 2) two groups of four warps take
    // alternate k-blocks, so that two conversions are in flight, and each
    // thread converts two 4 x 4 blocks; each operand tile and raw slot then
    // belongs to one group, whose waits on its barriers follow the phases in
    // order.  With one operand tile a single group of eight warps converts
    // every k-block (two groups waiting on one barrier could each see a phase
    // two ahead of the barrier as complete).
    constexpr int NG = NC >= 2 ? 2 : 1;
    static_assert(NG == 1 || (NC % 2 == 0 && NR % 2 == 0), "a slot per converter group");
    const int ct = threadIdx.x - 64;
    const int grp = ct / (256 / NG), gt = ct % (256 / NG);
    const int c4 = gt >> 5, mq = gt & 31;
    bool go = true;
    for (int lt = 0, it = 0; lt < nlt && go; ++lt)
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        if (it % NG != grp) continue;
        const int s = it % NR, c = it % NC;
        const uint32_t ph = (uint32_t)(it / NR) & 1u, phc = (uint32_t)(it / NC) & 1u;
        bool ok = mbar_wait(&rfull[s], ph, abort_flag);
        if (ok && it >= NC) ok = mbar_wait(&cempty[c], phc ^ 1u, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) { go = false; break; }
        const float* raw = (const float*)(smem + s * L::KB);  // column k at k * 128
        uint8_t* aop = conv_buf + c * L::CONV;
#pragma unroll
        for (int h = 0; h < NG; ++h) {
          const int cb = c4 + (8 / NG) * h;  // column block 4 cb .. 4 cb + 3
          float4 col[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            col[i] = *reinterpret_cast<const float4*>(raw + (4 * cb + i) * 128 + 4 * mq);
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const int r = (rr + (lane >> 1)) & 3;
            const float4 x = make_float4(pick4(col[0], r), pick4(col[1], r), pick4(col[2], r),
                                         pick4(col[3], r));
            const int m = 4 * mq + r;
            const float4 v = make_float4(tf32_rna(x.x), tf32_rna(x.y), tf32_rna(x.z), tf32_rna(x.w));
            const uint32_t off = (m >> 3) * 1024 + (m & 7) * 128 + ((cb ^ (m & 7)) << 4);
            *(float4*)(aop + off) = v;
            if (SPLIT == 2)
              *(float4*)(aop + L::KB + off) = make_float4(tf32_rna(x.x - v.x), tf32_rna(x.y - v.y),
                                                          tf32_rna(x.z - v.z), tf32_rna(x.w - v.w));
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&rempty[s]);
          mbar_arrive(&cfull[c]);
        }
      }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc(2, false, 128, 128);
    bool go = true, issued = false;
    for (int lt = 0, it = 0; lt < nlt && go; ++lt) {
      const int buf = lt & 1;
      if (lt >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((lt >> 1) - 1) & 1u, abort_flag)) break;
      tc_after();
      const uint32_t d = tmem + (uint32_t)(buf * 128);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int c = it % NC;
        const uint32_t phc = (uint32_t)(it / NC) & 1u;
        if (!mbar_wait(&cfull[c], phc, abort_flag)) { go = false; break; }
        tc_after();
        const uint32_t a = su32(conv_buf + c * L::CONV), b = su32(xop + kb * L::KB);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
          if (SPLIT == 2) {
            // smallest terms first: lo hi, hi lo, then hi hi
            mma<2>(d, sdesc(a + L::KB + 32 * kk, 16, 1024), sdesc(b + 32 * kk, 16, 1024), id, acc0);
            mma<2>(d, sdesc(a + 32 * kk, 16, 1024), sdesc(b + 4 * L::KB + 32 * kk, 16, 1024), id, 1u);
            mma<2>(d, sdesc(a + 32 * kk, 16, 1024), sdesc(b + 32 * kk, 16, 1024), id, 1u);
          } else {
            mma<2>(d, sdesc(a + 32 * kk, 16, 1024), sdesc(b + 32 * kk, 16, 1024), id, acc0);
          }
        }
        mma_commit(&cempty[c]);
        issued = true;
      }
      if (go) mma_commit(&tfull[buf]);
    }
    // every MMA of this CTA complete before the accumulators are freed
    if (issued) {
      mma_commit(mdone);
      mbar_wait_drain(mdone, 0);
    }
  } else if (warp >= 10) {
    // eight epilogue warps: warp w reads TMEM lane quarter w % 4 (rows
    // 32 (w % 4) .. + 31 of the tile) and one half of the columns.  Each
    // 32 x 32 block goes through this warp's staging buffer (column j of the
    // block at j * 32) and leaves as 16-byte stores along the rows of a
    // column: 4 (FP32) or 8 (16-bit) rows per lane, so one store instruction
    // writes 4 or 8 whole 128- or 64-byte column segments instead of 32
    // two- or four-byte pieces
    const int q = warp & 3;
    const int half = (warp - 10) >> 2;
    float* stg = reinterpret_cast<float*>(stage + (warp - 10) * L::STG);
    __nv_bfloat16* stgb = reinterpret_cast<__nv_bfloat16*>(stg);
    __half* stgh = reinterpret_cast<__half*>(stg);
    // 16-byte stores need 16-byte aligned columns
    const bool vq = Q && ((uintptr_t)Q & 15) == 0 && (ldq & 3) == 0;
    const bool vt = Qt && ((uintptr_t)Qt & 15) == 0 && (ldt & 3) == 0;
    const bool vh = Qh && ((uintptr_t)Qh & 15) == 0 && (ldh & 7) == 0;
    for (int lt = 0; lt < nlt; ++lt) {
      const int buf = lt & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], (uint32_t)(lt >> 1) & 1u, abort_flag));
      if (!ok) break;
      tc_after();
      const int64_t t = blockIdx.x + (int64_t)lt * gridDim.x;
      const int64_t m0 = t * 128 + q * 32;  // first row of this warp's block
      const int64_t m = m0 + lane;
      const bool full = m0 + 32 <= n;
      for (int cc = 64 * half; cc < ncol && cc < 64 * half + 64; cc += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 128 + cc), v);
        const int nc = ncol - cc < 32 ? ncol - cc : 32;
        // FP32 outputs: Q, then Q rounded to TF32
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          float* out = o == 0 ? Q : Qt;
          const int64_t ld = o == 0 ? ldq : ldt;
          if (!out) continue;
          if (full && (o == 0 ? vq : vt)) {
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 32; ++i) stg[i * 32 + lane] = o == 0 ? v[i] : tf32_rna(v[i]);
            __syncwarp();
            // lane: column cl = lane / 8 + 4 u, rows 4 (lane % 8) .. + 3
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int cl = (lane >> 3) + 4 * u;
              if (cl < nc)
                *reinterpret_cast<float4*>(out + m0 + 4 * (lane & 7) + (int64_t)(cc + cl) * ld) =
                    *reinterpret_cast<const float4*>(stg + cl * 32 + 4 * (lane & 7));
            }
          } else if (m < n) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < nc) out[m + (int64_t)(cc + i) * ld] = o == 0 ? v[i] : tf32_rna(v[i]);
          }
        }
        // Q rounded to the 16-bit type
        if (Qh) {
          if (full && vh) {
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if (KIND16 == 0)
                stgb[i * 32 + lane] = __float2bfloat16_rn(v[i]);
              else
                stgh[i * 32 + lane] = __float2half_rn(v[i]);
            }
            __syncwarp();
            // lane: column cl = lane / 4 + 8 u, rows 8 (lane % 4) .. + 7
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int cl = (lane >> 2) + 8 * u;
              if (cl < nc)
                *reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(Qh) + m0 + 8 * (lane & 3) +
                                          (int64_t)(cc + cl) * ldh) =
                    *reinterpret_cast<const uint4*>(reinterpret_cast<const uint16_t*>(stg) +
                                                    cl * 32 + 8 * (lane & 3));
            }
          } else if (m < n) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if (i < nc) {
                if (KIND16 == 0)
                  ((__nv_bfloat16*)Qh)[m + (int64_t)(cc + i) * ldh] = __float2bfloat16_rn(v[i]);
                else
                  ((__half*)Qh)[m + (int64_t)(cc + i) * ldh] = __float2half_rn(v[i]);
              }
            }
          }
        }
      }
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  __syncwarp();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  tc_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// host side
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

CUtensorMapDataType tmap_type(int dt) {
  switch (dt) {
    case RPOD_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    case RPOD_F16: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  }
}

int esize(int dt) { return (dt == RPOD_BF16 || dt == RPOD_F16) ? 2 : 4; }

// 2-D column-major matrix (rows contiguous): dims {rows, cols}, box {br, bc}.
int make_map(CUtensorMap* map, const void* ptr, int dt, int64_t rows, int64_t cols, int64_t ld,
             int br, int bc, bool swizzle = true) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return RPOD_ERR_CUDA;
  const int es = esize(dt);
  if (((uintptr_t)ptr & 15) || ((ld * es) & 15)) return RPOD_ERR_UNSUPPORTED;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)br, (cuuint32_t)bc};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, tmap_type(dt), 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RPOD_OK : RPOD_ERR_CUDA;
}

constexpr int kBN = 256;
constexpr int kStages = 4;
// passes over less than 1 GiB (the instances of a batch) use two stages
// (96 KB): two CTAs, of one pass or of two instances' passes, share an SM
// and hide each other's pipeline fill and drain
constexpr int kStagesSmall = 2;
constexpr size_t kSmallPassBytes = (size_t)1 << 30;
constexpr int kGramStages = 3;  // 96 KB: two CTAs per SM
constexpr int kYcvtStages = 3;  // 192 KB
constexpr int kGramXStages = 3;  // 144 KB of stages + 33 KB of sums
// apply: raw TMA slots and operand tiles (224 KB with X and the epilogue's
// 32 KB of staging in both forms)
constexpr int kApplyRaw = 6, kApplyConv = 2;    // 96 + 32 KB + 64 KB for X
constexpr int kApply2Raw = 2, kApply2Conv = 1;  // two-part form: 32 + 32 KB + 128 KB for X

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      n = 152;
  }
  return n;
}

}  // namespace

void prepare_kernels_tc() {
  static std::once_flag once;
  std::call_once(once, [] {
    using L = tc::Smem<kBN, kStages>;
    const int b = (int)L::TOTAL;
    cudaFuncSetAttribute(tc::k_wpass<0, kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(tc::k_wpass<1, kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(tc::k_wpass<2, kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(tc::k_ypass<0, kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(tc::k_ypass<1, kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    const int bs = (int)tc::Smem<kBN, kStagesSmall>::TOTAL;
    cudaFuncSetAttribute(tc::k_wpass<0, kBN, kStagesSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize, bs);
    cudaFuncSetAttribute(tc::k_wpass<1, kBN, kStagesSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize, bs);
    cudaFuncSetAttribute(tc::k_wpass<2, kBN, kStagesSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize, bs);
    cudaFuncSetAttribute(tc::k_ypass<0, kBN, kStagesSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize, bs);
    cudaFuncSetAttribute(tc::k_ypass<1, kBN, kStagesSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize, bs);
    cudaFuncSetAttribute(tc::k_gram3<kGramStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc::GramSmem<kGramStages>::TOTAL);
    cudaFuncSetAttribute(tc::k_gram_x<kGramXStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc::GramXSmem<kGramXStages>::TOTAL);
    const int yc = (int)tc::YcvtSmem<kYcvtStages>::TOTAL;
    cudaFuncSetAttribute(tc::k_ypass_cvt<0, kYcvtStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, yc);
    cudaFuncSetAttribute(tc::k_ypass_cvt<1, kYcvtStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, yc);
    const int ap = (int)tc::ApplySmem<kApplyRaw, kApplyConv, 1>::TOTAL;
    cudaFuncSetAttribute(tc::k_apply_tf32<0, kApplyRaw, kApplyConv, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, ap);
    cudaFuncSetAttribute(tc::k_apply_tf32<1, kApplyRaw, kApplyConv, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, ap);
    const int ap2 = (int)tc::ApplySmem<kApply2Raw, kApply2Conv, 2>::TOTAL;
    cudaFuncSetAttribute(tc::k_apply_tf32<0, kApply2Raw, kApply2Conv, 2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, ap2);
  });
}

int tc_wpass_splits(int64_t n, int64_t m, int dt) {
  const int bke = esize(dt) == 2 ? 64 : 32;
  const int64_t ktiles = (n + bke - 1) / bke;
  const int64_t cols = (m + kBN - 1) / kBN;
  // aim for about five waves of 152 SMs, at least 16 k-tiles per split
  int64_t s = (5 * 152 + cols - 1) / cols;
  if (s > ktiles / 16) s = ktiles / 16;
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return (int)s;
}

int tc_wpass(cudaStream_t st, int dt, const void* A, int64_t lda, int64_t n, int l, const void* S,
             int64_t lds, int64_t m, float* part, int nsplit, unsigned* status, int stages) {
  CUtensorMap ta, ts;
  const int bke = esize(dt) == 2 ? 64 : 32;
  if (int rc = make_map(&ta, A, dt, n, l, lda, bke, 128)) return rc;
  if (int rc = make_map(&ts, S, dt, n, m, lds, bke, kBN)) return rc;
  const int64_t ktiles = (n + bke - 1) / bke;
  const int kchunk = (int)((ktiles + nsplit - 1) / nsplit);
  dim3 grid((unsigned)((m + kBN - 1) / kBN), (unsigned)nsplit);
  prepare_kernels_tc();
  const bool small = stages == 2 || (stages != 4 && (size_t)n * (size_t)m * (size_t)esize(dt) < kSmallPassBytes);
  using L = tc::Smem<kBN, kStages>;
  using Ls = tc::Smem<kBN, kStagesSmall>;
  const unsigned nt = dt == RPOD_F32 ? 192 : 128;
  if (small) {
    switch (dt) {
      case RPOD_BF16:
        tc::k_wpass<0, kBN, kStagesSmall><<<grid, nt, Ls::TOTAL, st>>>(ta, ts, n, m, l, kchunk, part, status);
        break;
      case RPOD_F16:
        tc::k_wpass<1, kBN, kStagesSmall><<<grid, nt, Ls::TOTAL, st>>>(ta, ts, n, m, l, kchunk, part, status);
        break;
      default:
        tc::k_wpass<2, kBN, kStagesSmall><<<grid, nt, Ls::TOTAL, st>>>(ta, ts, n, m, l, kchunk, part, status);
        break;
    }
  } else {
    switch (dt) {
      case RPOD_BF16:
        tc::k_wpass<0, kBN, kStages><<<grid, nt, L::TOTAL, st>>>(ta, ts, n, m, l, kchunk, part, status);
        break;
      case RPOD_F16:
        tc::k_wpass<1, kBN, kStages><<<grid, nt, L::TOTAL, st>>>(ta, ts, n, m, l, kchunk, part, status);
        break;
      default:
        tc::k_wpass<2, kBN, kStages><<<grid, nt, L::TOTAL, st>>>(ta, ts, n, m, l, kchunk, part, status);
        break;
    }
  }
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}

// Chunks of snapshots for a Y-pass whose row tiles cannot fill the GPU (a
// standalone pass over a matrix with few rows and many snapshots, e.g. the
// paper's 8192 grid cells x 90225 snapshots): the smallest count that gives
// at least two waves of CTAs with the last wave at least 85 % full, each
// chunk at least 8 k-tiles.  1 for batch-instance-sized passes (other
// instances fill the GPU) and for matrices with enough rows.
int ypass_split(int64_t row_tiles, int64_t m, size_t pass_bytes, int ctas_per_sm) {
  if (pass_bytes < kSmallPassBytes) return 1;
  const int64_t slots = (int64_t)sm_count() * ctas_per_sm;
  if (row_tiles >= 2 * slots) return 1;
  const int64_t nk = (m + 63) / 64;
  int best = 1;
  for (int ns = 2; ns <= 32 && nk / ns >= 8; ++ns) {
    const int64_t total = row_tiles * ns;
    const int64_t waves = (total + slots - 1) / slots;
    best = ns;
    if (total >= 2 * slots && (double)total / (double)(waves * slots) >= 0.85) break;
  }
  return best;
}

// Chunk layout of a split Y-pass: kchunk k-tiles per chunk, ns chunks with
// none empty; 1 chunk when the partial buffer cannot hold ns slices.
void ypass_chunks(int64_t m, int want, size_t slice_elems, size_t part_elems, int* ns, int* kchunk) {
  const int nk = (int)((m + 63) / 64);
  int s = want;
  if ((size_t)s * slice_elems > part_elems) s = 1;
  int kc = (nk + s - 1) / s;
  s = (nk + kc - 1) / kc;
  *ns = s;
  *kchunk = kc;
}

// Work layout of a Y-pass over `tiles` row tiles that is not split over the
// snapshots: whole waves of tiles in one launch, and -- when the last wave
// would fill at most 60 % of the GPU, so that fewer than that many SMs draw
// on HBM while it runs -- the last tiles alone in a second launch, each split
// over the snapshots into the chunk count that leaves the fewest partly
// filled waves (partials in `part`, summed into Y after).
struct YTail {
  int64_t full = 0;  // tiles of the first launch (all tiles when no tail launch)
  int nst = 1;       // snapshot chunks of each tail tile (1: no tail launch)
  int kchunk = 0;    // 64-snapshot k-tiles per chunk
};

YTail ypass_tail(int64_t tiles, int64_t m, int64_t rows_per_tile, int64_t n, int l, int per_wave,
                 const float* part, size_t part_elems) {
  YTail t;
  t.full = tiles;
  const int64_t full = tiles / per_wave * per_wave, tail = tiles - full;
  if (!part || full == 0 || tail == 0 || tail * 10 > (int64_t)per_wave * 6) return t;
  const int nk = (int)((m + 63) / 64);
  int best = 1;
  double best_w = 1.0;
  for (int s = 2; s <= 8 && s <= nk; ++s) {
    const double w = (double)((tail * s + per_wave - 1) / per_wave) / s;
    if (w < best_w - 1e-9) { best_w = w; best = s; }
  }
  if (best == 1) return t;
  const int kc = (nk + best - 1) / best;
  best = (nk + kc - 1) / kc;
  const int64_t trows = n - full * rows_per_tile;
  if ((size_t)best * (size_t)trows * (size_t)l > part_elems) return t;
  t.full = full;
  t.nst = best;
  t.kchunk = kc;
  return t;
}

int tc_ypass(cudaStream_t st, int dt, const void* A, int64_t lda, const void* S, int64_t lds,
             int64_t n, int64_t m, int l, float* Y, int64_t ldy, unsigned* status, float* part,
             size_t part_elems, int stages) {
  if (dt != RPOD_BF16 && dt != RPOD_F16) return RPOD_ERR_UNSUPPORTED;
  CUtensorMap ta, ts;
  if (int rc = make_map(&ta, A, dt, m, l, lda, 64, 128)) return rc;
  if (int rc = make_map(&ts, S, dt, n, m, lds, 64, 64)) return rc;
  const int64_t tiles = (n + kBN - 1) / kBN;
  const size_t bytes = (size_t)n * (size_t)m * 2;
  int ns = 1, kchunk = 0;
  ypass_chunks(m, part ? ypass_split(tiles, m, bytes, 1) : 1, (size_t)n * l, part_elems, &ns, &kchunk);
  prepare_kernels_tc();
  const bool small = stages == 2 || (stages != 4 && bytes < kSmallPassBytes);
  using L = tc::Smem<kBN, kStages>;
  using Ls = tc::Smem<kBN, kStagesSmall>;
  auto launch = [&](int64_t ntile, int nsy, int64_t tile0, float* out, int64_t ldo, int64_t ysplit,
                    int kc) {
    dim3 grid((unsigned)ntile, (unsigned)nsy);
    if (small) {
      if (dt == RPOD_BF16)
        tc::k_ypass<0, kBN, kStagesSmall><<<grid, 128, Ls::TOTAL, st>>>(
            ta, ts, n, m, l, out, ldo, status, kc, ysplit, tile0, tile0 * kBN);
      else
        tc::k_ypass<1, kBN, kStagesSmall><<<grid, 128, Ls::TOTAL, st>>>(
            ta, ts, n, m, l, out, ldo, status, kc, ysplit, tile0, tile0 * kBN);
    } else {
      if (dt == RPOD_BF16)
        tc::k_ypass<0, kBN, kStages><<<grid, 128, L::TOTAL, st>>>(
            ta, ts, n, m, l, out, ldo, status, kc, ysplit, tile0, tile0 * kBN);
      else
        tc::k_ypass<1, kBN, kStages><<<grid, 128, L::TOTAL, st>>>(
            ta, ts, n, m, l, out, ldo, status, kc, ysplit, tile0, tile0 * kBN);
    }
    note_launch();
    return cudaGetLastError() == cudaSuccess;
  };
  if (ns > 1) {
    if (!launch(tiles, ns, 0, part, n, n * l, kchunk)) return RPOD_ERR_CUDA;
    if (reduce_splits<float, float>(st, n, l, ns, part, Y, 1, ldy) != cudaSuccess) return RPOD_ERR_CUDA;
    return RPOD_OK;
  }
  const YTail t = ypass_tail(tiles, m, kBN, n, l, sm_count() * (small ? 2 : 1), part, part_elems);
  if (!launch(t.full, 1, 0, Y, ldy, 0, kchunk)) return RPOD_ERR_CUDA;
  if (t.nst > 1) {
    const int64_t trows = n - t.full * kBN;
    if (!launch(tiles - t.full, t.nst, t.full, part, trows, trows * l, t.kchunk)) return RPOD_ERR_CUDA;
    if (reduce_splits<float, float>(st, trows, l, t.nst, part, Y + t.full * kBN, 1, ldy) != cudaSuccess)
      return RPOD_ERR_CUDA;
  }
  return RPOD_OK;
}

int tc_gram(cudaStream_t st, const float* Y, int64_t ldy, int64_t rows, int l, float* part,
            int nsplit, unsigned* status, bool exact) {
  if (l < 1 || l > 128 || rows < 1 || nsplit < 1) return RPOD_ERR_INVALID_ARG;
  CUtensorMap ty;
  if (int rc = make_map(&ty, Y, RPOD_F32, rows, l, ldy, 32, 128)) return rc;
  const int64_t ktiles = (rows + 31) / 32;
  const int kchunk = (int)((ktiles + nsplit - 1) / nsplit);
  prepare_kernels_tc();
  if (exact)
    tc::k_gram_x<kGramXStages><<<(unsigned)nsplit, 320, tc::GramXSmem<kGramXStages>::TOTAL, st>>>(
        ty, rows, l, kchunk, part, status);
  else
    tc::k_gram3<kGramStages><<<(unsigned)nsplit, 192, tc::GramSmem<kGramStages>::TOTAL, st>>>(
        ty, rows, l, kchunk, part, status);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}

int tc_ypass_cvt(cudaStream_t st, int dt, const void* A, int64_t lda, const float* S, int64_t lds,
                 int64_t n, int64_t m, int l, float* Y, int64_t ldy, void* Sh, int64_t ldh,
                 unsigned* status, float* part, size_t part_elems) {
  if (dt != RPOD_BF16 && dt != RPOD_F16) return RPOD_ERR_UNSUPPORTED;
  if (((uintptr_t)Sh & 15) || (ldh & 7)) return RPOD_ERR_UNSUPPORTED;
  CUtensorMap ta, tf;
  if (int rc = make_map(&ta, A, dt, m, l, lda, 64, 128)) return rc;
  if (int rc = make_map(&tf, S, RPOD_F32, n, m, lds, 32, 64)) return rc;
  constexpr int64_t BN = 128;
  const int64_t tiles = (n + BN - 1) / BN;
  int ns = 1, kchunk = 0;
  ypass_chunks(m, part ? ypass_split(tiles, m, (size_t)n * (size_t)m * 4, 1) : 1, (size_t)n * l,
               part_elems, &ns, &kchunk);
  using L = tc::YcvtSmem<kYcvtStages>;
  prepare_kernels_tc();
  auto launch = [&](int64_t ntile, int nsy, int64_t tile0, float* out, int64_t ldo, int64_t ysplit,
                    int kc) {
    dim3 grid((unsigned)ntile, (unsigned)nsy);
    if (dt == RPOD_BF16)
      tc::k_ypass_cvt<0, kYcvtStages><<<grid, 192, L::TOTAL, st>>>(
          ta, tf, n, m, l, out, ldo, Sh, ldh, status, kc, ysplit, tile0, tile0 * BN);
    else
      tc::k_ypass_cvt<1, kYcvtStages><<<grid, 192, L::TOTAL, st>>>(
          ta, tf, n, m, l, out, ldo, Sh, ldh, status, kc, ysplit, tile0, tile0 * BN);
    note_launch();
    return cudaGetLastError() == cudaSuccess;
  };
  if (ns > 1) {
    if (!launch(tiles, ns, 0, part, n, n * l, kchunk)) return RPOD_ERR_CUDA;
    if (reduce_splits<float, float>(st, n, l, ns, part, Y, 1, ldy) != cudaSuccess) return RPOD_ERR_CUDA;
    return RPOD_OK;
  }
  const YTail t = ypass_tail(tiles, m, BN, n, l, sm_count(), part, part_elems);
  if (!launch(t.full, 1, 0, Y, ldy, 0, kchunk)) return RPOD_ERR_CUDA;
  if (t.nst > 1) {
    const int64_t trows = n - t.full * BN;
    if (!launch(tiles - t.full, t.nst, t.full, part, trows, trows * l, t.kchunk)) return RPOD_ERR_CUDA;
    if (reduce_splits<float, float>(st, trows, l, t.nst, part, Y + t.full * BN, 1, ldy) != cudaSuccess)
      return RPOD_ERR_CUDA;
  }
  return RPOD_OK;
}

int tc_sm_count() { return sm_count(); }

int tc_apply(cudaStream_t st, const float* Y, int64_t ldy, int64_t n, int l, const float* X,
             int64_t ldx, float* Q, int64_t ldq, int dt16, void* Qh, int64_t ldh, float* Qt,
             int64_t ldt, unsigned* status, int ncol, bool precise) {
  if (ncol == 0) ncol = l;
  if (l < 1 || l > 128 || ncol < 1 || ncol > 128 || n < 1 || ldx < l) return RPOD_ERR_INVALID_ARG;
  if (Qh && dt16 != RPOD_BF16 && dt16 != RPOD_F16) return RPOD_ERR_INVALID_ARG;
  if (precise && (Qh || Qt)) return RPOD_ERR_INVALID_ARG;
  if ((Q && ldq < n) || (Qh && ldh < n) || (Qt && ldt < n)) return RPOD_ERR_INVALID_ARG;
  CUtensorMap ty;
  if (int rc = make_map(&ty, Y, RPOD_F32, n, l, ldy, 128, 32, false)) return rc;
  const int64_t ntiles = (n + 127) / 128;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sm_count());
  prepare_kernels_tc();
  using L1 = tc::ApplySmem<kApplyRaw, kApplyConv, 1>;
  using L2 = tc::ApplySmem<kApply2Raw, kApply2Conv, 2>;
  if (precise)
    tc::k_apply_tf32<0, kApply2Raw, kApply2Conv, 2><<<grid, 576, L2::TOTAL, st>>>(
        ty, X, ldx, n, l, ncol, Q, ldq, Qh, ldh, Qt, ldt, status);
  else if (dt16 == RPOD_F16)
    tc::k_apply_tf32<1, kApplyRaw, kApplyConv, 1><<<grid, 576, L1::TOTAL, st>>>(
        ty, X, ldx, n, l, ncol, Q, ldq, Qh, ldh, Qt, ldt, status);
  else
    tc::k_apply_tf32<0, kApplyRaw, kApplyConv, 1><<<grid, 576, L1::TOTAL, st>>>(
        ty, X, ldx, n, l, ncol, Q, ldq, Qh, ldh, Qt, ldt, status);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}

}  // namespace rpod
