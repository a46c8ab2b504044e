// Persistent LSTM rollout (the online stage of Sec. 4.3): autoregressive
// prediction of `steps` coefficient vectors in one cooperative launch.
//
// The network maps a window of T rows [mu, alpha] to the next alpha, with
// zero initial states for every window, so each prediction runs L x T cells.
// One CTA owns U consecutive hidden units of every layer: the 4U gate rows
// of W_x and W_h (widened to FP32 from the weights the products read), the
// biases, and the cell states of its units stay in shared memory for the
// whole rollout.  Cell (l, t) needs h(l, t - 1) and h(l - 1, t), so the cells
// of one anti-diagonal l + t run in the same phase: L + T - 1 phases per
// prediction, each ended by a grid barrier, then the linear head (rows of
// W_y spread over the CTAs) writes the prediction into a ring buffer of
// window rows, which replaces the oldest row, and a last barrier.
//
// Grid barrier: a monotonic arrival counter in the workspace; a CTA arrives
// (after a device-scope fence) and its first thread waits for the count of
// the barrier with a 2 s %globaltimer limit.  A wait that runs out records
// ST_TIMEOUT, raises an abort word that every waiting CTA checks, and the
// kernel returns; nothing waits without a limit.
#include <cooperative_groups.h>

#include "rpod_internal.cuh"

namespace rpod {
namespace {

constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier number k (0, 1, 2, ...) over gridDim.x CTAs: false when a
// wait ran out (here or in another CTA).
__device__ bool grid_sync(unsigned* count, unsigned k, volatile int* abort_word, unsigned* status,
                          uint64_t limit_ns, bool arrive = true) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    if (arrive) atomicAdd(count, 1u);
    const unsigned target = (k + 1) * gridDim.x;
    const uint64_t t0 = gtimer();
    while (*(volatile unsigned*)count < target) {
      if (*abort_word) {
        ok = 0;
        break;
      }
      if (gtimer() - t0 > limit_ns) {
        atomicOr(status, ST_TIMEOUT);
        *abort_word = 1;
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ float sigm_r(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float wld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float wld(const float* p) { return *p; }

struct RollArgs {
  int I, H, L, O, T, B, d, U, steps;
  const float* theta;          // FP32 parameters (biases, and weights when TW = float)
  const void* wbf;             // weight copies the products read (BF16) or theta
  int64_t off_w[4][3];         // per layer: W_x, W_h, b offsets into the flat vector
  int64_t off_wy, off_by;
  float* ring;                 // T x B x I window rows (ring buffer), time-major
  float* hbuf;                 // L x T x B x H hidden states of the current window
  float* out;                  // B x steps x O predictions
  unsigned* count;             // barrier arrivals (zeroed by the host)
  int* abort_word;
  unsigned* status;
};

// Dynamic shared memory per CTA: for every layer the 4U gate rows of
// [W_x | W_h] (K_l = I_l + H floats, stride K_l + 1), 4U biases, U x B cell
// states; the gathered inputs [x | h_prev] of the phase's cells (B x (I + H)
// per cell, two cells at most in flight per layer) reuse one staging area
// per layer; the gate pre-activations (4U x B per layer); W_y rows of the
// outputs this CTA computes.
__host__ __device__ inline size_t roll_smem_floats(int I, int H, int L, int O, int B, int U, int G) {
  size_t f = 0;
  for (int l = 0; l < L; ++l) {
    const int K = (l == 0 ? I : H) + H;
    f += (size_t)4 * U * (K + 1) + 4 * U + (size_t)U * B + (size_t)B * (K + 1) + (size_t)4 * U * B;
  }
  const int rows = (O + G - 1) / G;
  f += (size_t)rows * H + rows;
  return f;
}

template <typename TW>
__global__ void __launch_bounds__(512, 1) k_rollout(RollArgs a) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int I = a.I, H = a.H, L = a.L, O = a.O, T = a.T, B = a.B, U = a.U;
  const int G = gridDim.x, cta = blockIdx.x;
  const int u0 = cta * U;
  const TW* W = (const TW*)a.wbf;
  // ---- carve shared memory and load this CTA's rows once
  float* Wl[4];
  float* bl[4];
  float* cl[4];
  float* xl[4];
  float* zl[4];
  float* p = sm;
  for (int l = 0; l < L; ++l) {
    const int Il = l == 0 ? I : H, K = Il + H;
    Wl[l] = p; p += (size_t)4 * U * (K + 1);
    bl[l] = p; p += 4 * U;
    cl[l] = p; p += (size_t)U * B;
    xl[l] = p; p += (size_t)B * (K + 1);  // rows padded: samples of one warp on distinct banks
    zl[l] = p; p += (size_t)4 * U * B;
    for (int e = tid; e < 4 * U * K; e += nt) {
      const int r = e / K, k = e % K;
      const int g = r / U, u = u0 + r % U;
      const int64_t row = (int64_t)g * H + u;
      Wl[l][r * (K + 1) + k] = k < Il ? wld(W + a.off_w[l][0] + row * Il + k)
                                      : wld(W + a.off_w[l][1] + row * H + (k - Il));
    }
    for (int r = tid; r < 4 * U; r += nt) bl[l][r] = a.theta[a.off_w[l][2] + (r / U) * H + u0 + r % U];
  }
  const int yrows = (O + G - 1) / G;
  float* Wy = p; p += (size_t)yrows * H;
  float* byl = p;
  for (int e = tid; e < yrows * H; e += nt) {
    const int r = e / H, k = e % H, o = cta + r * G;
    Wy[e] = o < O ? wld(W + a.off_wy + (int64_t)o * H + k) : 0.f;
  }
  for (int r = tid; r < yrows; r += nt) {
    const int o = cta + r * G;
    byl[r] = o < O ? a.theta[a.off_by + o] : 0.f;
  }
  __syncthreads();

  unsigned bar = 0;
  const volatile int* abort_word = a.abort_word;
  for (int s = 0; s < a.steps; ++s) {
    // the window of this prediction: ring rows (s + t) mod T, t = 0..T-1
    for (int ph = 0; ph < L + T - 1; ++ph) {
      if (*abort_word) return;
      // gather the inputs of this phase's cells (l, t = ph - l): x, h_prev
      for (int l = 0; l < L; ++l) {
        const int t = ph - l;
        if (t < 0 || t >= T) continue;
        const int Il = l == 0 ? I : H, K = Il + H;
        const float* xin = l == 0 ? a.ring + (size_t)((s + t) % T) * B * I
                                  : a.hbuf + ((size_t)(l - 1) * T + t) * B * H;
        const float* hprev = t > 0 ? a.hbuf + ((size_t)l * T + t - 1) * B * H : nullptr;
        // x (B x Il) and h_prev (B x H) are contiguous in global memory: four
        // independent loads in flight per thread, then the padded stores
        for (int e0 = 0; e0 < B * Il; e0 += 4 * nt) {
          float v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int e = e0 + j * nt + tid;
            v[j] = e < B * Il ? __ldcg(xin + e) : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int e = e0 + j * nt + tid;
            if (e < B * Il) xl[l][(e / Il) * (K + 1) + e % Il] = v[j];
          }
        }
        for (int e0 = 0; e0 < B * H; e0 += 4 * nt) {
          float v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int e = e0 + j * nt + tid;
            v[j] = (e < B * H && hprev) ? __ldcg(hprev + e) : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int e = e0 + j * nt + tid;
            if (e < B * H) xl[l][(e / H) * (K + 1) + Il + e % H] = v[j];
          }
        }
        if (t == 0)
          for (int e = tid; e < U * B; e += nt) cl[l][e] = 0.f;
      }
      __syncthreads();
      // gate pre-activations: 4U rows x B samples, 4 threads per dot product
      for (int l = 0; l < L; ++l) {
        const int t = ph - l;
        if (t < 0 || t >= T) continue;
        const int Il = l == 0 ? I : H, K = Il + H;
        const int ndot = 4 * U * B;
        for (int q0 = 0; q0 < ndot * 4; q0 += nt) {
          const int q = q0 + tid;
          const int dot = q >> 2, part = q & 3;
          float acc = 0.f;
          if (dot < ndot) {
            const int r = dot / B, b = dot % B;
            const float* w = Wl[l] + (size_t)r * (K + 1);
            const float* x = xl[l] + (size_t)b * (K + 1);
            float acc2 = 0.f;
            int k = part;
            for (; k + 4 < K; k += 8) {
              acc = fmaf(w[k], x[k], acc);
              acc2 = fmaf(w[k + 4], x[k + 4], acc2);
            }
            if (k < K) acc = fmaf(w[k], x[k], acc);
            acc += acc2;
          }
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          acc += __shfl_xor_sync(0xffffffffu, acc, 2);
          if (dot < ndot && part == 0) zl[l][dot] = acc + bl[l][dot / B];
        }
      }
      __syncthreads();
      // cell updates of this CTA's units; h to the window's state buffer
      for (int l = 0; l < L; ++l) {
        const int t = ph - l;
        if (t < 0 || t >= T) continue;
        float* hout = a.hbuf + ((size_t)l * T + t) * B * H;
        for (int e = tid; e < U * B; e += nt) {
          const int uu = e / B, b = e % B;
          const float zi = zl[l][(0 * U + uu) * B + b], zf = zl[l][(1 * U + uu) * B + b];
          const float zg = zl[l][(2 * U + uu) * B + b], zo = zl[l][(3 * U + uu) * B + b];
          const float c = sigm_r(zf) * cl[l][e] + sigm_r(zi) * tanhf(zg);
          cl[l][e] = c;
          hout[(size_t)b * H + u0 + uu] = sigm_r(zo) * tanhf(c);
        }
      }
      if (!grid_sync(a.count, bar++, a.abort_word, a.status, kBarrierTimeoutNs)) return;
    }
    // head on the top layer's last state: this CTA's outputs o = cta + r G;
    // the prediction replaces the oldest ring row (s mod T), the parameters
    // of the newest row carry over
    const float* hT = a.hbuf + ((size_t)(L - 1) * T + T - 1) * B * H;
    float* newrow = a.ring + (size_t)(s % T) * B * I;
    const float* lastrow = a.ring + (size_t)((s + T - 1) % T) * B * I;
    for (int e = tid / 32; e < yrows * B; e += nt / 32) {
      const int r = e / B, b = e % B, o = cta + r * G;
      float acc = 0.f;
      for (int k = tid & 31; k < H; k += 32) acc = fmaf(Wy[r * H + k], __ldcg(hT + (size_t)b * H + k), acc);
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if ((tid & 31) == 0 && o < O) {
        const float y = acc + byl[r];
        newrow[(size_t)b * I + a.d + o] = y;
        a.out[((size_t)b * a.steps + s) * O + o] = y;
      }
    }
    if (cta == 0)
      for (int e = tid; e < B * a.d; e += nt) {
        const int b = e / a.d, k = e % a.d;
        newrow[(size_t)b * I + k] = __ldcg(lastrow + (size_t)b * I + k);
      }
    if (!grid_sync(a.count, bar++, a.abort_word, a.status, kBarrierTimeoutNs)) return;
  }
}

// Self-test of the grid barrier's limit: CTA 0 never arrives, so the wait
// of every CTA runs out and records the timeout.  Its words live here (the
// library allocates nothing): [0] arrivals, [1] abort word, [2] status.
__device__ unsigned g_selftest_words[4];

__global__ void k_grid_sync_selftest(uint64_t limit_ns) {
  grid_sync(&g_selftest_words[0], 0, (int*)&g_selftest_words[1], &g_selftest_words[2], limit_ns,
            blockIdx.x != 0);
}

}  // namespace

int rollout_units(int H, int sms) {
  // the fewest units per CTA that keep the grid within 64 CTAs and one CTA
  // per SM (every barrier waits for all CTAs' arrivals)
  const int cap = sms < 64 ? sms : 64;
  for (int U = 1; U <= H; ++U)
    if (H % U == 0 && H / U <= cap) return U;
  return H;
}

size_t rollout_smem_bytes(int I, int H, int L, int O, int B, int U) {
  return sizeof(float) * roll_smem_floats(I, H, L, O, B, U, H / U);
}

cudaError_t rollout_persistent(cudaStream_t st, bool bf16_weights, int I, int H, int L, int O, int T,
                               int B, int d, int steps, const float* theta, const void* wbf,
                               const int64_t (*off_w)[3], int64_t off_wy, int64_t off_by,
                               float* ring, float* hbuf, float* out, unsigned* count,
                               int* abort_word, unsigned* status, int sms) {
  RollArgs a;
  a.I = I; a.H = H; a.L = L; a.O = O; a.T = T; a.B = B; a.d = d; a.steps = steps;
  a.U = rollout_units(H, sms);
  a.theta = theta;
  a.wbf = wbf;
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < 3; ++j) a.off_w[l][j] = off_w[l][j];
  a.off_wy = off_wy;
  a.off_by = off_by;
  a.ring = ring;
  a.hbuf = hbuf;
  a.out = out;
  a.count = count;
  a.abort_word = abort_word;
  a.status = status;
  const size_t smem = rollout_smem_bytes(I, H, L, O, B, a.U);
  const dim3 grid((unsigned)(H / a.U)), block(512);
  void* args[] = {&a};
  cudaError_t e;
  if (bf16_weights) {
    e = cudaFuncSetAttribute(k_rollout<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel((void*)k_rollout<__nv_bfloat16>, grid, block, args, smem, st);
  } else {
    e = cudaFuncSetAttribute(k_rollout<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((void*)k_rollout<float>, grid, block, args, smem, st);
  }
  note_launch();
  return e;
}

// Runs the self-test kernel and returns the status word it left (after
// synchronising the stream).
cudaError_t grid_sync_selftest(cudaStream_t st, double seconds, unsigned* status_out) {
  const unsigned zero[4] = {0u, 0u, 0u, 0u};
  cudaError_t e = cudaMemcpyToSymbolAsync(g_selftest_words, zero, sizeof(zero), 0,
                                          cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  uint64_t limit = (uint64_t)(seconds * 1e9);
  void* args[] = {&limit};
  e = cudaLaunchCooperativeKernel((void*)k_grid_sync_selftest, dim3(2), dim3(32), args, 0, st);
  note_launch();
  if (e != cudaSuccess) return e;
  unsigned w[4];
  e = cudaMemcpyFromSymbolAsync(w, g_selftest_words, sizeof(w), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *status_out = w[2];
  return e;
}

}  // namespace rpod
