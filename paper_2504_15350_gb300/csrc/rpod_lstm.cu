// LSTM on modal coefficients (Sec. 4.3 of the paper; hyperparameters of
// Table tab:hyperparam): windows of sigma_L time steps of [mu, alpha_1..N]
// (Eq. (input)) map to the next coefficients.  Standard cell with gates
// [i, f, g, o], stacked layers, a linear head on the top layer's last state,
// MSE loss, backpropagation through time and Adam with weight decay.
//
// Precision: FP32 master parameters, BF16 copies of the weight matrices read
// by every product, FP32 activations and accumulation.
//
// Dropout (Table tab:hyperparam, 0.1 for the stream-function networks): in
// training passes (loss_grad, train_step) the input of every layer above the
// first is multiplied by keep / (1 - p); keep for element e = (t B + b) H + j
// of the input to layer l at training pass s is word e mod 4 of the
// Philox4x64-10 block with counter (e div 4, l, s, 0) and key (seed, 1),
// kept when that word shifted right by 11 is at least ceil(p 2^53).  The
// backward pass regenerates the same mask for the gradient it hands down.
//
// Kernels: the input projection of all T steps of a layer is one GEMM; each
// recurrent step is one fused kernel (h_{t-1} W_h^T tile GEMM whose epilogue
// applies the gate activations and the c/h update); BPTT runs one fused
// pointwise kernel (gate gradients, dc) and one GEMM (dz W_h) per step, then
// three GEMMs over all steps for dW_x, dW_h and the input gradient.
#include <math.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "rpod_internal.cuh"

struct rpod_lstm {
  int I, H, L, O, T, Bmax;
  int64_t P;
  int64_t off_w[8][3];  // per layer: W_x, W_h, b offsets into the flat vector
  int64_t off_wy, off_by;
  // workspace layout (bytes)
  size_t o_theta, o_m, o_v, o_grad, o_wbf, o_xtm, o_xtm2, o_gx, o_gates, o_c, o_h, o_y, o_dy,
      o_loss, o_dhext, o_dz, o_dhrec, o_dc, o_dx, o_part, total;
  size_t part_floats;
  int64_t step;
  int last_launches;
  int wfp32;  // products read the FP32 master weights instead of BF16 copies
  // dropout between stacked layers (training passes only)
  double drop_p;
  uint64_t drop_seed, drop_thr;
  int64_t drop_pass;
  size_t o_xd;  // masked inputs of layers 1..L-1 (T x Bmax x H each)
  size_t o_bx, o_by, o_lsum;  // train_epoch: the gathered batch, the loss sum
  size_t o_sync;  // persistent rollout: barrier arrivals, abort word, status word
  // state read by rpod_lstm_load, copied to a workspace by rpod_lstm_restore
  bool pending = false;
  int64_t pend_step = 0;
  std::vector<float> pend;  // theta, m, v (3 P floats)
};

namespace rpod {
namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }

// out[e] = keep(e) ? in[e] * scale : 0 for e < n (in == out allowed): one
// thread per Philox block of four elements
__global__ void k_dropout(int64_t n, const float* in, float* out, uint64_t seed, uint64_t layer,
                          uint64_t pass, uint64_t thr, float scale) {
  const int64_t nb = (n + 3) / 4;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nb;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)k, layer, pass, 0ull};
    philox4x64_10(c, seed, 1ull);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = 4 * k + q;
      if (e < n) out[e] = (c[q] >> 11) >= thr ? in[e] * scale : 0.f;
    }
  }
}

// *sum += *x (one thread); *sum = *sum / count (one thread)
__global__ void k_acc1(float* sum, const float* x) { *sum += *x; }
__global__ void k_div1(float* sum, float count) { *sum /= count; }

__global__ void k_to_time_major(int B, int T, int I, const float* __restrict__ X, float* __restrict__ Xt) {
  const int64_t n = (int64_t)B * T * I;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % I);
    const int64_t r = e / I;
    const int t = (int)(r % T), b = (int)(r / T);
    Xt[((int64_t)t * B + b) * I + k] = X[e];
  }
}

// One recurrent step of one layer for all batch rows: 256 threads, tile of
// 32 batch rows x 32 units (x 4 gates); thread (tb, tu) holds 4 rows x 4 gates
// of unit u0 + tu.
__device__ __forceinline__ float ldw(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldw(const float* p) { return *p; }

template <typename TW>
__global__ void __launch_bounds__(256)
k_lstm_fwd_step(int B, int H, const float* __restrict__ Gx, const float* __restrict__ bias,
                const float* __restrict__ h_prev, const TW* __restrict__ Wh,
                const float* __restrict__ c_prev, float* __restrict__ c_out, float* __restrict__ h_out,
                float* __restrict__ gates) {
  __shared__ float hs[32][33];
  __shared__ float wsm[128][33];
  const int tid = threadIdx.x, tb = tid >> 5, tu = tid & 31;
  const int b0 = blockIdx.x * 32, u0 = blockIdx.y * 32;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int g = 0; g < 4; ++g) acc[i][g] = 0.f;
  for (int k0 = 0; k0 < H; k0 += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int bb = e >> 5, kk = e & 31;
      const int b = b0 + bb, k = k0 + kk;
      hs[bb][kk] = (b < B && k < H) ? h_prev[(int64_t)b * H + k] : 0.f;
    }
    for (int e = tid; e < 128 * 32; e += 256) {
      const int rr = e >> 5, kk = e & 31;
      const int g = rr >> 5, uu = rr & 31;
      const int u = u0 + uu, k = k0 + kk;
      wsm[rr][kk] = (u < H && k < H) ? ldw(Wh + (int64_t)(g * H + u) * H + k) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = hs[tb * 4 + i][kk];
#pragma unroll
      for (int g = 0; g < 4; ++g) w[g] = wsm[g * 32 + tu][kk];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int g = 0; g < 4; ++g) acc[i][g] = fmaf(a[i], w[g], acc[i][g]);
    }
    __syncthreads();
  }
  const int u = u0 + tu;
  if (u >= H) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int b = b0 + tb * 4 + i;
    if (b >= B) continue;
    const int64_t gb = (int64_t)b * 4 * H;
    const float zi = acc[i][0] + Gx[gb + u] + bias[u];
    const float zf = acc[i][1] + Gx[gb + H + u] + bias[H + u];
    const float zg = acc[i][2] + Gx[gb + 2 * H + u] + bias[2 * H + u];
    const float zo = acc[i][3] + Gx[gb + 3 * H + u] + bias[3 * H + u];
    const float ig = sigm(zi), fg = sigm(zf), gg = tanhf(zg), og = sigm(zo);
    const float c = fg * c_prev[(int64_t)b * H + u] + ig * gg;
    c_out[(int64_t)b * H + u] = c;
    h_out[(int64_t)b * H + u] = og * tanhf(c);
    gates[gb + u] = ig;
    gates[gb + H + u] = fg;
    gates[gb + 2 * H + u] = gg;
    gates[gb + 3 * H + u] = og;
  }
}

// Gate gradients of one step (the oracle's backward in lstm.py, per element).
__global__ void k_lstm_bwd_point(int B, int H, const float* __restrict__ dh_ext,
                                 const float* __restrict__ dh_rec, const float* __restrict__ gates,
                                 const float* __restrict__ c_t, const float* __restrict__ c_prev,
                                 float* __restrict__ dc, float* __restrict__ dz) {
  const int64_t n = (int64_t)B * H;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / H), u = (int)(e % H);
    const int64_t gb = (int64_t)b * 4 * H;
    const float ig = gates[gb + u], fg = gates[gb + H + u], gg = gates[gb + 2 * H + u],
                og = gates[gb + 3 * H + u];
    const float dh = dh_ext[e] + (dh_rec ? dh_rec[e] : 0.f);
    const float tc = tanhf(c_t[e]);
    const float d_o = dh * tc;
    const float dcv = dc[e] + dh * og * (1.f - tc * tc);
    const float di = dcv * gg, dg = dcv * ig, df = dcv * c_prev[e];
    dc[e] = dcv * fg;
    dz[gb + u] = di * ig * (1.f - ig);
    dz[gb + H + u] = df * fg * (1.f - fg);
    dz[gb + 2 * H + u] = dg * (1.f - gg * gg);
    dz[gb + 3 * H + u] = d_o * og * (1.f - og);
  }
}

// y += b_y; with a target: loss = mean((y - t)^2), dy = 2 (y - t) / (B O).
__global__ void __launch_bounds__(1024)
k_head_loss(int B, int O, float* __restrict__ y, const float* __restrict__ by,
            const float* __restrict__ tgt, float* __restrict__ dy, float* __restrict__ loss) {
  __shared__ double red[32];
  const int64_t n = (int64_t)B * O;
  double s = 0.0;
  const float scale = 2.f / (float)n;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const float v = y[e] + by[e % O];
    y[e] = v;
    if (tgt) {
      const float d = v - tgt[e];
      dy[e] = scale * d;
      s += (double)d * d;
    }
  }
  if (!tgt) return;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a += red[k];
    *loss = (float)(a / (double)n);
  }
}

// out[c] = sum_i in[i * N + c]
__global__ void k_colsum(int64_t rows, int N, const float* __restrict__ in, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double s = 0.0;
  for (int64_t i = 0; i < rows; ++i) s += in[i * N + c];
  out[c] = (float)s;
}

// Adam (Kingma & Ba) with the weight decay added to the gradient; refreshes
// the BF16 copy.
__global__ void k_adam(int64_t P, float* __restrict__ th, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, __nv_bfloat16* __restrict__ wbf,
                       float lr, float b1, float b2, float eps, float wd, float c1, float c2) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    const float gr = g[e] + wd * th[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float t = th[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    th[e] = t;
    wbf[e] = __float2bfloat16_rn(t);
  }
}

__global__ void k_to_bf16(int64_t P, const float* __restrict__ th, __nv_bfloat16* __restrict__ wbf) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x)
    wbf[e] = __float2bfloat16_rn(th[e]);
}

// Windows for training: X[b][t] = [mu[s], series[s][t0 + t]] (t < T),
// Y[b] = series[s][t0 + T], with (s, t0) = idx[b].
__global__ void k_gather(int T, int O, int d, int t_len, const float* __restrict__ series,
                         const float* __restrict__ mu, const int* __restrict__ idx, int B,
                         float* __restrict__ X, float* __restrict__ Y) {
  const int I = d + O;
  const int64_t n = (int64_t)B * (T + 1) * I;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % I);
    const int64_t r = e / I;
    const int t = (int)(r % (T + 1)), b = (int)(r / (T + 1));
    const int s = idx[2 * b], t0 = idx[2 * b + 1];
    if (t < T) {
      X[((int64_t)b * T + t) * I + k] =
          k < d ? mu[(int64_t)s * d + k] : series[((int64_t)s * t_len + t0 + t) * O + (k - d)];
    } else if (k >= d) {
      Y[(int64_t)b * O + (k - d)] = series[((int64_t)s * t_len + t0 + T) * O + (k - d)];
    }
  }
}

// Rollout window shift (time-major): next[t] = cur[t + 1]; next[T-1] =
// [mu from cur[T-1], y]; out[b][s] = y.
__global__ void k_roll(int B, int T, int I, int d, const float* __restrict__ cur, float* __restrict__ next,
                       const float* __restrict__ y, float* __restrict__ out, int steps, int s) {
  const int O = I - d;
  const int64_t n = (int64_t)T * B * I;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % I);
    const int64_t r = e / I;
    const int b = (int)(r % B), t = (int)(r / B);
    float v;
    if (t < T - 1) v = cur[e + (int64_t)B * I];
    else v = k < d ? cur[e] : y[(int64_t)b * O + (k - d)];
    next[e] = v;
    if (t == T - 1 && k >= d) out[((int64_t)b * steps + s) * O + (k - d)] = y[(int64_t)b * O + (k - d)];
  }
}

unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)std::max<int64_t>(b, 1);
}

#define LK(x)                                            \
  do {                                                   \
    if ((x) != cudaSuccess) return RPOD_ERR_CUDA;        \
  } while (0)
#define LL()                                             \
  do {                                                   \
    note_launch();                                       \
    if (cudaGetLastError() != cudaSuccess) return RPOD_ERR_CUDA; \
  } while (0)

#define CR2(x)                                 \
  do {                                         \
    int r_ = (x);                              \
    if (r_ != RPOD_OK) return r_;              \
  } while (0)

struct Net {
  const rpod_lstm* N;
  char* ws;
  cudaStream_t st;
  float* f(size_t o) const { return (float*)(ws + o); }
  __nv_bfloat16* wbf() const { return (__nv_bfloat16*)(ws + N->o_wbf); }
  int in_dim(int l) const { return l == 0 ? N->I : N->H; }
  const float* wx_f(int l) const { return f(N->o_theta) + N->off_w[l][0]; }
  // per-layer activation blocks
  size_t layer_stride_gx() const { return (size_t)N->T * N->Bmax * 4 * N->H; }
  size_t layer_stride_ch() const { return (size_t)(N->T + 1) * N->Bmax * N->H; }
  float* gx(int l) const { return f(N->o_gx) + l * layer_stride_gx(); }
  float* gates(int l) const { return f(N->o_gates) + l * layer_stride_gx(); }
  float* cc(int l) const { return f(N->o_c) + l * layer_stride_ch(); }
  float* hh(int l) const { return f(N->o_h) + l * layer_stride_ch(); }
  float* xd(int l) const { return f(N->o_xd) + (size_t)(l - 1) * N->T * N->Bmax * N->H; }
  // the (masked, in training) input of layer l >= 1
  const float* layer_input(int l, int B) const {
    return train_drop ? xd(l) : hh(l - 1) + (size_t)B * N->H;
  }
  bool train_drop = false;  // this call is a training pass with dropout
  int dropout(int l, int B, const float* in, float* out) const {
    const int64_t n = (int64_t)N->T * B * N->H;
    k_dropout<<<blocks_for((n + 3) / 4), 256, 0, st>>>(n, in, out, N->drop_seed, (uint64_t)l,
                                                      (uint64_t)N->drop_pass, N->drop_thr,
                                                      (float)(1.0 / (1.0 - N->drop_p)));
    LL();
    return RPOD_OK;
  }

  template <typename TW>
  const TW* weights() const {
    return sizeof(TW) == 4 ? (const TW*)(ws + N->o_theta) : (const TW*)(ws + N->o_wbf);
  }
  int forward(const float* Xt, int B) {
    return N->wfp32 ? forward_t<float>(Xt, B) : forward_t<__nv_bfloat16>(Xt, B);
  }
  int backward(const float* Xt, int B) {
    return N->wfp32 ? backward_t<float>(Xt, B) : backward_t<__nv_bfloat16>(Xt, B);
  }

  // forward over the time-major input Xt (T x B x I); y (B x O) without bias
  template <typename TW>
  int forward_t(const float* Xt, int B) {
    const int H = N->H, T = N->T;
    const TW* W = weights<TW>();
    for (int l = 0; l < N->L; ++l) {
      const int Il = in_dim(l);
      // h_1..h_T of the layer below, masked in a training pass with dropout
      if (l > 0 && train_drop) CR2(dropout(l, B, hh(l - 1) + (size_t)B * H, xd(l)));
      const float* Xin = l == 0 ? Xt : layer_input(l, B);
      // hoisted input projection for all T steps
      LK((gemm_ex<float, TW, float, float>(st, true, true, (int64_t)T * B, 4 * H, Il, 1, Xin, Il,
                                                     W + N->off_w[l][0], Il, gx(l), 4 * H, 1, 0,
                                                     nullptr, false)));
      LK(cudaMemsetAsync(cc(l), 0, (size_t)B * H * 4, st));
      LK(cudaMemsetAsync(hh(l), 0, (size_t)B * H * 4, st));
      const float* bias = f(N->o_theta) + N->off_w[l][2];
      dim3 grid((B + 31) / 32, (H + 31) / 32);
      for (int t = 0; t < T; ++t) {
        k_lstm_fwd_step<TW><<<grid, 256, 0, st>>>(B, H, gx(l) + (size_t)t * B * 4 * H, bias,
                                              hh(l) + (size_t)t * B * H, W + N->off_w[l][1],
                                              cc(l) + (size_t)t * B * H, cc(l) + (size_t)(t + 1) * B * H,
                                              hh(l) + (size_t)(t + 1) * B * H,
                                              gates(l) + (size_t)t * B * 4 * H);
        LL();
      }
    }
    const float* hT = hh(N->L - 1) + (size_t)T * B * H;
    LK((gemm_ex<float, TW, float, float>(st, true, true, B, N->O, H, 1, hT, H, W + N->off_wy, H,
                                                   f(N->o_y), N->O, 1, 0, nullptr, false)));
    return RPOD_OK;
  }

  // dW = DZ^T * Xin over K = rows, split over rows, into grad (rows_out x cols, row-major)
  int wgrad(const float* DZ, int64_t rows, int nout, const float* Xin, int ncols, float* g) {
    const int ns = (int)std::min<int64_t>(32, std::max<int64_t>(1, rows / 128));
    float* part = f(N->o_part);
    LK((gemm_ex<float, float, float, float>(st, false, false, nout, ncols, rows, ns, DZ, nout, Xin, ncols,
                                           part, 1, nout, (int64_t)nout * ncols, nullptr, false)));
    LK((reduce_splits<float, float>(st, nout, ncols, ns, part, g, ncols, 1)));
    return RPOD_OK;
  }

  template <typename TW>
  int backward_t(const float* Xt, int B) {
    const int H = N->H, T = N->T, O = N->O;
    const TW* W = weights<TW>();
    float* G = f(N->o_grad);
    const float* hT = hh(N->L - 1) + (size_t)T * B * H;
    float* dy = f(N->o_dy);
    // head
    CR2(wgrad(dy, B, O, hT, H, G + N->off_wy));
    k_colsum<<<(O + 127) / 128, 128, 0, st>>>(B, O, dy, G + N->off_by);
    LL();
    float* dhext = f(N->o_dhext);
    LK(cudaMemsetAsync(dhext, 0, (size_t)T * B * H * 4, st));
    LK((gemm_ex<float, TW, float, float>(st, true, false, B, H, O, 1, dy, O, W + N->off_wy, H,
                                                   dhext + (size_t)(T - 1) * B * H, H, 1, 0, nullptr,
                                                   false)));
    float* dz = f(N->o_dz);
    float* dhrec = f(N->o_dhrec);
    float* dc = f(N->o_dc);
    for (int l = N->L - 1; l >= 0; --l) {
      const int Il = in_dim(l);
      LK(cudaMemsetAsync(dc, 0, (size_t)B * H * 4, st));
      for (int t = T - 1; t >= 0; --t) {
        k_lstm_bwd_point<<<blocks_for((int64_t)B * H), 256, 0, st>>>(
            B, H, dhext + (size_t)t * B * H, t == T - 1 ? nullptr : dhrec,
            gates(l) + (size_t)t * B * 4 * H, cc(l) + (size_t)(t + 1) * B * H, cc(l) + (size_t)t * B * H,
            dc, dz + (size_t)t * B * 4 * H);
        LL();
        if (t > 0)
          LK((gemm_ex<float, TW, float, float>(st, true, false, B, H, 4 * H, 1,
                                                         dz + (size_t)t * B * 4 * H, 4 * H,
                                                         W + N->off_w[l][1], H, dhrec, H, 1, 0, nullptr,
                                                         false)));
      }
      const float* Xin = l == 0 ? Xt : layer_input(l, B);
      const int64_t rows = (int64_t)T * B;
      CR2(wgrad(dz, rows, 4 * H, Xin, Il, G + N->off_w[l][0]));
      CR2(wgrad(dz, rows, 4 * H, hh(l), H, G + N->off_w[l][1]));  // h_0..h_{T-1}
      k_colsum<<<(4 * H + 127) / 128, 128, 0, st>>>(rows, 4 * H, dz, G + N->off_w[l][2]);
      LL();
      if (l > 0) {
        LK((gemm_ex<float, TW, float, float>(st, true, false, rows, Il, 4 * H, 1, dz, 4 * H,
                                                       W + N->off_w[l][0], Il, dhext, Il, 1, 0, nullptr,
                                                       false)));
        // the input of layer l was keep / (1 - p) times h of layer l - 1
        if (train_drop) CR2(dropout(l, B, dhext, dhext));
      }
    }
    return RPOD_OK;
  }
};

}  // namespace
}  // namespace rpod

using namespace rpod;

extern "C" {

int rpod_lstm_create(rpod_lstm** out, int32_t in_dim, int32_t hidden, int32_t layers,
                     int32_t out_dim, int32_t window, int32_t max_batch, uint32_t flags) {
  if (!out || in_dim < 1 || hidden < 1 || layers < 1 || layers > 8 || out_dim < 1 || window < 1 ||
      max_batch < 1 || out_dim > in_dim || (flags & ~(uint32_t)RPOD_LSTM_FP32_WEIGHTS))
    return RPOD_ERR_INVALID_ARG;
  rpod_lstm* N = new (std::nothrow) rpod_lstm();
  if (!N) return RPOD_ERR_INVALID_ARG;
  N->I = in_dim; N->H = hidden; N->L = layers; N->O = out_dim; N->T = window; N->Bmax = max_batch;
  N->wfp32 = (flags & RPOD_LSTM_FP32_WEIGHTS) ? 1 : 0;
  int64_t off = 0;
  for (int l = 0; l < layers; ++l) {
    const int64_t Il = l == 0 ? in_dim : hidden;
    N->off_w[l][0] = off; off += 4 * (int64_t)hidden * Il;
    N->off_w[l][1] = off; off += 4 * (int64_t)hidden * hidden;
    N->off_w[l][2] = off; off += 4 * (int64_t)hidden;
  }
  N->off_wy = off; off += (int64_t)out_dim * hidden;
  N->off_by = off; off += out_dim;
  N->P = off;
  const size_t P = (size_t)off, H = hidden, T = window, B = max_batch, I = in_dim;
  const size_t maxI = std::max(I, H);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = a256(o + bytes); return r; };
  N->o_theta = take(4 * P);
  N->o_m = take(4 * P);
  N->o_v = take(4 * P);
  N->o_grad = take(4 * P);
  N->o_wbf = take(2 * P);
  N->o_xtm = take(4 * T * B * I);
  N->o_xtm2 = take(4 * T * B * I);
  N->o_gx = take(4 * layers * T * B * 4 * H);
  N->o_gates = take(4 * layers * T * B * 4 * H);
  N->o_c = take(4 * layers * (T + 1) * B * H);
  N->o_h = take(4 * layers * (T + 1) * B * H);
  N->o_y = take(4 * B * out_dim);
  N->o_dy = take(4 * B * out_dim);
  N->o_loss = take(256);
  N->o_dhext = take(4 * T * B * maxI);
  N->o_dz = take(4 * T * B * 4 * H);
  N->o_dhrec = take(4 * B * H);
  N->o_dc = take(4 * B * H);
  N->o_dx = take(4);
  N->part_floats = (size_t)32 * 4 * H * maxI;
  N->o_part = take(4 * N->part_floats);
  N->o_xd = take(4 * (size_t)(layers - 1) * T * B * H);
  N->o_bx = take(4 * B * T * I);
  N->o_by = take(4 * B * (size_t)out_dim);
  N->o_lsum = take(4);
  N->o_sync = take(256);
  N->drop_p = 0.0;
  N->drop_seed = 0;
  N->drop_thr = 0;
  N->drop_pass = 0;
  N->total = o;
  N->step = 0;
  *out = N;
  return RPOD_OK;
}

int64_t rpod_lstm_param_count(const rpod_lstm* N) { return N ? N->P : -1; }

int rpod_lstm_workspace_bytes(const rpod_lstm* N, size_t* bytes) {
  if (!N || !bytes) return RPOD_ERR_INVALID_ARG;
  *bytes = N->total;
  return RPOD_OK;
}

void rpod_lstm_destroy(rpod_lstm* N) { delete N; }

static int lstm_ws(const rpod_lstm* N, void* ws, size_t bytes) {
  if (!ws || bytes < N->total || ((uintptr_t)ws & 255)) return RPOD_ERR_WORKSPACE;
  return RPOD_OK;
}

int rpod_lstm_set_params(rpod_lstm* N, const float* theta, void* ws, size_t bytes, void* stream) {
  if (!N || !theta) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  g_launches = 0;
  LK(cudaMemcpyAsync(w + N->o_theta, theta, 4 * N->P, cudaMemcpyDefault, st));
  LK(cudaMemsetAsync(w + N->o_m, 0, 4 * N->P, st));
  LK(cudaMemsetAsync(w + N->o_v, 0, 4 * N->P, st));
  k_to_bf16<<<blocks_for(N->P), 256, 0, st>>>(N->P, (const float*)(w + N->o_theta),
                                               (__nv_bfloat16*)(w + N->o_wbf));
  LL();
  N->step = 0;
  return RPOD_OK;
}

int rpod_lstm_get_params(const rpod_lstm* N, float* theta, void* ws, size_t bytes, void* stream) {
  if (!N || !theta) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  LK(cudaMemcpyAsync(theta, (char*)ws + N->o_theta, 4 * N->P, cudaMemcpyDefault, (cudaStream_t)stream));
  return RPOD_OK;
}

int rpod_lstm_forward(rpod_lstm* N, const float* X, int32_t B, float* Y, void* ws, size_t bytes,
                      void* stream) {
  if (!N || !X || !Y || B < 1 || B > N->Bmax) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Net net{N, (char*)ws, st};
  g_launches = 0;
  float* Xt = net.f(N->o_xtm);
  k_to_time_major<<<blocks_for((int64_t)B * N->T * N->I), 256, 0, st>>>(B, N->T, N->I, X, Xt);
  LL();
  if (int rc = net.forward(Xt, B)) return rc;
  k_head_loss<<<1, 1024, 0, st>>>(B, N->O, net.f(N->o_y), net.f(N->o_theta) + N->off_by, nullptr,
                                   nullptr, nullptr);
  LL();
  LK(cudaMemcpyAsync(Y, net.f(N->o_y), (size_t)4 * B * N->O, cudaMemcpyDeviceToDevice, st));
  N->last_launches = g_launches;
  return RPOD_OK;
}

int rpod_lstm_loss_grad(rpod_lstm* N, const float* X, const float* Yt, int32_t B, float* loss,
                        float* grad, void* ws, size_t bytes, void* stream) {
  if (!N || !X || !Yt || B < 1 || B > N->Bmax) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Net net{N, (char*)ws, st};
  g_launches = 0;
  float* Xt = net.f(N->o_xtm);
  k_to_time_major<<<blocks_for((int64_t)B * N->T * N->I), 256, 0, st>>>(B, N->T, N->I, X, Xt);
  LL();
  net.train_drop = N->drop_p > 0.0 && N->L > 1;
  if (int rc = net.forward(Xt, B)) return rc;
  k_head_loss<<<1, 1024, 0, st>>>(B, N->O, net.f(N->o_y), net.f(N->o_theta) + N->off_by, Yt,
                                   net.f(N->o_dy), net.f(N->o_loss));
  LL();
  if (int rc = net.backward(Xt, B)) return rc;
  if (net.train_drop) N->drop_pass += 1;
  if (loss) LK(cudaMemcpyAsync(loss, net.f(N->o_loss), 4, cudaMemcpyDefault, st));
  if (grad) LK(cudaMemcpyAsync(grad, net.f(N->o_grad), 4 * N->P, cudaMemcpyDefault, st));
  N->last_launches = g_launches;
  return RPOD_OK;
}

int rpod_lstm_train_step(rpod_lstm* N, const float* X, const float* Yt, int32_t B, float lr,
                         float weight_decay, float* loss, void* ws, size_t bytes, void* stream) {
  rpod::NvtxRange nv("rpod_lstm_train_step");
  if (int rc = rpod_lstm_loss_grad(N, X, Yt, B, loss, nullptr, ws, bytes, stream)) return rc;
  const int launches = N->last_launches;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  N->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)N->step), c2 = 1.f - powf(b2, (float)N->step);
  k_adam<<<blocks_for(N->P), 256, 0, st>>>(N->P, (float*)(w + N->o_theta), (const float*)(w + N->o_grad),
                                            (float*)(w + N->o_m), (float*)(w + N->o_v),
                                            (__nv_bfloat16*)(w + N->o_wbf), lr, b1, b2, 1e-8f,
                                            weight_decay, c1, c2);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return RPOD_ERR_CUDA;
  N->last_launches = launches + 1;
  return RPOD_OK;
}

int rpod_lstm_gather(const rpod_lstm* N, const float* series, const float* mu, int32_t n_series,
                     int32_t t_len, int32_t d, const int32_t* idx, int32_t B, float* X, float* Y,
                     void* stream) {
  if (!N || !series || !idx || !X || !Y || B < 1 || d < 0 || d + N->O != N->I || t_len <= N->T ||
      n_series < 1 || (d > 0 && !mu))
    return RPOD_ERR_INVALID_ARG;
  k_gather<<<blocks_for((int64_t)B * (N->T + 1) * N->I), 256, 0, (cudaStream_t)stream>>>(
      N->T, N->O, d, t_len, series, mu, idx, B, X, Y);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RPOD_OK : RPOD_ERR_CUDA;
}

// Persistent rollout possible: at most 4 layers, a CTA's rows and staging
// within 200 KB of shared memory, the grid co-resident (checked by the
// cooperative launch itself).
static bool rollout_fits(const rpod_lstm* N, int B, int sms) {
  if (N->L > 4) return false;
  const int U = rollout_units(N->H, sms);
  return rollout_smem_bytes(N->I, N->H, N->L, N->O, B, U) <= (size_t)200 * 1024;
}

int rpod_lstm_rollout(rpod_lstm* N, const float* window, int32_t B, int32_t mu_cols, int32_t steps,
                      float* out, void* ws, size_t bytes, void* stream) {
  rpod::NvtxRange nv("rpod_lstm_rollout");
  if (!N || !window || !out || B < 1 || B > N->Bmax || steps < 1 || mu_cols < 0 ||
      mu_cols + N->O != N->I)
    return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Net net{N, (char*)ws, st};
  g_launches = 0;
  float* cur = net.f(N->o_xtm);
  float* nxt = net.f(N->o_xtm2);
  k_to_time_major<<<blocks_for((int64_t)B * N->T * N->I), 256, 0, st>>>(B, N->T, N->I, window, cur);
  LL();
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RPOD_ERR_CUDA;
  if (rollout_fits(N, B, sms)) {
    // one cooperative launch for all steps (the window in o_xtm is its ring)
    unsigned* sync = (unsigned*)((char*)ws + N->o_sync);
    LK(cudaMemsetAsync(sync, 0, 16, st));
    const cudaError_t e = rollout_persistent(
        st, !N->wfp32, N->I, N->H, N->L, N->O, N->T, B, mu_cols, steps, net.f(N->o_theta),
        N->wfp32 ? (const void*)net.f(N->o_theta) : (const void*)net.wbf(), N->off_w, N->off_wy,
        N->off_by, cur, net.f(N->o_h), out, sync, (int*)(sync + 1), sync + 2, sms);
    if (e == cudaSuccess) {
      N->last_launches = g_launches;
      return RPOD_OK;
    }
    // a grid the device cannot hold at once: the per-step kernels below
    if (e != cudaErrorCooperativeLaunchTooLarge) return RPOD_ERR_CUDA;
    cudaGetLastError();
  }
  for (int s = 0; s < steps; ++s) {
    if (int rc = net.forward(cur, B)) return rc;
    k_head_loss<<<1, 1024, 0, st>>>(B, N->O, net.f(N->o_y), net.f(N->o_theta) + N->off_by, nullptr,
                                     nullptr, nullptr);
    LL();
    k_roll<<<blocks_for((int64_t)N->T * B * N->I), 256, 0, st>>>(B, N->T, N->I, mu_cols, cur, nxt,
                                                                 net.f(N->o_y), out, steps, s);
    LL();
    std::swap(cur, nxt);
  }
  N->last_launches = g_launches;
  return RPOD_OK;
}

int rpod_lstm_train_epoch(rpod_lstm* N, const float* series, const float* mu, int32_t n_series,
                          int32_t t_len, int32_t d, const int32_t* idx, int32_t n_windows,
                          int32_t batch, float lr, float weight_decay, float* loss_out, void* ws,
                          size_t bytes, void* stream) {
  rpod::NvtxRange nv("rpod_lstm_train_epoch");
  if (!N || !series || !idx || n_windows < 1 || batch < 1 || batch > N->Bmax || d < 0 ||
      d + N->O != N->I || t_len <= N->T || n_series < 1 || (d > 0 && !mu))
    return RPOD_ERR_INVALID_ARG;
  const int nb = n_windows / batch;
  if (nb < 1) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  float* X = (float*)(w + N->o_bx);
  float* Y = (float*)(w + N->o_by);
  float* lsum = (float*)(w + N->o_lsum);
  LK(cudaMemsetAsync(lsum, 0, 4, st));
  int launches = 0;
  for (int b = 0; b < nb; ++b) {
    if (int rc = rpod_lstm_gather(N, series, mu, n_series, t_len, d, idx + 2 * (int64_t)b * batch,
                                  batch, X, Y, stream))
      return rc;
    if (int rc = rpod_lstm_train_step(N, X, Y, batch, lr, weight_decay, nullptr, ws, bytes, stream))
      return rc;
    k_acc1<<<1, 1, 0, st>>>(lsum, (const float*)(w + N->o_loss));
    if (cudaGetLastError() != cudaSuccess) return RPOD_ERR_CUDA;
    launches += N->last_launches + 2;
  }
  k_div1<<<1, 1, 0, st>>>(lsum, (float)nb);
  if (cudaGetLastError() != cudaSuccess) return RPOD_ERR_CUDA;
  if (loss_out) LK(cudaMemcpyAsync(loss_out, lsum, 4, cudaMemcpyDefault, st));
  N->last_launches = launches + 1;
  return RPOD_OK;
}

// ---- model files: "RPODLSTM", version, dimensions, state, theta, m, v
namespace {
constexpr char kMagic[8] = {'R', 'P', 'O', 'D', 'L', 'S', 'T', 'M'};
constexpr uint32_t kVersion = 1;
struct FileHeader {
  char magic[8];
  uint32_t version;
  int32_t dims[7];  // in_dim, hidden, layers, out_dim, window, max_batch, flags
  int64_t step;
  double drop_p;
  uint64_t drop_seed;
  int64_t drop_pass;
  int64_t P;
};
}  // namespace

int rpod_lstm_save(const rpod_lstm* N, const char* path, void* ws, size_t bytes, void* stream) {
  if (!N || !path) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<float> buf;
  try {
    buf.resize(3 * (size_t)N->P);
  } catch (...) {
    return RPOD_ERR_INVALID_ARG;
  }
  const char* w = (const char*)ws;
  LK(cudaMemcpyAsync(buf.data(), w + N->o_theta, 4 * N->P, cudaMemcpyDeviceToHost, st));
  LK(cudaMemcpyAsync(buf.data() + N->P, w + N->o_m, 4 * N->P, cudaMemcpyDeviceToHost, st));
  LK(cudaMemcpyAsync(buf.data() + 2 * N->P, w + N->o_v, 4 * N->P, cudaMemcpyDeviceToHost, st));
  LK(cudaStreamSynchronize(st));
  FileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  const int32_t dims[7] = {N->I, N->H, N->L, N->O, N->T, N->Bmax,
                           N->wfp32 ? (int32_t)RPOD_LSTM_FP32_WEIGHTS : 0};
  memcpy(h.dims, dims, sizeof(dims));
  h.step = N->step;
  h.drop_p = N->drop_p;
  h.drop_seed = N->drop_seed;
  h.drop_pass = N->drop_pass;
  h.P = N->P;
  FILE* f = fopen(path, "wb");
  if (!f) return RPOD_ERR_IO;
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1 &&
            fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? RPOD_OK : RPOD_ERR_IO;
}

int rpod_lstm_load(rpod_lstm** out, const char* path) {
  if (!out || !path) return RPOD_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return RPOD_ERR_IO;
  FileHeader h;
  if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion) {
    fclose(f);
    return RPOD_ERR_IO;
  }
  rpod_lstm* N = nullptr;
  if (rpod_lstm_create(&N, h.dims[0], h.dims[1], h.dims[2], h.dims[3], h.dims[4], h.dims[5],
                       (uint32_t)h.dims[6]) != RPOD_OK ||
      N->P != h.P || !(h.drop_p >= 0.0 && h.drop_p < 1.0) || h.step < 0 || h.drop_pass < 0) {
    if (N) rpod_lstm_destroy(N);
    fclose(f);
    return RPOD_ERR_IO;
  }
  try {
    N->pend.resize(3 * (size_t)N->P);
  } catch (...) {
    rpod_lstm_destroy(N);
    fclose(f);
    return RPOD_ERR_INVALID_ARG;
  }
  const bool ok = fread(N->pend.data(), sizeof(float), N->pend.size(), f) == N->pend.size();
  fclose(f);
  if (!ok) {
    rpod_lstm_destroy(N);
    return RPOD_ERR_IO;
  }
  N->pending = true;
  N->pend_step = h.step;
  if (h.drop_p > 0.0) rpod_lstm_set_dropout(N, h.drop_p, h.drop_seed);
  N->drop_pass = h.drop_pass;
  *out = N;
  return RPOD_OK;
}

int rpod_lstm_restore(rpod_lstm* N, void* ws, size_t bytes, void* stream) {
  if (!N || !N->pending) return RPOD_ERR_INVALID_ARG;
  if (int rc = lstm_ws(N, ws, bytes)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  g_launches = 0;
  // pageable source: each copy returns once its data is staged
  LK(cudaMemcpyAsync(w + N->o_theta, N->pend.data(), 4 * N->P, cudaMemcpyHostToDevice, st));
  LK(cudaMemcpyAsync(w + N->o_m, N->pend.data() + N->P, 4 * N->P, cudaMemcpyHostToDevice, st));
  LK(cudaMemcpyAsync(w + N->o_v, N->pend.data() + 2 * N->P, 4 * N->P, cudaMemcpyHostToDevice, st));
  k_to_bf16<<<blocks_for(N->P), 256, 0, st>>>(N->P, (const float*)(w + N->o_theta),
                                               (__nv_bfloat16*)(w + N->o_wbf));
  LL();
  N->step = N->pend_step;
  N->last_launches = g_launches;
  return RPOD_OK;
}

int rpod_lstm_dims(const rpod_lstm* N, int32_t* dims) {
  if (!N || !dims) return RPOD_ERR_INVALID_ARG;
  const int32_t d[7] = {N->I, N->H, N->L, N->O, N->T, N->Bmax,
                        N->wfp32 ? (int32_t)RPOD_LSTM_FP32_WEIGHTS : 0};
  memcpy(dims, d, sizeof(d));
  return RPOD_OK;
}

int rpod_lstm_set_dropout(rpod_lstm* N, double p, uint64_t seed) {
  if (!N || !(p >= 0.0) || !(p < 1.0)) return RPOD_ERR_INVALID_ARG;
  N->drop_p = p;
  N->drop_seed = seed;
  N->drop_thr = (uint64_t)ceil(p * 9007199254740992.0);  // ceil(p 2^53), exact scaling
  N->drop_pass = 0;
  return RPOD_OK;
}

int rpod_lstm_status_sync(const rpod_lstm* N, void* ws, void* stream) {
  if (!N || !ws) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* d = (unsigned*)((char*)ws + N->o_sync) + 2;
  unsigned h = 0;
  if (cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaMemsetAsync(d, 0, sizeof(h), st) != cudaSuccess)
    return RPOD_ERR_CUDA;
  return (h & ST_TIMEOUT) ? RPOD_ERR_TIMEOUT : RPOD_OK;
}

int rpod_selftest_grid_barrier(double seconds, void* stream) {
  if (!(seconds > 0.0 && seconds <= 2.0)) return RPOD_ERR_INVALID_ARG;
  unsigned status = 0;
  if (grid_sync_selftest((cudaStream_t)stream, seconds, &status) != cudaSuccess) return RPOD_ERR_CUDA;
  return (status & ST_TIMEOUT) ? RPOD_ERR_TIMEOUT : RPOD_OK;
}

int rpod_lstm_last_launch_count(const rpod_lstm* N) { return N ? N->last_launches : -1; }

}  // extern "C"
