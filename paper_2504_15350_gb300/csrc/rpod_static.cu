// Allocation-free Galerkin projection (C' = U^T S', the coefficients of new
// snapshots on the basis, Sec. 4.3): the rpod_project computation with its
// split-K partial sums kept in a fixed device array of this library instead
// of a caller-provided workspace.
//
// Some callers cannot call cudaMalloc or hand out a workspace: a host
// framework that owns every byte of device memory through its own pool, a
// plugin whose execute callback may not allocate, or a latency-critical loop
// that must not risk the device synchronisation an allocation or free can
// cause.  They still pass U, S' and C' themselves; only the scratch is fixed.
//
// The array below occupies kStaticScratchBytes on every GPU that loads the
// library, until the process exits.  All calls share it, so calls whose
// kernels overlap on the GPU (other streams, other host threads) race on it;
// serialise them.  No part of it has to start at zero: every split writes its
// whole partial block (zeros for an empty range of rows) before the
// reduction reads it, so the contents left by the previous call are never
// read.
#include <mutex>

#include "rpod_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_project_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device.  The name is only a
// host-side stand-in for it.  Outside a stream capture the address is looked
// up on every call (a device reset or a new primary context reloads the
// module and may move the array); during a capture the address recorded by
// the last call outside one is used, since a lookup may load the module.
int scratch_address(cudaStream_t st, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RPOD_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return RPOD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_project_scratch) != cudaSuccess || !p) return RPOD_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RPOD_OK;
}

template <typename W>
int project_static(int64_t n, int nsplit_max, const W* U, int64_t ldu, int kc, const W* S,
                   int64_t lds, int64_t m_new, W* C, int64_t ldc, cudaStream_t st) {
  const size_t per_split = (size_t)kc * (size_t)m_new * sizeof(W);
  if (per_split > kStaticScratchBytes) return RPOD_ERR_UNSUPPORTED;
  int nsplit = (int)(kStaticScratchBytes / per_split);
  if (nsplit > nsplit_max) nsplit = nsplit_max;
  if (nsplit < 1) nsplit = 1;
  void* scratch = nullptr;
  if (int rc = scratch_address(st, &scratch)) return rc;
  W* part = (W*)scratch;
  // C'^T (m_new x kc) = S'^T U: partial sums per split of rows, then their
  // deterministic reduction into C'
  if (rpod::gemm<W, W, W, W>(st, true, m_new, kc, n, nsplit, S, lds, U, ldu, part, 1, m_new,
                             (int64_t)m_new * kc, nullptr, false) != cudaSuccess)
    return RPOD_ERR_CUDA;
  if (rpod::reduce_splits<W, W>(st, m_new, kc, nsplit, part, C, ldc, 1) != cudaSuccess)
    return RPOD_ERR_CUDA;
  return RPOD_OK;
}

}  // namespace

namespace rpod {
// Plan fields this file needs (defined beside the plan, not exported).
void plan_shape(const rpod_plan* plan, int64_t* n, int32_t* l, int32_t* compute, int32_t* nsplit);
}  // namespace rpod

extern "C" int rpod_project_static(const rpod_plan* plan, const void* U, int64_t ldu, int32_t kc,
                                   const void* S_new, int64_t lds, int64_t m_new, int32_t s_dtype,
                                   void* C, int64_t ldc, void* stream) {
  int64_t n = 0;
  int32_t l = 0, compute = 0, nsplit = 1;
  if (!plan) return RPOD_ERR_INVALID_ARG;
  rpod::plan_shape(plan, &n, &l, &compute, &nsplit);
  if (!U || !S_new || !C || kc < 1 || kc > l || m_new < 1) return RPOD_ERR_INVALID_ARG;
  if (ldu < n || lds < n || ldc < kc) return RPOD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (compute == RPOD_F64) {
    if (s_dtype != RPOD_F64) return RPOD_ERR_INVALID_ARG;
    return project_static<double>(n, nsplit, (const double*)U, ldu, kc, (const double*)S_new, lds,
                                  m_new, (double*)C, ldc, st);
  }
  if (s_dtype != RPOD_F32) return RPOD_ERR_INVALID_ARG;
  return project_static<float>(n, nsplit, (const float*)U, ldu, kc, (const float*)S_new, lds, m_new,
                               (float*)C, ldc, st);
}
