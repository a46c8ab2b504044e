// Tensor-core passes (placeholder until the tcgen05 kernels land).
#include "rpod_tc.cuh"

namespace rpod {

int tc_plan_extend(int64_t, int64_t, int, int, size_t*, size_t* off_lowp) {
  *off_lowp = 0;
  return RPOD_OK;
}
int tc_basis(const TcArgs&) { return RPOD_ERR_UNSUPPORTED; }
int tc_project(int64_t, const float*, int64_t, int, const void*, int64_t, int64_t, int, float*,
               int64_t, char*, size_t, size_t, int, size_t, cudaStream_t) {
  return RPOD_ERR_UNSUPPORTED;
}

}  // namespace rpod
