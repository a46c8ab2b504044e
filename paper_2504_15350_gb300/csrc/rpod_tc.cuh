// Tensor-core (tcgen05 + TMA) form of the rPOD passes for 16-bit snapshot
// matrices: interface between the C ABI and rpod_tc.cu.
#pragma once
#include "rpod_internal.cuh"

namespace rpod {

struct TcArgs {
  int64_t n, m;
  int k, l, q;
  uint64_t seed;
  int compute;
  uint32_t flags;
  const void* S;
  int64_t lds;
  int s_dtype;
  const float* Sref;
  int64_t ldr;
  float* U;
  int64_t ldu;
  double* sigma;
  float* C;
  int64_t ldc;
  char* ws;
  cudaStream_t stream;
  size_t off_status, off_lam, off_y, off_q, off_z, off_zq, off_tt, off_part, off_gpart, off_g,
      off_x, off_xw, off_eig, off_uhat, off_sign, off_lowp, sign_bytes;
  int nsplit_z, nsplit_t;
};

// Extra workspace the 16-bit forms need, appended at *off.
int tc_plan_extend(int64_t n, int64_t m, int l, int compute, size_t* off, size_t* off_lowp);
int tc_basis(const TcArgs& a);
int tc_project(int64_t n, const float* U, int64_t ldu, int kc, const void* S, int64_t lds,
               int64_t m, int s_dtype, float* C, int64_t ldc, char* ws, size_t off_part,
               size_t part_elems, int nsplit, size_t off_status, cudaStream_t st);

}  // namespace rpod
