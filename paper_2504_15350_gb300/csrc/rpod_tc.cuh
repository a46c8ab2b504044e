// Tensor-core (tcgen05 + TMA) passes over S for the 16-bit and TF32 forms.
#pragma once
#include "rpod_internal.cuh"

namespace rpod {

// Number of split-K chunks the W-pass uses for an n x m matrix of type dt.
int tc_wpass_splits(int64_t n, int64_t m, int dt);

// W-pass: part[z][c][j] = sum over rows i of split z of A(i, c) S(i, j) for
// c < l, j < m.  A: n x 128 column-major (ld lda, columns >= l zero), S: n x m
// (ld lds), both of type dt (RPOD_BF16, RPOD_F16, or RPOD_F32 read as TF32).
// Base pointers 16-byte aligned and ld * sizeof multiple of 16, else
// RPOD_ERR_UNSUPPORTED.
int tc_wpass(cudaStream_t st, int dt, const void* A, int64_t lda, int64_t n, int l, const void* S,
             int64_t lds, int64_t m, float* part, int nsplit, unsigned* status);

// Y-pass: Y(i, c) = sum_j S(i, j) A(j, c) for i < n, c < l; A: m x 128
// column-major (ld lda, columns >= l zero), S: n x m, both 16-bit of type dt;
// Y FP32 column-major (ld ldy).
int tc_ypass(cudaStream_t st, int dt, const void* A, int64_t lda, const void* S, int64_t lds,
             int64_t n, int64_t m, int l, float* Y, int64_t ldy, unsigned* status);

}  // namespace rpod
