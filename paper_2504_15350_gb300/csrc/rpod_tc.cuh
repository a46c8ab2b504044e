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
// `stages`: 0 picks the pipeline depth from the pass size (two 96 KB stages
// below 1 GiB, so that two CTAs share an SM, else four), 2 or 4 force it.
int tc_wpass(cudaStream_t st, int dt, const void* A, int64_t lda, int64_t n, int l, const void* S,
             int64_t lds, int64_t m, float* part, int nsplit, unsigned* status, int stages = 0);

// Y-pass: Y(i, c) = sum_j S(i, j) A(j, c) for i < n, c < l; A: m x 128
// column-major (ld lda, columns >= l zero), S: n x m, both 16-bit of type dt;
// Y FP32 column-major (ld ldy).  With a partial buffer (part_elems floats),
// a standalone pass whose row tiles cannot fill the GPU splits the snapshots
// into chunks summed there and then reduced into Y.
int tc_ypass(cudaStream_t st, int dt, const void* A, int64_t lda, const void* S, int64_t lds,
             int64_t n, int64_t m, int l, float* Y, int64_t ldy, unsigned* status,
             float* part = nullptr, size_t part_elems = 0, int stages = 0);

// First Y-pass over an FP32 S (n x m, ld lds): Y as tc_ypass with S rounded
// to the 16-bit type dt, and that rounded S written to Sh (n x m, ld ldh, a
// multiple of 8; Sh 16-byte aligned); records ST_NONFINITE for non-finite
// entries of S.  RPOD_ERR_UNSUPPORTED when S, A or Sh is not addressable.
int tc_ypass_cvt(cudaStream_t st, int dt, const void* A, int64_t lda, const float* S, int64_t lds,
                 int64_t n, int64_t m, int l, float* Y, int64_t ldy, void* Sh, int64_t ldh,
                 unsigned* status, float* part = nullptr, size_t part_elems = 0);

// Gram partials part[z][c + j l] (FP32 sums) = sum over rows of split z of
// Y(i, c) Y(i, j) for c, j < l <= 128, on the TF32 tensor path with FP32
// accumulation; nsplit CTAs, each a contiguous run of 32-row tiles.  Every
// element is split into TF32 parts: hi/lo with three products (about 2^-21
// relative error per product), or with `exact` an exact three-part split
// and the six products above 2^-33 (products as accurate as FP32 ones).
// The exact form writes only the upper triangle (c <= j) of each partial.
// Y FP32 column-major (ld ldy); base 16-byte aligned and ldy a multiple of
// 4, else RPOD_ERR_UNSUPPORTED.
int tc_gram(cudaStream_t st, const float* Y, int64_t ldy, int64_t rows, int l, float* part,
            int nsplit, unsigned* status, bool exact = false);

// CholeskyQR apply Q = Y X for Y n x l FP32 (column-major, ld ldy; base
// 16-byte aligned, ldy a multiple of 4, else RPOD_ERR_UNSUPPORTED) and X
// l x ncol FP32 (ld ldx; ncol = l when 0, at most 128).  Default: both
// rounded to TF32, one tensor-core product with FP32 accumulation (about
// 2^-11 relative error per entry); writes each output that is not null: Q
// (FP32, ld ldq), Q rounded to dt16 (RPOD_BF16 or RPOD_F16) into Qh (ld ldh),
// Q rounded to TF32 into Qt (ld ldt) -- for bases that are rounded to 16 bits
// next or re-orthonormalised from an exact Gram.  With `precise` both
// operands are split into TF32 hi and lo parts and three products are summed
// (about 2^-21 relative error), Q only -- for the lift of the returned basis.
// l <= 128.
int tc_apply(cudaStream_t st, const float* Y, int64_t ldy, int64_t n, int l, const float* X,
             int64_t ldx, float* Q, int64_t ldq, int dt16, void* Qh, int64_t ldh, float* Qt,
             int64_t ldt, unsigned* status, int ncol = 0, bool precise = false);

// Streaming multiprocessors of the current device.
int tc_sm_count();

}  // namespace rpod
