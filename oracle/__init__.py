"""FP64 CPU oracle for randomized POD (Alg. 1, Sec. 4.2) and its LSTM (Sec. 4.3).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the GPU path computes, used to check it.  Only the tests,
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
it.  It shares no code with the CUDA library (no kernels, headers, helpers,
tables or constant generators) and never imports it; the library never
imports this package.

Modules
  philox  -- Philox4x64-10 counter-based generator and the Gaussian sketch
             matrix Lambda of Alg. 1 (first step), by element counter.
  linalg  -- Householder QR, one-sided (Hestenes) Jacobi SVD, the column sign
             convention.
  rpod    -- Alg. 1 step by step (sketch, subspace iterations with
             re-orthonormalisation, QR, T = Q^T S, SVD of T, lift) plus the
             modal coefficients C = U_N^T S (Sec. 4.3), deterministic POD
             (Eq. (svd)), the per-sample time averages and fluctuation
             snapshots (Eqs. (time_av), (fluct_q)) and the energy-based rank
             (Eq. (energy)).
  lstm    -- LSTM forward, backpropagation through time and Adam in FP64,
             with dropout between stacked layers from counter-based masks.
  sharded -- Alg. 1 with the rows of S spread over ranks: one sum over ranks
             per pass (the algebra of a row-sharded multi-GPU rPOD, checked
             on gloo CPU ranks against the single-process oracle).

Every function is pinned by tests under tests/ against something other than
itself (numpy's Philox words, numpy.linalg.svd, closed forms, exact-rank
recovery, brute force, the randomized range-finder bound, central finite
differences).
"""
