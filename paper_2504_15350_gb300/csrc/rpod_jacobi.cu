// Small SVD of Alg. 1 (sixth step, T = Uhat Sigma V^T) for the FP64 form by
// one-sided Jacobi rotations, so that small singular values keep their
// relative accuracy.
//
// The l x m matrix T = Q^T S of a randomized POD is row-graded: row i has a
// norm close to sigma_i (the columns of Q come from a QR of S Lambda and are
// ordered by the energy they capture).  Its FP64 Gram G = T T^T then has
// rounding errors of size u sigma_i sigma_j in entry (i, j), and
//   1. the Cholesky factor G = R^T R (no pivoting) has a componentwise
//      backward error of the same graded size (Demmel, "On floating point
//      errors in Cholesky", LAPACK Working Note 14, 1989); R is graded by
//      columns and L = R^T by rows;
//   2. one-sided Jacobi rotations of the columns of L (Hestenes 1958) with the
//      stopping rule |l_i . l_j| <= tol ||l_i|| ||l_j|| compute the singular
//      values of L to a relative accuracy governed by the condition number of
//      the row-scaled factor, not by sigma_1 / sigma_i (Demmel & Veselic,
//      "Jacobi's method is more accurate than QR", SIAM J. Matrix Anal. Appl.
//      13, 1992).  For a decaying spectrum the columns of L are already
//      nearly orthogonal (their cosines scale like sigma_j / sigma_i), so few
//      sweeps are needed.
// L J = W with mutually orthogonal columns gives G = L L^T = W W^T: sigma_i =
// ||w_i|| and Uhat = W diag(1 / sigma) -- no rotation needs accumulating.
// (A dense orthogonal preconditioner, L X0, would not do: the absolute
// rounding of X0's entries puts errors of size u sigma_1 into every column.)
//
// One CTA, FP64: R packed (upper triangle) and W (l x l) in shared memory.
#include <float.h>

#include <mutex>

#include "rpod_internal.cuh"

namespace rpod {
namespace {

constexpr int kJacThreads = 1024;

__device__ __forceinline__ int pk(int a, int b) { return b * (b + 1) / 2 + a; }  // a <= b

// Sum over the gs lanes of a column-pair group (gs a power of two <= 16;
// every lane of the warp takes part).
__device__ __forceinline__ double group_sum(double v, int gs) {
  for (int o = gs >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Round r of the circle method over lp (even) players: pair p.
__device__ __forceinline__ void round_pair(int lp, int r, int p, int& i, int& j) {
  const int n1 = lp - 1;
  int a, b;
  if (p == 0) {
    a = n1;
    b = r;
  } else {
    a = (r + p) % n1;
    b = (r - p + n1) % n1;
  }
  i = a < b ? a : b;
  j = a < b ? b : a;
}

__global__ void __launch_bounds__(kJacThreads)
k_jacobi_svd(int l, const double* __restrict__ G, double* __restrict__ K, double* __restrict__ sigma,
             int max_sweeps, double tol, unsigned* status) {
  // K: the l x l output Uhat (column-major)
  extern __shared__ double sm[];
  const int np = l * (l + 1) / 2;
  double* Rp = sm;                       // packed upper triangle, np
  double* W = Rp + ((np + 1) / 2) * 2;   // l x l, column-major, ld l
  double* d0 = W + (size_t)l * l;        // l: diagonal of G
  double* nrm = d0 + l;                  // l: squared column norms of W
  __shared__ double s_dinv, s_rinv[2];  // reciprocal pivots of rows j (j & 1) and j - 1
  __shared__ int s_rot;
  __shared__ int s_rank[kMaxL];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  // ---- G = R^T R (upper triangle of G, column by column) -----------------
  for (int b = warp; b < l; b += nw)
    for (int a = lane; a <= b; a += 32) {
      const double g = G[a + (size_t)b * l];
      Rp[pk(a, b)] = g;
      if (a == b) d0[b] = g;
    }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    // pivot j (one thread); the other threads scale row j - 1 of R by its
    // pivot's reciprocal (nothing reads that row in this phase)
    if (tid == 0) {
      const double d = Rp[pk(j, j)];
      // a pivot that cancelled to rounding level against its own diagonal
      // entry is a numerically dependent row of T: the row of R is dropped
      const bool keep = d0[j] > 1e-300 && d > 1e-13 * d0[j];
      const double r = keep ? sqrt(d) : 0.0;
      s_dinv = keep ? 1.0 / d : 0.0;
      Rp[pk(j, j)] = r;
      // reciprocal of the pivot r for the row scaling in the next phase
      s_rinv[j & 1] = keep ? 1.0 / r : 0.0;
    } else if (j > 0) {
      const double ri = s_rinv[(j - 1) & 1];  // written before the last barrier
      for (int c = j - 1 + tid; c < l; c += nt - 1) Rp[pk(j - 1, c)] *= ri;
    }
    __syncthreads();
    // trailing update with the unscaled row j: A_ab -= A_ja A_jb / d
    const double dinv = s_dinv;
    for (int b = j + 1 + warp; b < l; b += nw) {
      const double ab = Rp[pk(j, b)] * dinv;
      for (int a = j + 1 + lane; a <= b; a += 32) Rp[pk(a, b)] -= Rp[pk(j, a)] * ab;
    }
    __syncthreads();
  }
  // (row l - 1 of R holds only its pivot: nothing left to scale)

  // ---- W = L = R^T: column c of W is row c of R ------------------------
  for (int e = tid; e < l * l; e += nt) {
    const int i = e % l, c = e / l;
    W[e] = i >= c ? Rp[pk(c, i)] : 0.0;
  }
  __syncthreads();

  // ---- one-sided Jacobi sweeps on the columns of W ------------------------
  // gs lanes per column pair (about four rows each, at most 16); warps that
  // hold no pair of the round skip its FP64 work -- GB300's FP64 pipe is
  // shared by every thread of the SM
  const int lp = l + (l & 1);
  int gs = 1;
  while (gs < 16 && gs * 4 < l) gs <<= 1;
  const int grp = tid / gs, g = tid % gs;
  const int warp_first_pair = (warp * 32) / gs;
  const bool warp_busy = warp_first_pair < lp / 2;
  int sweep = 0;
  bool converged = false;
  while (sweep < max_sweeps) {
    // exact squared norms at the start of every sweep (updated by each
    // rotation in between)
    for (int c = warp; c < l; c += nw) {
      double sq = 0.0;
      for (int i = lane; i < l; i += 32) sq = fma(W[i + c * l], W[i + c * l], sq);
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) nrm[c] = sq;
    }
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < lp - 1; ++r) {
      if (warp_busy) {
        int i = -1, j = -1;
        if (grp < lp / 2) {
          round_pair(lp, r, grp, i, j);
          if (j >= l) i = -1;  // the extra player of an odd l
        }
        double c = 0.0;
        if (i >= 0)
          for (int row = g; row < l; row += gs) c = fma(W[row + i * l], W[row + j * l], c);
        c = group_sum(c, gs);
        // the rotation is decided and formed by the group's first lane (FP64
        // square roots and divisions are long instruction sequences on
        // GB300) and broadcast
        double cs = 1.0, sn = 0.0, t = 0.0;
        int rot_i = 0;
        if (i >= 0 && g == 0) {
          const double a = nrm[i], b = nrm[j];
          // |c| > tol sqrt(a b), compared squared (a, b > 0)
          if (c != 0.0 && a > 0.0 && b > 0.0 && c * c > tol * tol * a * b) {
            rot_i = 1;
            // rotation that makes columns i and j orthogonal (Rutishauser's
            // form: t = tan of the angle, the smaller root of t^2 + 2 zeta t - 1)
            const double zeta = (b - a) / (2.0 * c);
            const double az = fabs(zeta);
            t = copysign(1.0, zeta) /
                (az > 1.0 ? az * (1.0 + sqrt(1.0 + 1.0 / (zeta * zeta))) : az + sqrt(1.0 + zeta * zeta));
            cs = 1.0 / sqrt(1.0 + t * t);
            sn = cs * t;
            // the rotated columns' squared norms: a - t c and b + t c
            nrm[i] = a - t * c;
            nrm[j] = b + t * c;
            s_rot = 1;
          }
        }
        const int src = lane & ~(gs - 1);
        rot_i = __shfl_sync(0xffffffffu, rot_i, src);
        cs = __shfl_sync(0xffffffffu, cs, src);
        sn = __shfl_sync(0xffffffffu, sn, src);
        if (rot_i)
          for (int row = g; row < l; row += gs) {
            const double wi = W[row + i * l], wj = W[row + j * l];
            W[row + i * l] = cs * wi - sn * wj;
            W[row + j * l] = sn * wi + cs * wj;
          }
      }
      __syncthreads();
    }
    ++sweep;
    const bool any = s_rot != 0;
    __syncthreads();
    if (!any) {
      converged = true;
      break;
    }
  }

  // ---- sigma_i = ||w_i||, Uhat = W diag(1 / sigma), descending (stable) ----
  for (int c = warp; c < l; c += nw) {
    double sq = 0.0;
    for (int i = lane; i < l; i += 32) sq = fma(W[i + c * l], W[i + c * l], sq);
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) nrm[c] = sqrt(sq);
  }
  __syncthreads();
  if (tid < l) {
    const double v = nrm[tid];
    int rk = 0;
    for (int c = 0; c < l; ++c) rk += (nrm[c] > v) || (nrm[c] == v && c < tid);
    s_rank[tid] = rk;
    sigma[rk] = v;
  }
  __syncthreads();
  for (int e = tid; e < l * l; e += nt) {
    const int row = e % l, c = e / l;
    const double sc = nrm[c];
    K[row + (size_t)s_rank[c] * l] = sc > 0.0 ? W[e] / sc : 0.0;
  }
  __syncthreads();
  // a direction with sigma = 0 (an exactly vanishing row of T) gets a unit
  // vector orthogonal to the others (Gram-Schmidt of the coordinate vectors,
  // twice), so that Uhat stays orthogonal
  if (tid == 0) {
    for (int c = 0; c < l; ++c) {
      if (sigma[c] > 0.0) continue;
      for (int e = 0; e < l; ++e) {
        double* u = K + (size_t)c * l;
        for (int i = 0; i < l; ++i) u[i] = (i == e) ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass)
          for (int o = 0; o < l; ++o) {
            if (o == c || (sigma[o] == 0.0 && o > c)) continue;
            const double* v = K + (size_t)o * l;
            double d = 0.0;
            for (int i = 0; i < l; ++i) d += v[i] * u[i];
            for (int i = 0; i < l; ++i) u[i] -= d * v[i];
          }
        double nn = 0.0;
        for (int i = 0; i < l; ++i) nn += u[i] * u[i];
        if (nn > 0.25) {
          const double inv = 1.0 / sqrt(nn);
          for (int i = 0; i < l; ++i) u[i] *= inv;
          break;
        }
      }
    }
  }
  if (tid == 0) {
    status[5] = (unsigned)sweep;  // diagnostic: sweeps run
    if (!converged) atomicOr(status, ST_NO_CONV);
  }
}

size_t jacobi_smem(int l) {
  const size_t np = (size_t)l * (l + 1) / 2;
  return (((np + 1) / 2) * 2 + (size_t)l * l + 2 * (size_t)l) * sizeof(double);
}

}  // namespace

void prepare_jacobi_kernels() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem(kMaxL));
  });
}

cudaError_t jacobi_svd(cudaStream_t st, int l, const double* G, double* Uhat, double* sigma,
                       unsigned* status, int max_sweeps) {
  prepare_jacobi_kernels();
  // tol: the rounding of a length-l FP64 dot product relative to the norms
  const double tol = fmax(1e-15, sqrt((double)l) * DBL_EPSILON);
  k_jacobi_svd<<<1, kJacThreads, jacobi_smem(l), st>>>(l, G, Uhat, sigma, max_sweeps, tol, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rpod
