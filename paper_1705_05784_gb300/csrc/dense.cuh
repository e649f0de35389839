// Small dense solves shared by the dual-block basis solves and the local
// problems of the flux reconstruction.
//
// A group of threads (one warp, or a whole CTA) eliminates [M | R] in place:
// M is n x n, R holds k right-hand sides, stored row-major with leading
// dimension ld = n + k in shared (or global) memory.  Gaussian elimination
// without pivoting, then back substitution, leaves M^-1 R in the R columns.
// No pivoting is needed for the matrices solved here: the dual-block
// matrices are symmetric positive definite, and the local problems are
// nonsingular M-matrices (weakly chained diagonally dominant); both have an
// LU factorisation without row exchanges whose Schur complements keep
// positive pivots.
//
// Step j reads row j and column j and writes only rows i > j and columns
// c > j, so one barrier per step suffices.  Rows whose entry in column j is
// exactly zero are skipped: with the band-like ordering of the blocks (cells
// sorted by index) fill-in stays inside the profile, so the work tracks the
// profile rather than n^3.
#pragma once

#include "common.cuh"

namespace fams {

struct WarpGroup {
  static constexpr bool per_warp = true;
  __device__ static int rank() { return threadIdx.x & 31; }
  __device__ static int size() { return 32; }
  __device__ static void sync() { __syncwarp(); }
};

struct CtaGroup {
  static constexpr bool per_warp = false;
  __device__ static int rank() { return threadIdx.x; }
  __device__ static int size() { return blockDim.x; }
  __device__ static void sync() { __syncthreads(); }
};

// Returns false (uniformly over the group) when a pivot is not positive and
// finite; M and R are then partly eliminated.
template <class G>
__device__ bool ge_solve(double* M, int ld, int n, int k) {
  const int gr = G::rank(), gs = G::size();
  const int nw = gs >> 5, w = gr >> 5, lane = gr & 31;
  const int ncol = n + k;
  for (int j = 0; j < n; ++j) {
    const double piv = M[(long long)j * ld + j];
    if (!(piv > 0.0) || !isfinite(piv)) return false;
    const double inv = 1.0 / piv;
    const double* rj = M + (long long)j * ld;
    for (int i = j + 1 + w; i < n; i += nw) {
      double* ri = M + (long long)i * ld;
      const double f = ri[j] * inv;
      if (f != 0.0)
        for (int c = j + 1 + lane; c < ncol; c += 32) ri[c] -= f * rj[c];
    }
    G::sync();
  }
  // back substitution on the unscaled right-hand sides: x_j = R_j / U_jj,
  // R_i -= U_ij x_j for i < j
  for (int j = n - 1; j > 0; --j) {
    const double inv = 1.0 / M[(long long)j * ld + j];
    const double* xj = M + (long long)j * ld + n;
    for (int i = w; i < j; i += nw) {
      double* ri = M + (long long)i * ld;
      const double u = ri[j];
      if (u != 0.0)
        for (int q = lane; q < k; q += 32) ri[n + q] -= u * (xj[q] * inv);
    }
    G::sync();
  }
  for (int t = gr; t < n * k; t += gs) {
    int i = t / k, q = t - i * k;
    M[(long long)i * ld + n + q] /= M[(long long)i * ld + i];
  }
  G::sync();
  return true;
}

}  // namespace fams
