// Small dense solves shared by the dual-block basis solves and the local
// problems of the flux reconstruction.
//
// A group of threads (one warp, or a whole CTA) eliminates [M | R] in place:
// M is n x n with lower bandwidth bl and upper bandwidth bu, R holds k
// right-hand sides; each row keeps its band and its right-hand sides (band
// storage, below) in shared (or global) memory.  Gaussian elimination without pivoting, then
// back substitution, leaves M^-1 R in the R columns.  No pivoting is needed
// for the matrices solved here: the dual-block matrices are symmetric
// positive definite, and the local problems are nonsingular M-matrices
// (weakly chained diagonally dominant); both have an LU factorisation
// without row exchanges whose pivots stay positive.  Without row exchanges
// the factors keep the bandwidths of M, so step j touches only rows
// j+1..j+bl and columns j+1..j+bu (plus the right-hand sides).
//
// FP64 issue slots are scarce on this GPU, so each step is one flat pass over
// its (row, column) pairs, and pivots enter as reciprocals: the thread that
// finishes the next pivot in step j stores its reciprocal for step j + 1.
// Step j reads row j and column j and writes only rows and columns beyond
// j, so one barrier per step suffices.
#pragma once

#include "common.cuh"

namespace fams {

struct WarpGroup {
  static constexpr bool per_warp = true;
  __device__ static int rank() { return threadIdx.x & 31; }
  __device__ static int size() { return 32; }
  __device__ static void sync() { __syncwarp(); }
  __device__ static int max(int v, int*) { return __reduce_max_sync(0xffffffffu, v); }
};

struct CtaGroup {
  static constexpr bool per_warp = false;
  __device__ static int rank() { return threadIdx.x; }
  __device__ static int size() { return blockDim.x; }
  __device__ static void sync() { __syncthreads(); }
  // scratch: 32 ints of shared memory
  __device__ static int max(int v, int* scratch) {
    v = __reduce_max_sync(0xffffffffu, v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = m > scratch[w] ? m : scratch[w];
    __syncthreads();
    return m;
  }
};

// pivot usable: positive and finite (integer test, no FP64 issue slot)
__device__ inline bool pivot_ok(double v) {
  long long b = __double_as_longlong(v);
  return b > 0 && b < 0x7ff0000000000000LL;
}

// Band storage: row i holds M(i, i - bl .. i + bu) at offsets 0 .. W - 1
// (column c at c - i + bl, W = bl + bu + 1), then its k right-hand sides at
// offsets W .. W + k - 1; ld >= W + k.  Without row exchanges the factors
// fill only the band.  inv: n doubles of scratch (same memory space as M).
// Returns false (uniformly over the group) when a pivot is not positive and
// finite; M and R are then partly eliminated.
template <class G>
__device__ bool ge_solve(double* M, int ld, int n, int k, int bl, int bu, double* inv) {
  const int gr = G::rank(), gs = G::size();
  const int W = bl + bu + 1;
  if (n == 0) return true;
  if (gr == 0) inv[0] = 1.0 / M[bl];
  G::sync();
  for (int j = 0; j < n; ++j) {
    const double* rj = M + (long long)j * ld;
    if (!pivot_ok(rj[bl])) return false;
    const int rows = min(n - 1, j + bl) - j;
    const int wb = min(n - 1, j + bu) - j;
    const int w = wb + k;
    const double ij = inv[j];
    for (int t = gr; t < rows * w; t += gs) {
      int r = t / w, cc = t - r * w;
      double* ri = M + (long long)(j + 1 + r) * ld;
      // column j + 1 + cc (band) or right-hand side cc - wb, in row i = j + 1 + r and in row j
      int oi = cc < wb ? cc - r + bl : W + (cc - wb);
      int oj = cc < wb ? cc + 1 + bl : W + (cc - wb);
      double v = ri[oi] - (ri[bl - 1 - r] * ij) * rj[oj];
      ri[oi] = v;
      if (r == 0 && cc == 0) inv[j + 1] = 1.0 / v;   // (j+1, j+1): the next pivot is final
    }
    if ((rows == 0 || wb == 0) && j + 1 < n && gr == 0) inv[j + 1] = 1.0 / M[(long long)(j + 1) * ld + bl];
    G::sync();
  }
  // back substitution on the unscaled right-hand sides: x_j = R_j / U_jj,
  // R_i -= U_ij x_j for j - bu <= i < j
  for (int j = n - 1; j > 0; --j) {
    const int i0 = max(0, j - bu);
    const int rows = j - i0;
    const double ij = inv[j];
    const double* xj = M + (long long)j * ld + W;
    for (int t = gr; t < rows * k; t += gs) {
      int r = t / k, q = t - r * k;
      int i = i0 + r;
      double* ri = M + (long long)i * ld;
      ri[W + q] -= ri[j - i + bl] * (xj[q] * ij);
    }
    G::sync();
  }
  for (int t = gr; t < n * k; t += gs) {
    int i = t / k, q = t - i * k;
    M[(long long)i * ld + W + q] *= inv[i];
  }
  G::sync();
  return true;
}

}  // namespace fams
