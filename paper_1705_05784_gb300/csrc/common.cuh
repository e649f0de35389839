// Internal declarations shared by the libfams translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fams.h"

namespace fams {

// Status word written by kernels when they detect a failure they cannot
// report otherwise (they never trap): the host reads it after each phase.
enum DevErr {
  DERR_NONE = 0,
  DERR_BREAKDOWN = 1,   // zero / non-finite pivot
  DERR_CAPACITY = 2,    // local problem larger than the compiled limit
  DERR_INVAL = 3,       // input the method cannot handle
  DERR_TIMEOUT = 4,     // bounded wait gave up
  DERR_FLOATING = 5     // dual block with no link to known basis values
};

constexpr int RANK_I = 0, RANK_F = 1, RANK_E = 2, RANK_V = 3;
// per-instance solve statistics: iterations, relative residual, converged,
// ||q||, SM cycles of the six phases of a sweep (residual, restriction, band
// solve, prolongation + r1, L sweep, U sweep), singular-coarse flag, spare
constexpr int STAT_W = 12;
constexpr int STAT_BAD = 10;
constexpr int PK = 4;  // factor entries per row kept inline in the level-ordered layout
constexpr int MAX_OVERLAP = 8;        // matrix columns one fracture cell may cross
constexpr double ZERO_PIECE = 1e-12;  // x h_f
constexpr double DIST_FLOOR = 1e-3;   // x h_f
// a pivot at most this fraction of the largest entry of its row (as
// assembled) is numerically zero: the coarse system is singular
constexpr double SING_EPS = 1e-13;

// Per-instance description, mirrored on the device.  Offsets index the
// concatenated (block-diagonal) arrays of a batch.
struct Inst {
  int dim, nx, ny, nz;
  double dx, dy, dz;
  int bc_mask;
  double bc_val[6];
  double aperture, hf;
  int cx, cy, cz, dmin, fcz, basis, restriction, precision, max_iter;
  int krylov, restart;  // outer iteration; GMRES cycle length
  int merge_cap;        // Coupled: largest block merged across the media (0: none)
  int grid_solve;       // single instance on every SM: 0 auto, 1 always, -1 never
  int subblock;         // 1: the sub-block smoothing stage after ILU(0)
  int bf16_p;           // mixed precision: P and P^T values stored in BF16
  int coarse_mode;      // whole-GPU coarse solve: 0 auto, 1 A_c^-1, 2 band factors
  double alpha;
  // sizes and offsets
  int nm, m_off;      // matrix cells
  int nfr, fr_off;    // input fractures
  int nf, fc_off;     // fracture cells
  int ns, s_off;      // strike (x-y projection) cells
  int n, row_off;     // unknowns
  int nw, w_off;      // rate-controlled wells (unknowns after the fracture cells)
  int nperf, perf_off;  // well perforations (rate wells first, then pressure wells)
  int nnc, nnc_off;   // matrix-fracture connections
  int nff, ff_off;    // fracture-fracture connections
  int ninter, inter_off;  // fracture pairs examined for intersections
  int nc, nc_off;     // coarse unknowns
  int ncm;            // matrix coarse unknowns
  int nbx, nby, nbz;  // matrix primal blocks per axis
  int nnet, net_off;  // fracture networks
  long long nnz_off; int nnz;  // CSR of A
  int nlev;           // ILU(0) levels
  int band_kl, band_ku;        // coarse band LU
  long long band_off;          // offset of the band storage (doubles)
  long long ac_off;            // offset of the dense coarse operator (doubles)
};

struct Dev;  // device arrays of a batch (defined in batch.cuh)

#define FAMS_CUDA(call)                                                        \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      fams::set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " + \
                      __FILE__ + ":" + std::to_string(__LINE__));              \
      return FAMS_ECUDA;                                                       \
    }                                                                          \
  } while (0)

#define FAMS_TRY(expr)          \
  do {                          \
    int s_ = (expr);            \
    if (s_ != FAMS_OK) return s_; \
  } while (0)

void set_error(const std::string& msg);
void note_launch();  // counts every kernel launch of the library (fams_launch_count)
void note_alloc();   // counts every device allocation of the library (fams_alloc_count)

inline int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (int)g;
}

// upper_bound-1 on a non-decreasing int array: index i with a[i] <= v < a[i+1]
__host__ __device__ inline int find_segment(const int* a, int n, long long v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if ((long long)a[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace fams
