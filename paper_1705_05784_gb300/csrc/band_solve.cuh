// Solve with band LU factors (LAPACK gbtrs steps: row interchanges and unit
// L, then U with kl + ku superdiagonals) by one CTA, the right-hand side in
// shared (or global) memory, the band staged through shared memory in
// chunks.  Shared by the one-CTA-per-instance iteration (solve.cu) and the
// whole-GPU iteration's large coarse systems (solve_grid.cu).
#pragma once

namespace fams {
namespace band {

constexpr int CH_MAX = 64;       // band columns per chunk

// Coarse band solve (LAPACK gbtrs steps on the band factors).  Warps
// 0..CS_WARPS-1 run the recurrences column by column, splitting each
// column's rows among them and meeting at a named barrier; the other warps
// stage the next chunk of band columns into shared memory meanwhile (double
// buffer, one CTA barrier per chunk).  The staging warps also turn U's
// diagonal into its reciprocal, so the recurrences never divide.
constexpr int CS_WARPS = 4;
constexpr int CS_T = 32 * CS_WARPS;

__device__ inline void cs_sync() { asm volatile("bar.sync 1, %0;" ::"n"(CS_T) : "memory"); }

// bb: doubles per staged chunk (two chunks in buf), at least kl + ku + 1
__device__ inline void coarse_solve(const double* AB, const int* ipiv, int n, int kl, int ku,
                                    double* yb, double* buf, int* pbuf, int bb) {
  const int kv = kl + ku, ldab = 2 * kl + ku + 1, stride = kv + 1;
  int ch = bb / stride;
  ch = max(1, min(CH_MAX, ch));
  const int nch = (n + ch - 1) / ch;
  const int tid = threadIdx.x;
  const bool comp = tid < CS_T;
  const int T = blockDim.x;
  // forward (L with row interchanges), chunk c holds columns [c ch, (c+1) ch)
  auto load_fwd = [&](int c, double* dst, int* pdst, int t0, int nt) {
    int j0 = c * ch;
    for (int idx = t0; idx < ch * kl; idx += nt) {
      int jj = idx / kl, t = idx % kl + 1, j = j0 + jj;
      dst[jj * stride + t - 1] = (j < n && t <= n - 1 - j) ? AB[(long long)(kv + t) + (long long)ldab * j] : 0.0;
    }
    for (int jj = t0; jj < ch; jj += nt) pdst[jj] = (j0 + jj < n) ? ipiv[j0 + jj] : 0;
  };
  load_fwd(0, buf, pbuf, tid, T);
  __syncthreads();
  for (int c = 0; c < nch; ++c) {
    double* cur = buf + (c & 1) * bb;
    int* pcur = pbuf + (c & 1) * CH_MAX;
    if (comp) {
      int j0 = c * ch;
      for (int jj = 0; jj < ch && j0 + jj < n; ++jj) {
        int j = j0 + jj;
        int km = min(kl, n - 1 - j);
        int pj = pcur[jj];
        if (pj != j) {
          if (tid == 0) {
            double t = yb[j];
            yb[j] = yb[pj];
            yb[pj] = t;
          }
          cs_sync();
        }
        double yj = yb[j];
        for (int t = 1 + tid; t <= km; t += CS_T) yb[j + t] -= cur[jj * stride + t - 1] * yj;
        cs_sync();
      }
    } else if (c + 1 < nch) {
      load_fwd(c + 1, buf + ((c + 1) & 1) * bb, pbuf + ((c + 1) & 1) * CH_MAX, tid - CS_T,
               T - CS_T);
    }
    __syncthreads();
  }
  // backward (U, kv superdiagonals, reciprocal diagonal); chunk c holds
  // columns [n-(c+1)ch, n-c ch).  Rows are updated with x_j = y_j / U_jj
  // while y_j itself is overwritten one column later, when nothing reads it.
  auto load_bwd = [&](int c, double* dst, int t0, int nt) {
    int jhi = n - c * ch, jlo = max(0, jhi - ch);
    for (int idx = t0; idx < (jhi - jlo) * stride; idx += nt) {
      int jj = idx / stride, rr = idx % stride, j = jlo + jj;
      int i = j - kv + rr;
      double v = (i >= 0) ? AB[(long long)rr + (long long)ldab * j] : 0.0;
      dst[jj * stride + rr] = rr == kv ? 1.0 / v : v;
    }
  };
  load_bwd(0, buf, tid, T);
  __syncthreads();
  int prev = -1;
  double xprev = 0.0;
  for (int c = 0; c < nch; ++c) {
    double* cur = buf + (c & 1) * bb;
    if (comp) {
      int jhi = n - c * ch, jlo = max(0, jhi - ch);
      for (int j = jhi - 1; j >= jlo; --j) {
        const double* colj = cur + (j - jlo) * stride;
        double xj = yb[j] * colj[kv];
        if (tid == 0 && prev >= 0) yb[prev] = xprev;
        for (int i = max(0, j - kv) + tid; i < j; i += CS_T) yb[i] -= colj[kv + i - j] * xj;
        prev = j;
        xprev = xj;
        cs_sync();
      }
    } else if (c + 1 < nch) {
      load_bwd(c + 1, buf + ((c + 1) & 1) * bb, tid - CS_T, T - CS_T);
    }
    __syncthreads();
  }
  if (tid == 0 && prev >= 0) yb[prev] = xprev;
  __syncthreads();
}


}  // namespace band
}  // namespace fams
