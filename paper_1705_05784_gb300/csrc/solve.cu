// The two-stage F-AMS iteration (Sec. 3.2, Table 1, steps 3 and 5-8):
//   r = q - A p;  dp1 = P (R A P)^-1 R r;  r1 = r - A dp1;
//   dp2 = (L U)^-1 r1;  p = p + dp1 + dp2
// until ||q - A p||_2 <= tol ||q||_2.
//
// One persistent CTA per instance runs the whole loop, so instances of a
// batch never wait for each other and each result is independent of the
// batch it ran in (every reduction has a fixed order).  The coarse vectors
// live in shared memory; the band triangular solves run in one warp.
#include <algorithm>

#include "batch.cuh"

namespace fams {

namespace {

constexpr int SOLVE_T = 512;

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__global__ void k_make_q(long long n, const double* rhs, const double* qD, double* q) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (rhs ? rhs[i] : 0.0) + qD[i];
}

struct SolveArgs {
  const Inst* inst;
  CoarseSys cs;
  int fe;
  const int* rowptr;
  const int* col;
  const double* val;
  const int* diag;
  const int* p_ptr;
  const int* p_col;
  const double* p_val;
  const int* pt_ptr;
  const int* pt_col;
  const double* pt_val;
  const int* blk_ptr;
  const int* blk_cell;
  const double* F;
  const int* lev_off;
  const int* lev_ptr;
  const int* lev_rows;
  const double* q;
  double* x;
  double* r;
  double* dp;
  double* y;
  double* stat;
  double* hist;
  long long hist_len;
  double* crhs;   // coarse right-hand side of the last sweep (coarse order)
  double* csol;   // coarse solution of the last sweep
  double tol;
};

// coarse solve of the band LU (gbtrs scheme) by warp 0, vector in shared memory
__device__ void band_solve_warp(const double* AB, const int* ipiv, int n, int kl, int ku,
                                double* yb) {
  int lane = threadIdx.x & 31;
  int kv = kl + ku, ldab = 2 * kl + ku + 1;
  // L: forward with row interchanges
  for (int j = 0; j < n; ++j) {
    int km = min(kl, n - 1 - j);
    int pj = ipiv[j];
    if (lane == 0 && pj != j) {
      double t = yb[j];
      yb[j] = yb[pj];
      yb[pj] = t;
    }
    __syncwarp();
    double yj = yb[j];
    for (int t = 1 + lane; t <= km; t += 32)
      yb[j + t] -= AB[(long long)(kv + t) + (long long)ldab * j] * yj;
    __syncwarp();
  }
  // U: backward, kv superdiagonals
  for (int j = n - 1; j >= 0; --j) {
    double yj = yb[j] / AB[(long long)kv + (long long)ldab * j];
    __syncwarp();
    if (lane == 0) yb[j] = yj;
    int lo = max(0, j - kv);
    for (int i = lo + lane; i < j; i += 32)
      yb[i] -= AB[(long long)(kv + i - j) + (long long)ldab * j] * yj;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(SOLVE_T) k_solve(SolveArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ int s_done;
  int ii = blockIdx.x;
  const Inst& I = a.inst[ii];
  int n = I.n, ro = I.row_off, nc = I.nc, co = I.nc_off;
  double* yb = sm;        // coarse vector in band order
  double* ecs = sm + nc;  // coarse correction in coarse order
  const double* AB = a.cs.band + a.cs.band_off[ii];
  const int* ipiv = a.cs.ipiv + co;
  const int* perm = a.cs.perm + co;
  int kl = a.cs.kl[ii], ku = a.cs.ku[ii];
  const int* lp = a.lev_ptr + a.lev_off[ii];
  int nlev = I.nlev;
  // ||q||
  double acc = 0.0;
  for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) acc += a.q[i] * a.q[i];
  double qn = sqrt(block_sum(acc, red));
  if (!(qn > 0.0)) qn = 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    // step 3: r = q - A p
    acc = 0.0;
    for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
      double s = a.q[i];
      for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) s -= a.val[p] * a.x[a.col[p]];
      a.r[i] = s;
      acc += s * s;
    }
    rel = sqrt(block_sum(acc, red)) / qn;
    if (threadIdx.x == 0) {
      a.hist[(long long)ii * a.hist_len + it] = rel;
      s_done = (rel <= a.tol || it >= I.max_iter || !isfinite(rel));
    }
    __syncthreads();
    if (s_done) break;
    // step 5: coarse right-hand side R r, in band order
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      int c = co + perm[k];
      double s = 0.0;
      if (I.restriction == FAMS_R_FE) {
        for (int p = a.pt_ptr[c]; p < a.pt_ptr[c + 1]; ++p) s += a.pt_val[p] * a.r[a.pt_col[p]];
      } else {
        for (int p = a.blk_ptr[c]; p < a.blk_ptr[c + 1]; ++p) s += a.r[a.blk_cell[p]];
      }
      yb[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) a.crhs[co + perm[k]] = yb[k];
    if (threadIdx.x < 32) band_solve_warp(AB, ipiv, nc, kl, ku, yb);
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      ecs[perm[k]] = yb[k];
      a.csol[co + perm[k]] = yb[k];
    }
    __syncthreads();
    // dp1 = P e_c
    for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
      double s = 0.0;
      for (int p = a.p_ptr[i]; p < a.p_ptr[i + 1]; ++p) s += a.p_val[p] * ecs[a.p_col[p]];
      a.dp[i] = s;
    }
    __syncthreads();
    // steps 6-7, L sweep: y = L^-1 (r - A dp1)
    for (int l = 0; l < nlev; ++l) {
      for (int t = lp[l] + threadIdx.x; t < lp[l + 1]; t += blockDim.x) {
        int i = a.lev_rows[t];
        double s = a.r[i];
        int d = a.diag[i];
        for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) s -= a.val[p] * a.dp[a.col[p]];
        for (int p = a.rowptr[i]; p < d; ++p) s -= a.F[p] * a.y[a.col[p]];
        a.y[i] = s;
      }
      __syncthreads();
    }
    // U sweep and step 8: p = p + dp1 + dp2
    for (int l = nlev - 1; l >= 0; --l) {
      for (int t = lp[l] + threadIdx.x; t < lp[l + 1]; t += blockDim.x) {
        int i = a.lev_rows[t];
        int d = a.diag[i];
        double s = a.y[i];
        for (int p = d + 1; p < a.rowptr[i + 1]; ++p) s -= a.F[p] * a.y[a.col[p]];
        double xi = s / a.F[d];
        a.y[i] = xi;
        a.x[i] = (a.x[i] + a.dp[i]) + xi;
      }
      __syncthreads();
    }
    ++it;
  }
  if (threadIdx.x == 0) {
    a.stat[4 * ii + 0] = it;
    a.stat[4 * ii + 1] = rel;
    a.stat[4 * ii + 2] = (rel <= a.tol) ? 1.0 : 0.0;
    a.stat[4 * ii + 3] = qn;
  }
}

}  // namespace

int phase_alloc_work(Batch& b) {
  long long n = b.tot_row;
  FAMS_TRY(b.alloc((void**)&b.q, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.x, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.r, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.dp, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.y, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.stat, sizeof(double) * 4 * b.B));
  int mi = 0;
  for (auto& I : b.h) mi = std::max(mi, I.max_iter);
  b.hist_len = mi + 1;
  FAMS_TRY(b.alloc((void**)&b.rc, sizeof(double) * (b.tot_nc + 1)));
  FAMS_TRY(b.alloc((void**)&b.ec, sizeof(double) * (b.tot_nc + 1)));
  FAMS_TRY(b.alloc((void**)&b.hist, sizeof(double) * b.hist_len * b.B));
  return FAMS_OK;
}

int make_q(Batch& b, const double* rhs_dev) {
  long long n = b.tot_row;
  fams::note_launch(), k_make_q<<<grid_for(n, 256), 256, 0, b.stream>>>(n, rhs_dev, b.qD, b.q);
  FAMS_CUDA(cudaGetLastError());
  return FAMS_OK;
}

int run_solve(Batch& b, double tol, float* ms) {
  SolveArgs a;
  a.inst = b.d_inst;
  a.cs = b.cs[0];
  a.fe = b.h[0].restriction == FAMS_R_FE;
  a.rowptr = b.rowptr; a.col = b.col; a.val = b.val; a.diag = b.diag;
  a.p_ptr = b.p_ptr; a.p_col = b.p_col; a.p_val = b.p_val;
  a.pt_ptr = b.pt_ptr; a.pt_col = b.pt_col; a.pt_val = b.pt_val;
  a.blk_ptr = b.blk_ptr; a.blk_cell = b.blk_cell;
  a.F = b.ilu; a.lev_off = b.lev_off; a.lev_ptr = b.lev_ptr; a.lev_rows = b.lev_rows;
  a.q = b.q; a.x = b.x; a.r = b.r; a.dp = b.dp; a.y = b.y; a.stat = b.stat;
  a.hist = b.hist; a.hist_len = b.hist_len;
  a.crhs = b.rc; a.csol = b.ec;
  a.tol = tol;
  int maxnc = 0;
  for (auto& I : b.h) maxnc = std::max(maxnc, I.nc);
  size_t smem = sizeof(double) * 2 * (size_t)maxnc;
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  if ((long long)smem + 1024 > max_smem) {
    set_error("coarse system too large for the shared-memory coarse solve");
    return FAMS_ECAPACITY;
  }
  FAMS_CUDA(cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - 1024));
  cudaEvent_t e0, e1;
  FAMS_CUDA(cudaEventCreate(&e0));
  FAMS_CUDA(cudaEventCreate(&e1));
  FAMS_CUDA(cudaEventRecord(e0, b.stream));
  fams::note_launch(), k_solve<<<b.B, SOLVE_T, smem, b.stream>>>(a);
  FAMS_CUDA(cudaGetLastError());
  FAMS_CUDA(cudaEventRecord(e1, b.stream));
  FAMS_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  FAMS_CUDA(cudaEventElapsedTime(&t, e0, e1));
  if (ms) *ms = t;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return FAMS_OK;
}

}  // namespace fams
