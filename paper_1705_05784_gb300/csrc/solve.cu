// The two-stage F-AMS iteration (Sec. 3.2, Table 1, steps 3 and 5-8):
//   r = q - A p;  dp1 = P (R A P)^-1 R r;  r1 = r - A dp1;
//   dp2 = (L U)^-1 r1;  p = p + dp1 + dp2
// until ||q - A p||_2 <= tol ||q||_2.
//
// One persistent CTA per instance runs the whole loop, so instances of a
// batch never wait for each other and each result is independent of the
// batch it ran in (every reduction has a fixed order).  Everything on the
// loop's critical path is arranged so that a step waits for at most one
// memory round trip:
//  * row-parallel passes (residual, r1, P e_c) keep four rows per thread in
//    flight;
//  * the coarse band solve runs in warp 0 on factor columns that the other
//    warps stage into shared memory one chunk ahead (double buffer);
//  * the ILU(0) sweeps go level by level; the row data of the next level
//    (indices, factors, right-hand side) is loaded before the barrier, so a
//    level costs one gather of the previous level's results.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>

#include "batch.cuh"

namespace fams {

namespace {

constexpr int SOLVE_T = 512;
constexpr int ROWS_ILP = 4;
constexpr int BAND_BUF = 3072;   // doubles per staged chunk of band columns (24 KiB)
constexpr int CH_MAX = 64;       // band columns per chunk

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
  // level-ordered factors (position t) and right-hand side
  const int* pk_pos;
  const int* pk_nl;
  const int* pk_lp;
  const int* pk_lc;
  const double* pk_lv;
  const int* pk_nu;
  const int* pk_uc;
  const double* pk_uv;
  const double* pk_ud;
  double* ylev;
  long long ntot;  // rows of the batch (stride of the PK arrays)
  double tol;
};

// y[i] = b[i] - sum_p val[p] v[col[p]] for the instance's rows, four rows per
// thread in flight; returns this thread's sum of y^2 when `norm`
__device__ inline double rows_residual(const SolveArgs& a, int ro, int n, const double* b,
                                       const double* v, double* y, bool norm,
                                       double* ylev = nullptr) {
  double acc = 0.0;
  const int T = blockDim.x;
  for (int i0 = ro + threadIdx.x; i0 < ro + n; i0 += ROWS_ILP * T) {
    int rs[ROWS_ILP], re[ROWS_ILP];
    double s[ROWS_ILP];
    int m = 0;
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * T;
      bool ok = i < ro + n;
      rs[k] = ok ? a.rowptr[i] : 0;
      re[k] = ok ? a.rowptr[i + 1] : 0;
      s[k] = ok ? b[i] : 0.0;
      m = max(m, re[k] - rs[k]);
    }
    for (int e = 0; e < m; ++e) {
#pragma unroll
      for (int k = 0; k < ROWS_ILP; ++k) {
        int p = rs[k] + e;
        if (p < re[k]) s[k] -= a.val[p] * v[a.col[p]];
      }
    }
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * T;
      if (i < ro + n) {
        y[i] = s[k];
        if (ylev) ylev[a.pk_pos[i]] = s[k];
        if (norm) acc += s[k] * s[k];
      }
    }
  }
  return acc;
}

// coarse band solve: warp 0 runs the recurrences on columns staged in shared
// memory, the other warps stage the next chunk meanwhile
__device__ void coarse_solve(const double* AB, const int* ipiv, int n, int kl, int ku, double* yb,
                             double* buf, int* pbuf) {
  const int kv = kl + ku, ldab = 2 * kl + ku + 1, stride = kv + 1;
  int ch = BAND_BUF / stride;
  ch = max(1, min(CH_MAX, ch));
  const int nch = (n + ch - 1) / ch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  load_fwd(0, buf, pbuf, threadIdx.x, T);
  __syncthreads();
  for (int c = 0; c < nch; ++c) {
    double* cur = buf + (c & 1) * BAND_BUF;
    int* pcur = pbuf + (c & 1) * CH_MAX;
    if (warp == 0) {
      int j0 = c * ch;
      for (int jj = 0; jj < ch && j0 + jj < n; ++jj) {
        int j = j0 + jj;
        int km = min(kl, n - 1 - j);
        int pj = pcur[jj];
        if (lane == 0 && pj != j) {
          double t = yb[j];
          yb[j] = yb[pj];
          yb[pj] = t;
        }
        __syncwarp();
        double yj = yb[j];
        for (int t = 1 + lane; t <= km; t += 32) yb[j + t] -= cur[jj * stride + t - 1] * yj;
        __syncwarp();
      }
    } else if (c + 1 < nch) {
      load_fwd(c + 1, buf + ((c + 1) & 1) * BAND_BUF, pbuf + ((c + 1) & 1) * CH_MAX,
               threadIdx.x - 32, T - 32);
    }
    __syncthreads();
  }
  // backward (U, kv superdiagonals); chunk c holds columns [n-(c+1)ch, n-c ch)
  auto load_bwd = [&](int c, double* dst, int t0, int nt) {
    int jhi = n - c * ch, jlo = max(0, jhi - ch);
    for (int idx = t0; idx < (jhi - jlo) * stride; idx += nt) {
      int jj = idx / stride, rr = idx % stride, j = jlo + jj;
      int i = j - kv + rr;
      dst[jj * stride + rr] = (i >= 0) ? AB[(long long)rr + (long long)ldab * j] : 0.0;
    }
  };
  load_bwd(0, buf, threadIdx.x, T);
  __syncthreads();
  for (int c = 0; c < nch; ++c) {
    double* cur = buf + (c & 1) * BAND_BUF;
    if (warp == 0) {
      int jhi = n - c * ch, jlo = max(0, jhi - ch);
      for (int j = jhi - 1; j >= jlo; --j) {
        const double* colj = cur + (j - jlo) * stride;
        double yj = yb[j] / colj[kv];
        __syncwarp();
        if (lane == 0) yb[j] = yj;
        for (int i = max(0, j - kv) + lane; i < j; i += 32) yb[i] -= colj[kv + i - j] * yj;
        __syncwarp();
      }
    } else if (c + 1 < nch) {
      load_bwd(c + 1, buf + ((c + 1) & 1) * BAND_BUF, threadIdx.x - 32, T - 32);
    }
    __syncthreads();
  }
}

// one row of a triangular sweep, loaded from the level-ordered layout: every
// address depends only on the position t, so the loads of a whole level are
// coalesced and independent of the sweep's results
struct SweepRow {
  int t, i, cnt, p;
  double base, diag;
  int c[PK];
  double f[PK];
};

__device__ inline void sweep_load(const SolveArgs& a, const int* lp, int l, int nlev, bool lower,
                                  SweepRow& s) {
  s.t = -1;
  if (l < 0 || l >= nlev) return;
  int t = lp[l] + threadIdx.x;
  if (t >= lp[l + 1]) return;
  s.t = t;
  s.i = a.lev_rows[t];
  s.base = a.ylev[t];
  if (lower) {
    s.cnt = a.pk_nl[t];
    s.p = a.pk_lp[t];
    s.diag = 1.0;
  } else {
    s.cnt = a.pk_nu[t];
    s.diag = a.pk_ud[t];
  }
  const int* pc = lower ? a.pk_lc : a.pk_uc;
  const double* pv = lower ? a.pk_lv : a.pk_uv;
#pragma unroll
  for (int k = 0; k < PK; ++k) {
    s.c[k] = pc[(long long)k * a.ntot + t];
    s.f[k] = pv[(long long)k * a.ntot + t];
  }
}

// shared-memory layout of the solve kernels (doubles): the coarse vector in
// band order, the coarse correction in coarse order, two staged chunks of
// band columns; the GMRES kernel adds its small dense arrays after them
struct SolveSmem {
  double* yb;
  double* ecs;
  double* buf;
  int* pbuf;
};

// Steps 5-7 of Table 1 on a residual r (SM cycles of the phases added to cyc
// by thread 0):
//   dp = P A_c^-1 R r;  y = r - A dp (also in level order);
//   out = (base + dp) + (LU)^-1 y   (base null: out = dp + (LU)^-1 y)
// out may alias base; r, dp and out must not alias y or ylev.
__device__ __forceinline__ void two_stage(const SolveArgs& a, const Inst& I, int ii, const double* r, double* dp,
                          double* out, const double* base, const SolveSmem& S, long long* cyc) {
  const int n = I.n, ro = I.row_off, nc = I.nc, co = I.nc_off;
  const double* AB = a.cs.band + a.cs.band_off[ii];
  const int* ipiv = a.cs.ipiv + co;
  const int* perm = a.cs.perm + co;
  const int kl = a.cs.kl[ii], ku = a.cs.ku[ii];
  const int* lp = a.lev_ptr + a.lev_off[ii];
  const int nlev = I.nlev;
  const int T = blockDim.x;
  long long t1 = clock64();
  // step 5: coarse right-hand side R r, in band order
  for (int k = threadIdx.x; k < nc; k += T) {
    int c = co + perm[k];
    double s0 = 0.0, s1 = 0.0;
    if (I.restriction == FAMS_R_FE) {
      int p = a.pt_ptr[c], e = a.pt_ptr[c + 1];
      for (; p + 1 < e; p += 2) {
        s0 += a.pt_val[p] * r[a.pt_col[p]];
        s1 += a.pt_val[p + 1] * r[a.pt_col[p + 1]];
      }
      if (p < e) s0 += a.pt_val[p] * r[a.pt_col[p]];
    } else {
      int p = a.blk_ptr[c], e = a.blk_ptr[c + 1];
      for (; p + 1 < e; p += 2) {
        s0 += r[a.blk_cell[p]];
        s1 += r[a.blk_cell[p + 1]];
      }
      if (p < e) s0 += r[a.blk_cell[p]];
    }
    S.yb[k] = s0 + s1;
    a.crhs[co + perm[k]] = s0 + s1;
  }
  __syncthreads();
  long long t1b = clock64();
  coarse_solve(AB, ipiv, nc, kl, ku, S.yb, S.buf, S.pbuf);
  for (int k = threadIdx.x; k < nc; k += T) {
    S.ecs[perm[k]] = S.yb[k];
    a.csol[co + perm[k]] = S.yb[k];
  }
  __syncthreads();
  long long t2 = clock64();
  // dp1 = P e_c
  for (int i0 = ro + threadIdx.x; i0 < ro + n; i0 += ROWS_ILP * T) {
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * T;
      if (i < ro + n) {
        double s = 0.0;
        for (int p = a.p_ptr[i]; p < a.p_ptr[i + 1]; ++p) s += a.p_val[p] * S.ecs[a.p_col[p]];
        dp[i] = s;
      }
    }
  }
  __syncthreads();
  // step 6: r1 = r - A dp1, stored in y (natural order) and ylev (level order)
  rows_residual(a, ro, n, r, dp, a.y, false, a.ylev);
  __syncthreads();
  long long t3 = clock64();
  // step 7, L sweep in place: y_i = r1_i - sum_{j<i} L_ij y_j
  SweepRow cur, nxt;
  sweep_load(a, lp, 0, nlev, true, cur);
  for (int l = 0; l < nlev; ++l) {
    sweep_load(a, lp, l + 1, nlev, true, nxt);
    if (cur.t >= 0) {
      double s = cur.base;
#pragma unroll
      for (int k = 0; k < PK; ++k)
        if (k < cur.cnt) s -= cur.f[k] * a.y[cur.c[k]];
      for (int p = cur.p + PK; p < cur.p + cur.cnt; ++p) s -= a.F[p] * a.y[a.col[p]];
      a.y[cur.i] = s;
      a.ylev[cur.t] = s;
    }
    for (int t = lp[l] + threadIdx.x + T; t < lp[l + 1]; t += T) {
      int i = a.lev_rows[t];
      double s = a.ylev[t];
      for (int p = a.rowptr[i]; p < a.diag[i]; ++p) s -= a.F[p] * a.y[a.col[p]];
      a.y[i] = s;
      a.ylev[t] = s;
    }
    __syncthreads();
    cur = nxt;
  }
  long long t4 = clock64();
  // U sweep and step 8: out = (base + dp1) + dp2
  sweep_load(a, lp, nlev - 1, nlev, false, cur);
  for (int l = nlev - 1; l >= 0; --l) {
    sweep_load(a, lp, l - 1, nlev, false, nxt);
    if (cur.t >= 0) {
      double s = cur.base;
      double xo = base ? base[cur.i] : 0.0, dpo = dp[cur.i];
#pragma unroll
      for (int k = 0; k < PK; ++k)
        if (k < cur.cnt) s -= cur.f[k] * a.y[cur.c[k]];
      if (cur.cnt > PK) {
        int d = a.diag[cur.i];
        for (int p = d + 1 + PK; p <= d + cur.cnt; ++p) s -= a.F[p] * a.y[a.col[p]];
      }
      double xi = s / cur.diag;
      a.y[cur.i] = xi;
      out[cur.i] = (xo + dpo) + xi;
    }
    for (int t = lp[l] + threadIdx.x + T; t < lp[l + 1]; t += T) {
      int i = a.lev_rows[t];
      int d = a.diag[i];
      double s = a.ylev[t];
      for (int p = d + 1; p < a.rowptr[i + 1]; ++p) s -= a.F[p] * a.y[a.col[p]];
      double xi = s / a.F[d];
      a.y[i] = xi;
      out[i] = ((base ? base[i] : 0.0) + dp[i]) + xi;
    }
    __syncthreads();
    cur = nxt;
  }
  long long t5 = clock64();
  if (cyc) {
    cyc[1] += t1b - t1;
    cyc[2] += t2 - t1b;
    cyc[3] += t3 - t2;
    cyc[4] += t4 - t3;
    cyc[5] += t5 - t4;
  }
}

__device__ inline SolveSmem solve_smem(double* sm, int nc, int* pbuf) {
  return SolveSmem{sm, sm + nc, sm + 2 * nc, pbuf};
}

__device__ inline void write_stats(const SolveArgs& a, int ii, int it, double rel, double qn,
                                   const long long* cyc) {
  if (threadIdx.x == 0) {
    a.stat[STAT_W * ii + 0] = it;
    a.stat[STAT_W * ii + 1] = rel;
    a.stat[STAT_W * ii + 2] = (rel <= a.tol) ? 1.0 : 0.0;
    a.stat[STAT_W * ii + 3] = qn;
    for (int k = 0; k < 6; ++k) a.stat[STAT_W * ii + 4 + k] = (double)cyc[k];
    a.stat[STAT_W * ii + STAT_BAD] = a.cs.bad[ii] ? 1.0 : 0.0;  // singular coarse system
  }
}

__global__ void __launch_bounds__(SOLVE_T, 2) k_solve(SolveArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ int s_done;
  __shared__ int pbuf[2 * CH_MAX];
  int ii = blockIdx.x;
  const Inst& I = a.inst[ii];
  if (I.krylov != FAMS_KRYLOV_NONE) return;
  const int n = I.n, ro = I.row_off;
  const SolveSmem S = solve_smem(sm, I.nc, pbuf);
  const int T = blockDim.x;
  // ||q||
  double acc = 0.0;
  for (int i = ro + threadIdx.x; i < ro + n; i += T) acc += a.q[i] * a.q[i];
  double qn = sqrt(block_sum(acc, red));
  if (!(qn > 0.0)) qn = 1.0;
  int it = 0;
  double rel = 0.0;
  // SM cycles per phase (thread 0, between barriers): residual, restriction,
  // band solve, prolongation + r1, L sweep, U sweep
  long long cyc[6] = {0, 0, 0, 0, 0, 0};
  for (;;) {
    long long t0 = clock64();
    // step 3: r = q - A p
    acc = rows_residual(a, ro, n, a.q, a.x, a.r, true);
    rel = sqrt(block_sum(acc, red)) / qn;
    if (threadIdx.x == 0) {
      a.hist[(long long)ii * a.hist_len + it] = rel;
      s_done = (rel <= a.tol || it >= I.max_iter || !isfinite(rel) || a.cs.bad[ii]);
    }
    __syncthreads();
    cyc[0] += clock64() - t0;
    if (s_done) break;
    // steps 5-8: p = p + dp1 + dp2
    two_stage(a, I, ii, a.r, a.dp, a.x, a.x, S, cyc);
    ++it;
  }
  write_stats(a, ii, it, rel, qn, cyc);
}

// GMRES helpers on the vectors of one instance (rows [ro, ro + n)); every
// reduction has a fixed order, so results do not depend on the batch

// y = A v; returns this thread's sum of y^2
__device__ inline double rows_apply(const SolveArgs& a, int ro, int n, const double* v, double* y) {
  double acc = 0.0;
  const int T = blockDim.x;
  for (int i0 = ro + threadIdx.x; i0 < ro + n; i0 += ROWS_ILP * T) {
    int rs[ROWS_ILP], re[ROWS_ILP];
    double s[ROWS_ILP];
    int m = 0;
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * T;
      bool ok = i < ro + n;
      rs[k] = ok ? a.rowptr[i] : 0;
      re[k] = ok ? a.rowptr[i + 1] : 0;
      s[k] = 0.0;
      m = max(m, re[k] - rs[k]);
    }
    for (int e = 0; e < m; ++e) {
#pragma unroll
      for (int k = 0; k < ROWS_ILP; ++k) {
        int p = rs[k] + e;
        if (p < re[k]) s[k] += a.val[p] * v[a.col[p]];
      }
    }
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * T;
      if (i < ro + n) {
        y[i] = s[k];
        acc += s[k] * s[k];
      }
    }
  }
  return acc;
}

constexpr int GS_CHUNK = 8;   // basis vectors per pass of the Gram-Schmidt dot products

// h[0..k] = V[0..k]^T w over rows [ro, ro + n), reduced over the CTA into h
// (shared memory); V_c at V + c ld
__device__ void block_dots(const double* V, long long ld, int k1, int ro, int n, const double* w,
                           double* h, double* red8) {
  const int T = blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  for (int c0 = 0; c0 < k1; c0 += GS_CHUNK) {
    double s[GS_CHUNK];
#pragma unroll
    for (int c = 0; c < GS_CHUNK; ++c) s[c] = 0.0;
    for (int i = ro + threadIdx.x; i < ro + n; i += T) {
      double wi = w[i];
#pragma unroll
      for (int c = 0; c < GS_CHUNK; ++c)
        if (c0 + c < k1) s[c] += V[(long long)(c0 + c) * ld + i] * wi;
    }
#pragma unroll
    for (int c = 0; c < GS_CHUNK; ++c) {
      double v = s[c];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red8[warp * GS_CHUNK + c] = v;
    }
    __syncthreads();
    if (threadIdx.x < GS_CHUNK && c0 + threadIdx.x < k1) {
      double v = 0.0;
      for (int q = 0; q < nw; ++q) v += red8[q * GS_CHUNK + threadIdx.x];
      h[c0 + threadIdx.x] = v;
    }
    __syncthreads();
  }
}

// w -= V[0..k] h; returns this thread's sum of w^2
__device__ inline double block_update(const double* V, long long ld, int k1, int ro, int n, double* w,
                                      const double* h) {
  double acc = 0.0;
  for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
    double wi = w[i];
    for (int c = 0; c < k1; ++c) wi -= h[c] * V[(long long)c * ld + i];
    w[i] = wi;
    acc += wi * wi;
  }
  return acc;
}

// GMRES(m) with the two-stage step as right preconditioner (Sec. 4.5, 4.6;
// Saad's right-preconditioned GMRES, Givens rotations).  The Arnoldi vectors
// are orthogonalised by classical Gram-Schmidt applied twice, whose two
// passes over the basis replace the k + 1 dependent reductions of modified
// Gram-Schmidt (same result in exact arithmetic, orthogonality to working
// precision).  Iterations count preconditioner applications; the history
// holds the least-squares residual estimate inside a cycle and the true
// residual at each cycle's end.
__global__ void __launch_bounds__(SOLVE_T, 2) k_gmres(SolveArgs a, double* krylov) {
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ double red8[(SOLVE_T / 32) * GS_CHUNK];
  __shared__ int s_done;
  __shared__ int pbuf[2 * CH_MAX];
  int ii = blockIdx.x;
  const Inst& I = a.inst[ii];
  if (I.krylov != FAMS_KRYLOV_GMRES) return;
  const int n = I.n, ro = I.row_off, m = I.restart;
  const SolveSmem S = solve_smem(sm, I.nc, pbuf);
  // dense arrays after the coarse buffers: H ((m+1) x m, column k at
  // H + k (m+1)), g (m+1), cs, sn, hv (m+1 scratch dot products), y (m)
  double* H = sm + 2 * I.nc + 2 * BAND_BUF;
  double* g = H + (m + 1) * m;
  double* cs = g + (m + 1);
  double* sn = cs + m;
  double* hv = sn + m;
  double* yv = hv + (m + 1);
  double* V = krylov;   // V_k at V + k ntot, rows indexed like every batch vector
  const long long ld = a.ntot;
  const int T = blockDim.x;
  double acc = 0.0;
  for (int i = ro + threadIdx.x; i < ro + n; i += T) acc += a.q[i] * a.q[i];
  double qn = sqrt(block_sum(acc, red));
  if (!(qn > 0.0)) qn = 1.0;
  long long cyc[6] = {0, 0, 0, 0, 0, 0};
  long long t0 = clock64();
  int it = 0;
  acc = rows_residual(a, ro, n, a.q, a.x, a.r, true);
  double beta = sqrt(block_sum(acc, red));
  double rel = beta / qn;
  if (threadIdx.x == 0) a.hist[(long long)ii * a.hist_len] = rel;
  cyc[0] += clock64() - t0;
  for (;;) {
    if (threadIdx.x == 0)
      s_done = (rel <= a.tol || it >= I.max_iter || !isfinite(rel) || a.cs.bad[ii] || !(beta > 0.0));
    __syncthreads();
    if (s_done) break;
    // V_0 = r / beta, g = beta e_1
    t0 = clock64();
    for (int i = ro + threadIdx.x; i < ro + n; i += T) V[i] = a.r[i] / beta;
    for (int k = threadIdx.x; k <= m; k += T) g[k] = k == 0 ? beta : 0.0;
    __syncthreads();
    cyc[0] += clock64() - t0;
    int k = 0;
    for (;;) {
      // z = M^-1 V_k (in r), w = A z (in V_{k+1})
      double* Vk = V + (long long)k * ld;
      double* w = V + (long long)(k + 1) * ld;
      two_stage(a, I, ii, Vk, a.dp, a.r, nullptr, S, cyc);
      t0 = clock64();
      rows_apply(a, ro, n, a.r, w);
      __syncthreads();
      // classical Gram-Schmidt, twice: H(0..k, k) = V^T w, w -= V H(0..k, k)
      double* Hk = H + (long long)k * (m + 1);
      block_dots(V, ld, k + 1, ro, n, w, Hk, red8);
      block_update(V, ld, k + 1, ro, n, w, Hk);
      __syncthreads();
      block_dots(V, ld, k + 1, ro, n, w, hv, red8);
      acc = block_update(V, ld, k + 1, ro, n, w, hv);
      double hn = sqrt(block_sum(acc, red));
      if (threadIdx.x <= k) Hk[threadIdx.x] += hv[threadIdx.x];
      if (hn > 0.0)
        for (int i = ro + threadIdx.x; i < ro + n; i += T) w[i] /= hn;
      __syncthreads();
      // Givens rotations on column k and the right-hand side g
      if (threadIdx.x == 0) {
        Hk[k + 1] = hn;
        for (int i = 0; i < k; ++i) {
          double t = cs[i] * Hk[i] + sn[i] * Hk[i + 1];
          Hk[i + 1] = -sn[i] * Hk[i] + cs[i] * Hk[i + 1];
          Hk[i] = t;
        }
        double d = hypot(Hk[k], Hk[k + 1]);
        cs[k] = Hk[k] / d;
        sn[k] = Hk[k + 1] / d;
        Hk[k] = d;
        Hk[k + 1] = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        double est = fabs(g[k + 1]) / qn;
        a.hist[(long long)ii * a.hist_len + it + 1] = est;
        s_done = (est <= a.tol || k + 1 >= m || it + 1 >= I.max_iter || !isfinite(est));
      }
      __syncthreads();
      cyc[0] += clock64() - t0;
      ++k;
      ++it;
      if (s_done) break;
    }
    // y = H^-1 g (upper triangular k x k), u = V y (in V_k), x += M^-1 u
    t0 = clock64();
    if (threadIdx.x == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k; ++j) s -= H[(long long)j * (m + 1) + i] * yv[j];
        yv[i] = s / H[(long long)i * (m + 1) + i];
      }
    }
    __syncthreads();
    double* u = V + (long long)k * ld;
    for (int i = ro + threadIdx.x; i < ro + n; i += T) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += yv[j] * V[(long long)j * ld + i];
      u[i] = s;
    }
    __syncthreads();
    cyc[0] += clock64() - t0;
    two_stage(a, I, ii, u, a.dp, a.x, a.x, S, cyc);
    t0 = clock64();
    acc = rows_residual(a, ro, n, a.q, a.x, a.r, true);
    beta = sqrt(block_sum(acc, red));
    rel = beta / qn;
    if (threadIdx.x == 0) a.hist[(long long)ii * a.hist_len + it] = rel;
    cyc[0] += clock64() - t0;
  }
  write_stats(a, ii, it, rel, qn, cyc);
}

}  // namespace

int phase_alloc_work(Batch& b) {
  long long n = b.tot_row;
  FAMS_TRY(b.alloc((void**)&b.q, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.x, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.r, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.dp, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.y, sizeof(double) * (n + 1)));
  FAMS_TRY(b.alloc((void**)&b.stat, sizeof(double) * STAT_W * b.B));
  int mi = 0;
  for (auto& I : b.h) mi = std::max(mi, I.max_iter);
  b.hist_len = mi + 1;
  FAMS_TRY(b.alloc((void**)&b.rc, sizeof(double) * (b.tot_nc + 1)));
  FAMS_TRY(b.alloc((void**)&b.ec, sizeof(double) * (b.tot_nc + 1)));
  FAMS_TRY(b.alloc((void**)&b.hist, sizeof(double) * b.hist_len * b.B));
  // GMRES bases: (restart + 1) vectors indexed like the batch rows
  int mr = 0;
  for (auto& I : b.h) mr = std::max(mr, I.restart);
  if (mr > 0)
    FAMS_TRY(b.alloc((void**)&b.krylov, sizeof(double) * (size_t)(mr + 1) * (size_t)(n + 1)));
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
  a.rowptr = b.rowptr; a.col = b.col; a.val = b.val; a.diag = b.diag;
  a.p_ptr = b.p_ptr; a.p_col = b.p_col; a.p_val = b.p_val;
  a.pt_ptr = b.pt_ptr; a.pt_col = b.pt_col; a.pt_val = b.pt_val;
  a.blk_ptr = b.blk_ptr; a.blk_cell = b.blk_cell;
  a.F = b.ilu; a.lev_off = b.lev_off; a.lev_ptr = b.lev_ptr; a.lev_rows = b.lev_rows;
  a.q = b.q; a.x = b.x; a.r = b.r; a.dp = b.dp; a.y = b.y; a.stat = b.stat;
  a.hist = b.hist; a.hist_len = b.hist_len;
  a.crhs = b.rc; a.csol = b.ec;
  a.pk_pos = b.pk_pos; a.pk_nl = b.pk_nl; a.pk_lp = b.pk_lp; a.pk_lc = b.pk_lc; a.pk_lv = b.pk_lv;
  a.pk_nu = b.pk_nu; a.pk_uc = b.pk_uc; a.pk_uv = b.pk_uv; a.pk_ud = b.pk_ud;
  a.ylev = b.ylev;
  a.ntot = b.tot_row;
  a.tol = tol;
  int maxnc = 0;
  for (auto& I : b.h) maxnc = std::max(maxnc, I.nc);
  for (int i = 0; i < b.B; ++i)
    if (b.csh[0].kl[i] + b.csh[0].ku[i] + 1 > BAND_BUF) {
      set_error("coarse band wider than the staged band buffer");
      return FAMS_ECAPACITY;
    }
  size_t smem = sizeof(double) * (2 * (size_t)maxnc + 2 * BAND_BUF);
  int mr = 0, nrich = 0;
  for (auto& I : b.h) {
    mr = std::max(mr, I.restart);
    nrich += I.krylov == FAMS_KRYLOV_NONE;
  }
  size_t smem_g = smem + sizeof(double) * ((size_t)mr * mr + 6 * (size_t)mr + 2);
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  if ((long long)(mr > 0 ? smem_g : smem) + 2048 > max_smem) {
    set_error("coarse system too large for the shared-memory coarse solve");
    return FAMS_ECAPACITY;
  }
  FAMS_CUDA(cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - 2048));
  FAMS_CUDA(cudaFuncSetAttribute(k_gmres, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - 3072));
  cudaEvent_t e0, e1;
  FAMS_CUDA(cudaEventCreate(&e0));
  FAMS_CUDA(cudaEventCreate(&e1));
  FAMS_CUDA(cudaEventRecord(e0, b.stream));
  // each kernel leaves the other kind of instance alone
  if (nrich > 0) {
    fams::note_launch(), k_solve<<<b.B, SOLVE_T, smem, b.stream>>>(a);
    FAMS_CUDA(cudaGetLastError());
  }
  if (mr > 0) {
    fams::note_launch(), k_gmres<<<b.B, SOLVE_T, smem_g, b.stream>>>(a, b.krylov);
    FAMS_CUDA(cudaGetLastError());
  }
  FAMS_CUDA(cudaEventRecord(e1, b.stream));
  FAMS_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  FAMS_CUDA(cudaEventElapsedTime(&t, e0, e1));
  if (ms) *ms = t;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return FAMS_OK;
}

// ---------------------------------------------------------------------------
// The same iteration with its work vectors in a fixed device array, for
// callers that cannot allocate device memory when they solve.  Layout in
// doubles, every part starting on a 256-byte boundary:
//   q, x, r, dp, y, ylev   STATIC_ROWS each
//   crhs, csol             STATIC_COARSE each
//   stat                   STATIC_STAT (STAT_W used)
//   hist                   STATIC_HIST
namespace {
constexpr long long STATIC_ROWS = FAMS_STATIC_MAX_ROWS;
constexpr long long STATIC_COARSE = FAMS_STATIC_MAX_COARSE;
constexpr long long STATIC_STAT = 32;
constexpr long long STATIC_HIST = (long long)FAMS_STATIC_MAX_ITER + 1;
constexpr long long STATIC_DOUBLES = 6 * STATIC_ROWS + 2 * STATIC_COARSE + STATIC_STAT + STATIC_HIST;
static_assert(STATIC_ROWS % 32 == 0 && STATIC_COARSE % 32 == 0 && STATIC_STAT % 32 == 0,
              "parts of the static work array must stay 256-byte aligned");
static_assert(STATIC_STAT >= STAT_W, "status words do not fit");
constexpr int MAX_DEVICES = 64;
}  // namespace

// In host code this name only stands for the device array: its device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_solve_static_work[STATIC_DOUBLES];

namespace {
std::mutex g_static_mu;
double* g_static_ptr[MAX_DEVICES] = {};

// device address of the work array on `dev` (current device); looked up on
// the first call on each device
int static_work(int dev, double** out) {
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device ordinal beyond the static work table");
    return FAMS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_solve_static_work);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress of the static work array: ") +
                cudaGetErrorString(e));
      return FAMS_ECUDA;
    }
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_ptr[dev];
  return FAMS_OK;
}

int solve_static_on_device(Batch& b, const double* rhs, double* x, double tol, fams_stats* st) {
  const Inst& I = b.h[0];
  if (I.n > STATIC_ROWS) {
    set_error("instance has " + std::to_string(I.n) + " unknowns; fams_solve_static holds at most " +
              std::to_string(STATIC_ROWS));
    return FAMS_ECAPACITY;
  }
  if (I.nc > STATIC_COARSE) {
    set_error("instance has " + std::to_string(I.nc) + " coarse unknowns; fams_solve_static holds "
              "at most " + std::to_string(STATIC_COARSE));
    return FAMS_ECAPACITY;
  }
  if ((long long)I.max_iter + 1 > STATIC_HIST) {
    set_error("max_iter " + std::to_string(I.max_iter) + " above fams_solve_static's limit " +
              std::to_string(STATIC_HIST - 1));
    return FAMS_ECAPACITY;
  }
  if (b.csh[0].kl[0] + b.csh[0].ku[0] + 1 > BAND_BUF) {
    set_error("coarse band wider than the staged band buffer");
    return FAMS_ECAPACITY;
  }
  size_t smem = sizeof(double) * (2 * (size_t)I.nc + 2 * BAND_BUF);
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  if ((long long)smem + 2048 > max_smem) {
    set_error("coarse system too large for the shared-memory coarse solve");
    return FAMS_ECAPACITY;
  }
  double* w = nullptr;
  FAMS_TRY(static_work(b.device, &w));
  double* q = w;
  double* xs = w + STATIC_ROWS;
  double* dp = w + 3 * STATIC_ROWS;
  double* stat = w + 6 * STATIC_ROWS + 2 * STATIC_COARSE;

  SolveArgs a;
  a.inst = b.d_inst;
  a.cs = b.cs[0];
  a.rowptr = b.rowptr; a.col = b.col; a.val = b.val; a.diag = b.diag;
  a.p_ptr = b.p_ptr; a.p_col = b.p_col; a.p_val = b.p_val;
  a.pt_ptr = b.pt_ptr; a.pt_col = b.pt_col; a.pt_val = b.pt_val;
  a.blk_ptr = b.blk_ptr; a.blk_cell = b.blk_cell;
  a.F = b.ilu; a.lev_off = b.lev_off; a.lev_ptr = b.lev_ptr; a.lev_rows = b.lev_rows;
  a.q = q; a.x = xs; a.r = w + 2 * STATIC_ROWS; a.dp = dp; a.y = w + 4 * STATIC_ROWS;
  a.ylev = w + 5 * STATIC_ROWS;
  a.crhs = w + 6 * STATIC_ROWS; a.csol = w + 6 * STATIC_ROWS + STATIC_COARSE;
  a.stat = stat;
  a.hist = stat + STATIC_STAT; a.hist_len = STATIC_HIST;
  a.pk_pos = b.pk_pos; a.pk_nl = b.pk_nl; a.pk_lp = b.pk_lp; a.pk_lc = b.pk_lc; a.pk_lv = b.pk_lv;
  a.pk_nu = b.pk_nu; a.pk_uc = b.pk_uc; a.pk_uv = b.pk_uv; a.pk_ud = b.pk_ud;
  a.ntot = b.tot_row;
  a.tol = tol;

  // the array keeps the previous call's values: clear the status words; q,
  // the iterate and the staged rhs are written below, every other vector is
  // written by the kernel before it is read
  FAMS_CUDA(cudaMemsetAsync(stat, 0, sizeof(double) * STATIC_STAT, b.stream));
  if (rhs)
    FAMS_CUDA(cudaMemcpyAsync(dp, rhs, sizeof(double) * I.n, cudaMemcpyDefault, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(xs, x, sizeof(double) * I.n, cudaMemcpyDefault, b.stream));
  fams::note_launch(),
      k_make_q<<<grid_for(I.n, 256), 256, 0, b.stream>>>(I.n, rhs ? dp : nullptr, b.qD, q);
  FAMS_CUDA(cudaGetLastError());
  FAMS_CUDA(cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - 2048));
  auto t0 = std::chrono::steady_clock::now();
  fams::note_launch(), k_solve<<<1, SOLVE_T, smem, b.stream>>>(a);
  FAMS_CUDA(cudaGetLastError());
  double hs[STAT_W];
  FAMS_CUDA(cudaMemcpyAsync(hs, stat, sizeof(double) * STAT_W, cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(x, xs, sizeof(double) * I.n, cudaMemcpyDefault, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) {
    st->iterations = (int)hs[0];
    st->rel_residual = hs[1];
    st->converged = hs[2] > 0.5;
    st->solve_ms = ms;
  }
  if (hs[STAT_BAD] > 0.5) {
    set_error("numerically singular coarse system (zero pivot at LU step " +
              std::to_string(b.csh[0].bad[0] - 1) + ")");
    return FAMS_EBREAKDOWN;
  }
  if (!std::isfinite(hs[1])) {
    set_error("the iteration produced a non-finite residual");
    return FAMS_EBREAKDOWN;
  }
  if (hs[2] < 0.5) {
    set_error("max_iter reached before the tolerance");
    return FAMS_ENOCONV;
  }
  return FAMS_OK;
}
}  // namespace

int solve_static(Batch& b, const double* rhs, double* x, double tol, fams_stats* st) {
  int prev = -1;
  FAMS_CUDA(cudaGetDevice(&prev));
  if (prev != b.device) FAMS_CUDA(cudaSetDevice(b.device));
  int s = solve_static_on_device(b, rhs, x, tol, st);
  if (prev != b.device) cudaSetDevice(prev);
  return s;
}

}  // namespace fams
