// One large instance on the whole GPU: GMRES(m) with the two-stage step of
// Table 1 as right preconditioner (Sec. 3.2, Sec. 4.5-4.6), run by a
// cooperative persistent kernel whose CTAs -- all resident, a few per SM --
// share every step of the iteration.  The one-CTA-per-instance kernels of
// solve.cu keep a single instance on one SM; an instance of a million cells
// (the paper's 3D scale study, Sec. 4.6.3) needs all 152.
//
//  * row-parallel passes (A v, P e_c, r - A dp, the Gram-Schmidt passes,
//    vector updates) stride over every thread of the grid;
//  * R r and e_c = A_c^-1 r_c take one warp per coarse row; A_c^-1 is formed
//    once per coarse system from its band factors (k_coarse_inverse: each CTA
//    solves a group of unit right-hand sides), so the per-iteration coarse
//    solve is a dense matrix-vector product spread over the grid instead of a
//    sequential band substitution on one SM;
//  * the ILU(0) sweeps go level by level with a grid barrier per level;
//  * dot products: a CTA sum, then every CTA adds the CTAs' partial sums in
//    the same fixed order, so all CTAs hold the same value and take the same
//    decisions (Givens rotations, stopping) without further communication.
//
// Grid barriers are a counter and a generation word in global memory; a CTA
// that waits longer than GRID_SPIN polls, or sees another CTA's error flag,
// sets the flag and returns, and every other CTA leaves at its next barrier;
// the host reports FAMS_ETIMEOUT.  The launch is cooperative, so all CTAs are
// resident and the barrier cannot wait on a CTA that never started.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "band_solve.cuh"
#include "batch.cuh"

namespace fams {

namespace {

constexpr int GT = 512;                     // threads per CTA
constexpr long long GRID_SPIN = 1LL << 24;  // polls of a barrier (~2-3 s with the back-off)
constexpr int INV_NR = 8;                   // right-hand sides per CTA pass of the inverse
// The iteration's coarse solve: A_c^-1 formed once (about 2.5 nc^2 kl FMAs
// on every SM, then a product per iteration), or the band factors solved by
// one CTA per iteration (band mode).  Measured on 14k and 16k coarse
// unknowns the one-CTA band solve takes 26-240 ms per iteration (a
// synchronisation per band column), so the inverse stays the automatic
// choice while it fits in GRID_INV_BYTES of device memory.
constexpr long long GRID_INV_BYTES = 8LL << 30;
constexpr int GRID_BAND_BUF = 3072;         // doubles per band chunk (at least kl + ku + 1)

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

struct GArgs {
  int n, nc, ncm, restriction, restart, max_iter, nlev, bad;
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
  const int* lev_ptr;
  const int* lev_rows;
  const int* pk_pos;
  const int* pk_nl;
  const int* pk_lp;
  const int* pk_lc;
  const double* pk_lv;
  const int* pk_nu;
  const int* pk_uc;
  const double* pk_uv;
  const double* pk_ud;
  const double* Fb;      // the sub-block stage's factors (subblock: 1), same layout
  const double* pk_lvb;
  const double* pk_uvb;
  const double* pk_udb;
  int subblock;
  long long ntot;        // stride of the PK arrays
  const double* ainv;    // A_c^-1, nc x nc, row-major, coarse order (null: band mode)
  // band mode: the band LU factors, pivots and band order; CTA 0 solves with
  // them in shared memory (hsm doubles of Hessenberg data, then nc + 2 bb)
  const double* band;
  const int* ipiv;
  const int* perm;
  int kl, ku, bb, hsm;
  const double* q;
  double* x;
  double* r;
  double* dp;
  double* y;
  double* ylev;
  double* rc;
  double* ec;
  double* V;             // (restart + 1) vectors of ntot
  double* stat;
  double* hist;
  long long hist_len;
  double* part;          // 2 x gridDim.x partial sums
  GridBar* bar;          // bar[0]: the grid; bar[1]: the CTAs of the ILU(0) sweeps
  int sweep_ctas;        // CTAs that run the sweeps (enough threads for the widest level)
  double tol;
};

__device__ inline long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ inline long long gthreads() { return (long long)gridDim.x * blockDim.x; }

// loads of vectors written by other CTAs during the kernel: from L2
__device__ inline double ldv(const double* p) { return __ldcg(p); }

// false: the kernel must return (a barrier gave up, here or in another CTA).
// `parties` CTAs take part (the whole grid by default); the error word of
// the grid's barrier (err) is shared by every barrier of the launch
__device__ bool grid_sync(GridBar* bar, unsigned int parties = 0, int* err_word = nullptr) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &bar->gen;
    int* ew = err_word ? err_word : &bar->err;
    volatile int* verr = ew;
    const unsigned int np = parties ? parties : gridDim.x;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&bar->count, 1u) == np - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long polls = 0;
      while (*vgen == g) {
        if (*verr) { ok = 0; break; }
        if (++polls > GRID_SPIN) {
          atomicCAS(ew, 0, DERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(polls < 64 ? 20 : 128);
      }
    }
    __threadfence();
    s_ok = ok && !*verr;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ inline double cta_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
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

// sum of v over the grid, the same value in every CTA (partial sums added in
// CTA order); `buf` alternates between the two halves of part, so a fast CTA
// never overwrites partials another CTA is still adding
__device__ bool grid_sum(const GArgs& a, double v, double* red, int& buf, double* out) {
  double s = cta_sum(v, red);
  double* part = a.part + (long long)buf * gridDim.x;
  buf ^= 1;
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!grid_sync(a.bar)) return false;
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += ldv(part + i);
  *out = cta_sum(t, red);
  return true;
}

__device__ inline double warp_sum(double s) {
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Steps 5-7 of Table 1 on r over the grid:
//   dp = P A_c^-1 R r;  y = r - A dp;  out = (base + dp) + (LU)^-1 y
__device__ bool two_stage_grid(const GArgs& a, const double* r, double* out, const double* base) {
  const long long T = gthreads(), t0 = gtid();
  const long long nw = T >> 5, gw = t0 >> 5;
  const int lane = threadIdx.x & 31;
  // r_c = R r: a warp per coarse row
  for (long long k = gw; k < a.nc; k += nw) {
    double s = 0.0;
    if (a.restriction == FAMS_R_FE || (a.restriction == FAMS_R_MIX && k < a.ncm)) {
      for (int p = a.pt_ptr[k] + lane; p < a.pt_ptr[k + 1]; p += 32) s += a.pt_val[p] * ldv(r + a.pt_col[p]);
    } else {
      for (int p = a.blk_ptr[k] + lane; p < a.blk_ptr[k + 1]; p += 32) s += ldv(r + a.blk_cell[p]);
    }
    s = warp_sum(s);
    if (lane == 0) a.rc[k] = s;
  }
  if (!grid_sync(a.bar)) return false;
  if (a.ainv) {
    // e_c = A_c^-1 r_c: a warp per coarse row of the inverse
    for (long long k = gw; k < a.nc; k += nw) {
      const double* row = a.ainv + k * a.nc;
      double s = 0.0;
      for (int j = lane; j < a.nc; j += 32) s += row[j] * ldv(a.rc + j);
      s = warp_sum(s);
      if (lane == 0) a.ec[k] = s;
    }
  } else if (blockIdx.x == 0) {
    // e_c by the band factors on CTA 0 (the others wait at the barrier): r_c
    // gathered into band order in shared memory, the gbtrs steps, scattered
    // back in coarse order
    extern __shared__ double sm[];
    __shared__ int pbuf[2 * band::CH_MAX];
    double* yb = sm + a.hsm;
    double* bbuf = yb + a.nc;
    for (int k = threadIdx.x; k < a.nc; k += blockDim.x) yb[k] = ldv(a.rc + a.perm[k]);
    __syncthreads();
    band::coarse_solve(a.band, a.ipiv, a.nc, a.kl, a.ku, yb, bbuf, pbuf, a.bb);
    for (int k = threadIdx.x; k < a.nc; k += blockDim.x) a.ec[a.perm[k]] = yb[k];
  }
  if (!grid_sync(a.bar)) return false;
  // dp = P e_c
  for (long long i = t0; i < a.n; i += T) {
    double s = 0.0;
    for (int p = a.p_ptr[i]; p < a.p_ptr[i + 1]; ++p) s += a.p_val[p] * ldv(a.ec + a.p_col[p]);
    a.dp[i] = s;
  }
  if (!grid_sync(a.bar)) return false;
  // y = r - A dp, in natural and level order
  for (long long i = t0; i < a.n; i += T) {
    double s = ldv(r + i);
    for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) s -= a.val[p] * ldv(a.dp + a.col[p]);
    a.y[i] = s;
    a.ylev[a.pk_pos[i]] = s;
  }
  if (!grid_sync(a.bar)) return false;
  // the ILU(0) sweeps on the first sweep_ctas CTAs, level by level with a
  // barrier among them (a level holds at most their threads' rows at once
  // in 3D wavefronts; fewer parties make each barrier cheaper); each thread
  // loads its row of the next level before the barrier.  The other CTAs wait
  // at the grid barrier after the sweeps.
  for (int pass = 0; pass < (a.subblock ? 2 : 1); ++pass) {
  // pass 1, the sub-block smoothing stage: r2 = r - A (dp1 + dp2), swept
  // with the media blocks' factors and added to out
  if (pass == 1) {
    for (long long i = t0; i < a.n; i += T) a.dp[i] = ldv(a.dp + i) + ldv(a.y + i);
    if (!grid_sync(a.bar)) return false;
    for (long long i = t0; i < a.n; i += T) {
      double s = ldv(r + i);
      for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) s -= a.val[p] * ldv(a.dp + a.col[p]);
      a.y[i] = s;
      a.ylev[a.pk_pos[i]] = s;
    }
    if (!grid_sync(a.bar)) return false;
  }
  const double* Fs = pass ? a.Fb : a.F;
  const double* lvs = pass ? a.pk_lvb : a.pk_lv;
  const double* uvs = pass ? a.pk_uvb : a.pk_uv;
  const double* uds = pass ? a.pk_udb : a.pk_ud;
  if ((int)blockIdx.x < a.sweep_ctas) {
    const long long nt = a.ntot;
    const long long ST = (long long)a.sweep_ctas * blockDim.x;
    GridBar* sb = a.bar + 1;
    int* ew = &a.bar->err;
    // L sweep: y_t = r1_t - sum_{j<t} L_tj y_j
    long long t = a.nlev > 0 ? a.lev_ptr[0] + t0 : 0;
    int cnt = 0, p0 = 0, c[PK];
    double yb = 0.0, f[PK];
    auto load_l = [&](int l) {
      t = a.lev_ptr[l] + t0;
      if (t < a.lev_ptr[l + 1]) {
        yb = ldv(a.ylev + t);
        cnt = a.pk_nl[t];
        p0 = a.pk_lp[t];
#pragma unroll
        for (int k = 0; k < PK; ++k) {
          c[k] = a.pk_lc[k * nt + t];
          f[k] = lvs[k * nt + t];
        }
      }
    };
    if (a.nlev > 0) load_l(0);
    for (int l = 0; l < a.nlev; ++l) {
      const long long te = a.lev_ptr[l + 1];
      if (t < te) {
        double s = yb;
#pragma unroll
        for (int k = 0; k < PK; ++k)
          if (k < cnt) s -= f[k] * ldv(a.ylev + c[k]);
        for (int p = p0 + PK; p < p0 + cnt; ++p) s -= Fs[p] * ldv(a.ylev + a.pk_pos[a.col[p]]);
        a.ylev[t] = s;
        for (long long u = t + ST; u < te; u += ST) {   // rows beyond one per thread
          double s2 = ldv(a.ylev + u);
          const int c2 = a.pk_nl[u], q0 = a.pk_lp[u];
          for (int k = 0; k < PK && k < c2; ++k) s2 -= lvs[k * nt + u] * ldv(a.ylev + a.pk_lc[k * nt + u]);
          for (int p = q0 + PK; p < q0 + c2; ++p) s2 -= Fs[p] * ldv(a.ylev + a.pk_pos[a.col[p]]);
          a.ylev[u] = s2;
        }
      }
      if (l + 1 < a.nlev) load_l(l + 1);
      if (!grid_sync(sb, (unsigned)a.sweep_ctas, ew)) return false;
    }
    // U sweep and the update: out = (base + dp) + x_t, x_t = (y_t - sum_{j>t} U_tj x_j) / U_tt
    double ud = 0.0, xo = 0.0, dpo = 0.0;
    int row = 0;
    auto load_u = [&](int l) {
      t = a.lev_ptr[l] + t0;
      if (t < a.lev_ptr[l + 1]) {
        row = a.lev_rows[t];
        yb = ldv(a.ylev + t);
        cnt = a.pk_nu[t];
        ud = uds[t];
        dpo = pass ? 0.0 : ldv(a.dp + row);
        xo = pass ? ldv(out + row) : (base ? ldv(base + row) : 0.0);
#pragma unroll
        for (int k = 0; k < PK; ++k) {
          c[k] = a.pk_uc[k * nt + t];
          f[k] = uvs[k * nt + t];
        }
      }
    };
    if (a.nlev > 0) load_u(a.nlev - 1);
    for (int l = a.nlev - 1; l >= 0; --l) {
      const long long te = a.lev_ptr[l + 1];
      if (t < te) {
        double s = yb;
#pragma unroll
        for (int k = 0; k < PK; ++k)
          if (k < cnt) s -= f[k] * ldv(a.ylev + c[k]);
        if (cnt > PK) {
          const int d = a.diag[row];
          for (int p = d + 1 + PK; p <= d + cnt; ++p) s -= Fs[p] * ldv(a.ylev + a.pk_pos[a.col[p]]);
        }
        const double xi = s * ud;
        a.ylev[t] = xi;
        a.y[row] = xi;
        out[row] = (xo + dpo) + xi;
        for (long long u = t + ST; u < te; u += ST) {   // rows beyond one per thread
          const int i = a.lev_rows[u];
          double s2 = ldv(a.ylev + u);
          const int c2 = a.pk_nu[u];
          for (int k = 0; k < PK && k < c2; ++k) s2 -= uvs[k * nt + u] * ldv(a.ylev + a.pk_uc[k * nt + u]);
          if (c2 > PK) {
            const int d = a.diag[i];
            for (int p = d + 1 + PK; p <= d + c2; ++p) s2 -= Fs[p] * ldv(a.ylev + a.pk_pos[a.col[p]]);
          }
          const double x2 = s2 * uds[u];
          a.ylev[u] = x2;
          a.y[i] = x2;
          out[i] = pass ? ldv(out + i) + x2 : ((base ? ldv(base + i) : 0.0) + ldv(a.dp + i)) + x2;
        }
      }
      if (l > 0) load_u(l - 1);
      if (!grid_sync(sb, (unsigned)a.sweep_ctas, ew)) return false;
    }
  }
  if (!grid_sync(a.bar)) return false;
  }
  return true;
}

// y = b - A v over the grid (b null: y = A v); returns this thread's sum of y^2
__device__ double rows_grid(const GArgs& a, const double* b, const double* v, double* y) {
  const long long T = gthreads();
  double acc = 0.0;
  for (long long i = gtid(); i < a.n; i += T) {
    double s = 0.0;
    for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) s += a.val[p] * ldv(v + a.col[p]);
    s = b ? ldv(b + i) - s : s;
    y[i] = s;
    acc += s * s;
  }
  return acc;
}

__global__ void __launch_bounds__(GT) k_gmres_grid(GArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ int s_done;
  const int m = a.restart;
  double* H = sm;              // (m + 1) x m, column k at H + k (m + 1)
  double* g = H + (m + 1) * m;
  double* cs = g + (m + 1);
  double* sn = cs + m;
  double* yv = sn + m;
  const long long T = gthreads(), t0 = gtid();
  const long long ld = a.ntot;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  int buf = 0;
  double acc = 0.0, qn = 0.0, beta = 0.0;
  for (long long i = t0; i < a.n; i += T) acc += a.q[i] * a.q[i];
  if (!grid_sum(a, acc, red, buf, &qn)) return;
  qn = sqrt(qn);
  if (!(qn > 0.0)) qn = 1.0;
  acc = rows_grid(a, a.q, a.x, a.r);
  if (!grid_sum(a, acc, red, buf, &beta)) return;
  beta = sqrt(beta);
  double rel = beta / qn;
  if (lead) a.hist[0] = rel;
  int it = 0;
  while (!(rel <= a.tol || it >= a.max_iter || !isfinite(rel) || a.bad || !(beta > 0.0))) {
    // one GMRES(m) cycle: V_0 = r / beta, g = beta e_1
    for (long long i = t0; i < a.n; i += T) a.V[i] = ldv(a.r + i) / beta;
    for (int k = threadIdx.x; k <= m; k += blockDim.x) g[k] = k == 0 ? beta : 0.0;
    if (!grid_sync(a.bar)) return;
    int k = 0;
    for (;;) {
      double* Vk = a.V + (long long)k * ld;
      double* w = a.V + (long long)(k + 1) * ld;
      // z = M^-1 V_k (in r), w = A z
      if (!two_stage_grid(a, Vk, a.r, nullptr)) return;
      rows_grid(a, nullptr, a.r, w);
      if (!grid_sync(a.bar)) return;
      // modified Gram-Schmidt, each projection applied in the pass that
      // forms the next dot product (the oracle's order of operations)
      double* Hk = H + (long long)k * (m + 1);
      double hprev = 0.0;
      for (int i = 0; i <= k + 1; ++i) {
        const double* Vp = i > 0 ? a.V + (long long)(i - 1) * ld : nullptr;
        const double* Vi = i <= k ? a.V + (long long)i * ld : nullptr;
        double s = 0.0;
        for (long long rr = t0; rr < a.n; rr += T) {
          double wr = ldv(w + rr);
          if (Vp) {
            wr -= hprev * ldv(Vp + rr);
            w[rr] = wr;
          }
          s += Vi ? ldv(Vi + rr) * wr : wr * wr;
        }
        double h;
        if (!grid_sum(a, s, red, buf, &h)) return;
        if (i <= k) {
          if (threadIdx.x == 0) Hk[i] = h;
          hprev = h;
        } else {
          hprev = sqrt(h);
        }
      }
      const double hn = hprev;
      if (hn > 0.0) {
        const double inv = 1.0 / hn;
        for (long long i = t0; i < a.n; i += T) w[i] = ldv(w + i) * inv;
      }
      // Givens rotations, the same in every CTA
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
        if (blockIdx.x == 0) a.hist[it + 1] = est;
        s_done = (est <= a.tol || k + 1 >= m || it + 1 >= a.max_iter || !isfinite(est));
      }
      if (!grid_sync(a.bar)) return;   // w complete before the next step reads it
      ++k;
      ++it;
      if (s_done) break;
    }
    // y = H^-1 g, then u = V y (in V_k) and x += M^-1 u
    if (threadIdx.x == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k; ++j) s -= H[(long long)j * (m + 1) + i] * yv[j];
        yv[i] = s / H[(long long)i * (m + 1) + i];
      }
    }
    __syncthreads();
    double* u = a.V + (long long)k * ld;
    for (long long i = t0; i < a.n; i += T) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += yv[j] * ldv(a.V + (long long)j * ld + i);
      u[i] = s;
    }
    if (!grid_sync(a.bar)) return;
    if (!two_stage_grid(a, u, a.x, a.x)) return;
    acc = rows_grid(a, a.q, a.x, a.r);
    if (!grid_sum(a, acc, red, buf, &beta)) return;
    beta = sqrt(beta);
    rel = beta / qn;
    if (lead) a.hist[it] = rel;
  }
  if (lead) {
    a.stat[0] = it;
    a.stat[1] = rel;
    a.stat[2] = (rel <= a.tol) ? 1.0 : 0.0;
    a.stat[3] = qn;
    for (int k = 0; k < 6; ++k) a.stat[4 + k] = 0.0;
    a.stat[STAT_BAD] = a.bad ? 1.0 : 0.0;
  }
}

// A_c^-1 from the band factors (LAPACK gbtrs steps: row interchanges and unit
// L, then U with kl + ku superdiagonals, in band order), INV_NR unit
// right-hand sides per CTA pass: column j of the inverse (coarse order) is
// the solve for e_j, written to row-major ainv[I nc + j].  work: INV_NR x nc
// doubles per CTA.
__global__ void __launch_bounds__(GT) k_coarse_inverse(const double* AB, const int* ipiv,
                                                     const int* perm, int n, int kl, int ku,
                                                     double* work, double* ainv) {
  const int kv = kl + ku, ldab = 2 * kl + ku + 1;
  double* Y = work + (long long)blockIdx.x * INV_NR * n;   // Y[c n + i]
  for (int j0 = blockIdx.x * INV_NR; j0 < n; j0 += gridDim.x * INV_NR) {
    const int nr = min(INV_NR, n - j0);
    // e_{j0 + c} in band order: band position k holds coarse unknown perm[k]
    for (long long e = threadIdx.x; e < (long long)INV_NR * n; e += blockDim.x) {
      const int c = (int)(e / n), k = (int)(e - (long long)c * n);
      Y[e] = (c < nr && perm[k] == j0 + c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      const int km = min(kl, n - 1 - j), pj = ipiv[j];
      if (pj != j && threadIdx.x < nr) {
        double t = Y[threadIdx.x * n + j];
        Y[threadIdx.x * n + j] = Y[threadIdx.x * n + pj];
        Y[threadIdx.x * n + pj] = t;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < km * nr; e += blockDim.x) {
        const int c = e / km, t = e - c * km + 1;
        Y[c * n + j + t] -= AB[(long long)(kv + t) + (long long)ldab * j] * Y[c * n + j];
      }
      __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
      const double* colj = AB + (long long)ldab * j;
      if (threadIdx.x < nr) Y[threadIdx.x * n + j] /= colj[kv];
      __syncthreads();
      const int i0 = max(0, j - kv), cnt = j - i0;
      for (int e = threadIdx.x; e < cnt * nr; e += blockDim.x) {
        const int c = e / cnt, i = i0 + (e - c * cnt);
        Y[c * n + i] -= colj[kv + i - j] * Y[c * n + j];
      }
      __syncthreads();
    }
    for (long long e = threadIdx.x; e < (long long)nr * n; e += blockDim.x) {
      const int c = (int)(e / n), k = (int)(e - (long long)c * n);
      ainv[(long long)perm[k] * n + j0 + c] = Y[e];
    }
    __syncthreads();
  }
}

// IKJ ILU(0) of one instance on the whole GPU, level by level (rows of a
// level are independent), a grid barrier per level.  Factor values of rows of
// earlier levels, written by other CTAs, are read from L2.
__global__ void __launch_bounds__(GT) k_ilu_factor_grid(const int* rowptr, const int* col,
                                                      const int* diag, const int* lev_ptr,
                                                      const int* rows, int nlev, double* F,
                                                      GridBar* bar) {
  const long long T = gthreads(), t0 = gtid();
  int bad = 0;
  for (int l = 0; l < nlev; ++l) {
    for (long long t = lev_ptr[l] + t0; t < lev_ptr[l + 1]; t += T) {
      const int i = rows[t];
      const int e = rowptr[i + 1], d = diag[i];
      for (int p = rowptr[i]; p < d; ++p) {
        const int k = col[p];
        const double lik = F[p] / ldv(F + diag[k]);
        F[p] = lik;
        int u = p + 1;
        for (int q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
          const int j = col[q];
          while (u < e && col[u] < j) ++u;
          if (u < e && col[u] == j) F[u] -= lik * ldv(F + q);
        }
      }
      const double piv = F[d];
      if (!(piv != 0.0) || !isfinite(piv)) bad = 1;
    }
    if (!grid_sync(bar)) return;
  }
  if (bad) atomicCAS(&bar->err, 0, DERR_BREAKDOWN);
}

// Band LU with partial pivoting (LAPACK gbtf2 steps) of one coarse system on
// the whole GPU, in place in the band storage (ldab = 2 kl + ku + 1, the fill
// rows zero on entry).  Step j: the owner of column j picks its pivot (largest
// magnitude, lowest row on ties), applies the scaled singularity test of the
// one-CTA factorisations (pivot at most SING_EPS times the largest entry of
// its row as assembled; row scales follow the interchanges), stores the pivot
// row and the multipliers (column j of L) and publishes the multipliers; each
// CTA then interchanges and updates its own columns (column c belongs to CTA
// c mod gridDim) among j + 1 .. j + kl + ku, and the owner of column j + 1
// chooses step j + 1's pivot as soon as that column is updated, so a step
// ends with one grid barrier.  ctl[1]: 1 + the step of a singular pivot (0:
// none); ctl[2 + (j & 1)]: pivot offset of step j.
__global__ void __launch_bounds__(GT) k_band_lu_grid(double* AB, int* ipiv, int n, int kl, int ku,
                                                   double* sc, double* mult, int* ctl,
                                                   GridBar* bar) {
  const int kv = kl + ku, ldab = 2 * kl + ku + 1;
  const long long T = gthreads(), t0 = gtid();
  const int G = (int)gridDim.x;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p;
  __shared__ double s_piv;
#define BEL(i, c) AB[(long long)(kv + (i) - (c)) + (long long)ldab * (c)]
  // row scales of the matrix as assembled
  for (long long i = t0; i < n; i += T) {
    double m = 0.0;
    for (int c = (int)max(0LL, i - kl); c <= (int)min((long long)n - 1, i + ku); ++c)
      m = fmax(m, fabs(BEL(i, c)));
    sc[i] = m;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // Step j's pivot, by the CTA that owns column j (c mod G = blockIdx): the
  // largest entry of the column below the diagonal, the row interchange of
  // the scales, the multipliers (into the half of `mult` for j's parity)
  // and the interchange for the other CTAs (ctl[2 + parity]); a numerically
  // singular column sets ctl[1] = 1 + j.
  auto pivot = [&](int j) {
    const int km = min(kl, n - 1 - j);
    double best = -1.0;
    int bi = 0;
    for (int t = threadIdx.x; t <= km; t += blockDim.x) {
      const double v = fabs(ldv(&BEL(j + t, j)));
      if (v > best) { best = v; bi = t; }
    }
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[w] = best; si[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b0 = -1.0;
      int i0 = 0;
      for (int q = 0; q < nw; ++q)
        if (sv[q] > b0 || (sv[q] == b0 && si[q] < i0)) { b0 = sv[q]; i0 = si[q]; }
      const double p0 = ldv(&BEL(j + i0, j));
      if (!(b0 > 0.0) || !isfinite(b0) || !(fabs(p0) > SING_EPS * ldv(sc + j + i0))) {
        ctl[1] = 1 + j;
      } else {
        ipiv[j] = j + i0;
        const double t = ldv(sc + j);
        sc[j] = ldv(sc + j + i0);
        sc[j + i0] = t;
      }
      ctl[2 + (j & 1)] = i0;
      s_p = i0;
      s_piv = p0;
    }
    __syncthreads();
    const int p = s_p;
    const double inv = 1.0 / s_piv;
    double* mj = mult + (long long)(j & 1) * (kl + 2);
    // multipliers of the interchanged column j: row j + p holds the old row j
    const double ajj = ldv(&BEL(j, j));
    for (int t = 1 + threadIdx.x; t <= km; t += blockDim.x) {
      const double v = (t == p ? ajj : ldv(&BEL(j + t, j))) * inv;
      mj[t] = v;
    }
    __syncthreads();
    for (int t = 1 + threadIdx.x; t <= km; t += blockDim.x) BEL(j + t, j) = mj[t];
    if (threadIdx.x == 0) BEL(j, j) = s_piv;
  };
  if (!grid_sync(bar)) return;
  if (n > 0 && blockIdx.x == 0) pivot(0);
  if (!grid_sync(bar)) return;
  for (int j = 0; j < n; ++j) {
    if (*(volatile int*)(ctl + 1)) return;
    const int km = min(kl, n - 1 - j);
    const int p = *(volatile int*)(ctl + 2 + (j & 1));
    const double* mj = mult + (long long)(j & 1) * (kl + 2);
    // interchange and update the columns (j, j + kl + ku] this CTA owns (c mod
    // G = blockIdx), a warp per column; the owner's first column is j + 1
    const int cend = min(n - 1, j + kv);
    const int c0 = j + 1 + (((int)blockIdx.x - (j + 1) % G) % G + G) % G;
    int idx = 0;
    for (int c = c0; c <= cend; c += G, ++idx) {
      if (idx % nw != w) continue;
      if (p != 0) {
        if (lane == 0) {
          const double a0 = BEL(j, c), ap = BEL(j + p, c);
          BEL(j, c) = ap;
          BEL(j + p, c) = a0;
        }
        __syncwarp();
      }
      const double ujc = BEL(j, c);
      if (ujc != 0.0)
        for (int t = 1 + lane; t <= km; t += 32) BEL(j + t, c) -= ldv(mj + t) * ujc;
      __syncwarp();
    }
    // look-ahead: the owner of column j + 1, whose warp 0 has just updated
    // it, chooses step j + 1's pivot before the barrier (one grid barrier
    // per step; the search overlaps the other CTAs' updates)
    if (j + 1 < n && (int)blockIdx.x == (j + 1) % G) {
      __syncthreads();
      pivot(j + 1);
    }
    if (!grid_sync(bar)) return;
  }
#undef BEL
}

int grid_blocks(Batch& b, const void* kernel, size_t smem, int* out) {
  int per_sm = 0, sms = 0, coop = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b.device));
  if (!coop) {
    set_error("the device does not support cooperative launches");
    return FAMS_ECUDA;
  }
  FAMS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  FAMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, GT, smem));
  if (per_sm < 1) {
    set_error("the whole-GPU solve kernel does not fit on an SM");
    return FAMS_ECAPACITY;
  }
  *out = sms * std::min(per_sm, 2);
  return FAMS_OK;
}

// A_c^-1 of the iteration's coarse system (built on first use, and again
// after any change of the coarse system)
int coarse_inverse(Batch& b) {
  if (b.ainv_ready) return FAMS_OK;
  const Inst& I = b.h[0];
  const long long nc = I.nc;
  if (!b.ainv) FAMS_TRY(b.alloc((void**)&b.ainv, sizeof(double) * (nc * nc + 1)));
  int sms = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  const int nb = (int)std::min<long long>(2LL * sms, (nc + INV_NR - 1) / INV_NR);
  double* work = nullptr;
  FAMS_TRY(b.scratch((void**)&work, sizeof(double) * ((long long)nb * INV_NR * nc + 1)));
  const CoarseSys& cs = b.cs[0];
  fams::note_launch(), k_coarse_inverse<<<std::max(nb, 1), GT, 0, b.stream>>>(
      cs.band + b.csh[0].band_off[0], cs.ipiv, cs.perm, (int)nc, b.csh[0].kl[0], b.csh[0].ku[0],
      work, b.ainv);
  FAMS_CUDA(cudaGetLastError());
  b.ainv_ready = true;
  return FAMS_OK;
}

}  // namespace

bool whole_gpu(const Batch& b) {
  if (b.B != 1) return false;
  const Inst& I = b.h[0];
  if (I.grid_solve < 0) return false;
  return I.grid_solve > 0 || (long long)I.n >= GRID_SOLVE_ROWS;
}

bool solve_on_grid(const Batch& b) {
  return whole_gpu(b) && b.h[0].krylov == FAMS_KRYLOV_GMRES && b.h[0].precision == FAMS_FP64;
}

namespace {
int grid_bar(Batch& b, int nblk) {
  if (!b.gbar) FAMS_TRY(b.alloc((void**)&b.gbar, 2 * sizeof(GridBar)));
  if (b.gpart_n < nblk) {
    b.release(b.gpart);
    FAMS_TRY(b.alloc((void**)&b.gpart, sizeof(double) * (2 * (size_t)nblk + 16)));
    b.gpart_n = nblk;
  }
  FAMS_CUDA(cudaMemsetAsync(b.gbar, 0, 2 * sizeof(GridBar), b.stream));
  return FAMS_OK;
}

int bar_status(Batch& b, const char* what) {
  GridBar hb{};
  FAMS_CUDA(cudaMemcpyAsync(&hb, b.gbar, sizeof(GridBar), cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  if (hb.err == DERR_TIMEOUT) {
    set_error(std::string(what) + ": a grid barrier gave up (bounded wait)");
    return FAMS_ETIMEOUT;
  }
  if (hb.err == DERR_BREAKDOWN) {
    set_error(std::string(what) + ": zero or non-finite pivot");
    return FAMS_EBREAKDOWN;
  }
  return FAMS_OK;
}
}  // namespace

int ilu_factor_grid(Batch& b, double* F) {
  const Inst& I = b.h[0];
  int nblk = 0;
  FAMS_TRY(grid_blocks(b, (const void*)k_ilu_factor_grid, 0, &nblk));
  FAMS_TRY(grid_bar(b, nblk));
  const int* rowptr = b.rowptr;
  const int* col = b.col;
  const int* diag = b.diag;
  const int* lev_ptr = b.lev_ptr;
  const int* rows = b.lev_rows;
  int nlev = I.nlev;
  GridBar* bar = static_cast<GridBar*>(b.gbar);
  void* params[] = {&rowptr, &col, &diag, &lev_ptr, &rows, &nlev, &F, &bar};
  fams::note_launch();
  FAMS_CUDA(cudaLaunchCooperativeKernel((const void*)k_ilu_factor_grid, dim3(nblk), dim3(GT),
                                        params, 0, b.stream));
  return bar_status(b, "ILU(0)");
}

int band_lu_grid(Batch& b, CoarseSys& cs, CoarseHost& ch) {
  const int n = b.h[0].nc, kl = ch.kl[0], ku = ch.ku[0];
  int nblk = 0;
  FAMS_TRY(grid_blocks(b, (const void*)k_band_lu_grid, 0, &nblk));
  FAMS_TRY(grid_bar(b, nblk));
  double *sc = nullptr, *mult = nullptr;
  int* ctl = nullptr;
  FAMS_TRY(b.scratch((void**)&sc, sizeof(double) * (n + 1)));
  FAMS_TRY(b.scratch((void**)&mult, sizeof(double) * 2 * (kl + 2)));
  FAMS_TRY(b.scratch((void**)&ctl, sizeof(int) * 4));
  FAMS_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * 4, b.stream));
  double* AB = cs.band + ch.band_off[0];
  int* ipiv = cs.ipiv;
  GridBar* bar = static_cast<GridBar*>(b.gbar);
  int nn = n, kkl = kl, kku = ku;
  void* params[] = {&AB, &ipiv, &nn, &kkl, &kku, &sc, &mult, &ctl, &bar};
  fams::note_launch();
  FAMS_CUDA(cudaLaunchCooperativeKernel((const void*)k_band_lu_grid, dim3(nblk), dim3(GT), params,
                                        0, b.stream));
  FAMS_TRY(bar_status(b, "coarse LU"));
  int hc[2] = {0, 0};
  FAMS_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  FAMS_CUDA(cudaMemcpyAsync(cs.bad, &hc[1], sizeof(int), cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemsetAsync(cs.nopiv, 0, sizeof(int), b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  ch.bad.assign(1, hc[1]);
  return FAMS_OK;
}

int run_solve_grid(Batch& b, double tol, float* ms) {
  const Inst& I = b.h[0];
  if (b.csh[0].bad[0]) {
    // a numerically singular coarse system: no iteration, as in the
    // one-CTA kernels (their stat reports it)
    double st[STAT_W] = {0};
    st[STAT_BAD] = 1.0;
    FAMS_CUDA(cudaMemcpyAsync(b.stat, st, sizeof(st), cudaMemcpyHostToDevice, b.stream));
    FAMS_CUDA(cudaStreamSynchronize(b.stream));
    if (ms) *ms = 0.f;
    return FAMS_OK;
  }
  const int m = I.restart;
  const size_t hsm = (size_t)(m + 1) * m + 4 * (size_t)m + 2;
  size_t smem = sizeof(double) * hsm;
  // large coarse systems: band mode when CTA 0 holds the right-hand side and
  // two band chunks in shared memory; otherwise A_c^-1
  const int kl = b.csh[0].kl[0], ku = b.csh[0].ku[0];
  const int bb = std::max(GRID_BAND_BUF, kl + ku + 1);
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  const size_t smem_band = sizeof(double) * (hsm + (size_t)I.nc + 2 * (size_t)bb);
  const bool fits = (long long)smem_band + 2048 <= max_smem;
  const bool big = (long long)I.nc * I.nc * (long long)sizeof(double) > GRID_INV_BYTES;
  const bool band_mode = fits && (I.coarse_mode == 2 || (I.coarse_mode == 0 && big));
  if (band_mode) {
    smem = smem_band;
    FAMS_CUDA(cudaFuncSetAttribute(k_gmres_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  } else {
    FAMS_TRY(coarse_inverse(b));
  }
  int nblk = 0;
  FAMS_TRY(grid_blocks(b, (const void*)k_gmres_grid, smem, &nblk));
  FAMS_TRY(grid_bar(b, nblk));
  GArgs a{};
  a.n = I.n; a.nc = I.nc; a.ncm = I.ncm; a.restriction = I.restriction; a.restart = m;
  a.max_iter = I.max_iter; a.nlev = I.nlev; a.bad = 0;
  a.rowptr = b.rowptr; a.col = b.col; a.val = b.val; a.diag = b.diag;
  a.p_ptr = b.p_ptr; a.p_col = b.p_col; a.p_val = b.p_val;
  a.pt_ptr = b.pt_ptr; a.pt_col = b.pt_col; a.pt_val = b.pt_val;
  a.blk_ptr = b.blk_ptr; a.blk_cell = b.blk_cell;
  a.F = b.ilu; a.lev_ptr = b.lev_ptr; a.lev_rows = b.lev_rows;
  a.pk_pos = b.pk_pos; a.pk_nl = b.pk_nl; a.pk_lp = b.pk_lp; a.pk_lc = b.pk_lc; a.pk_lv = b.pk_lv;
  a.pk_nu = b.pk_nu; a.pk_uc = b.pk_uc; a.pk_uv = b.pk_uv; a.pk_ud = b.pk_ud;
  a.Fb = b.ilu_b; a.pk_lvb = b.pk_lv_b; a.pk_uvb = b.pk_uv_b; a.pk_udb = b.pk_ud_b;
  a.subblock = I.subblock;
  a.ntot = b.tot_row;
  a.ainv = band_mode ? nullptr : b.ainv;
  a.band = b.cs[0].band + b.csh[0].band_off[0];
  a.ipiv = b.cs[0].ipiv;
  a.perm = b.cs[0].perm;
  a.kl = kl; a.ku = ku; a.bb = bb; a.hsm = (int)hsm;
  a.q = b.q; a.x = b.x; a.r = b.r; a.dp = b.dp; a.y = b.y; a.ylev = b.ylev;
  a.rc = b.rc; a.ec = b.ec; a.V = b.krylov;
  a.stat = b.stat; a.hist = b.hist; a.hist_len = b.hist_len;
  a.part = static_cast<double*>(b.gpart);
  a.bar = static_cast<GridBar*>(b.gbar);
  a.tol = tol;
  // CTAs of the sweeps: enough threads for the widest level at one row each
  {
    std::vector<int> lp(I.nlev + 1);
    FAMS_CUDA(cudaMemcpyAsync(lp.data(), b.lev_ptr, sizeof(int) * (I.nlev + 1),
                              cudaMemcpyDeviceToHost, b.stream));
    FAMS_CUDA(cudaStreamSynchronize(b.stream));
    int widest = 1;
    for (int l = 0; l < I.nlev; ++l) widest = std::max(widest, lp[l + 1] - lp[l]);
    a.sweep_ctas = std::max(1, std::min(nblk, (widest + GT - 1) / GT));
  }
  cudaEvent_t e0, e1;
  FAMS_CUDA(cudaEventCreate(&e0));
  FAMS_CUDA(cudaEventCreate(&e1));
  FAMS_CUDA(cudaEventRecord(e0, b.stream));
  void* params[] = {&a};
  fams::note_launch();
  FAMS_CUDA(cudaLaunchCooperativeKernel((const void*)k_gmres_grid, dim3(nblk), dim3(GT), params,
                                        smem, b.stream));
  FAMS_CUDA(cudaEventRecord(e1, b.stream));
  FAMS_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  FAMS_CUDA(cudaEventElapsedTime(&t, e0, e1));
  if (ms) *ms = t;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return bar_status(b, "whole-GPU solve");
}

}  // namespace fams
