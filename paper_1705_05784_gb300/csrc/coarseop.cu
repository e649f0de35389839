// Restriction and coarse system (Sec. 3.2): A_c = R A P with R^FV (the
// indicator of the primal blocks) or R^FE = P^T, factorised by LU with
// partial pivoting (the paper solves the coarse system with a direct LU).
//
// A_c is assembled densely per instance, reordered by reverse Cuthill-McKee
// (one thread per instance) and stored as a band matrix; the band LU
// (partial pivoting inside the band, the LAPACK gbtf2 scheme) runs in one CTA
// per instance.  Any row permutation and pivot order gives the same solution
// up to rounding.
#include <algorithm>

#include "batch.cuh"

namespace fams {

namespace {

__device__ inline int row_of_nnz(const int* rowptr, int lo, int hi, long long p) {
  // rowptr[lo] <= p < rowptr[hi]
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (rowptr[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_rap(const Inst* inst, int B, const int* off_row, long long nnz_tot,
                      const int* rowptr, const int* col, const double* val, long long nrow,
                      const int* primal, const int* p_ptr, const int* p_col, const double* p_val,
                      CoarseSys cs, int mode) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz_tot) return;
  int i = row_of_nnz(rowptr, 0, (int)nrow - 1, p);
  int ii = find_segment(off_row, B + 1, i);
  const Inst& I = inst[ii];
  int fe = mode < 0 ? (I.restriction == FAMS_R_FE) : mode;
  int j = col[p];
  double a = val[p];
  double* Ac = cs.Ac + cs.ac_off[ii];
  int nc = I.nc;
  if (mode < 0 && I.restriction == FAMS_R_MIX) {
    // MSMIX: the fracture coarse rows as R^FV, the matrix coarse rows as R^FE
    int Ib = primal[i];
    if (Ib >= I.ncm)
      for (int q = p_ptr[j]; q < p_ptr[j + 1]; ++q)
        atomicAdd(&Ac[(long long)Ib * nc + p_col[q]], a * p_val[q]);
    for (int t = p_ptr[i]; t < p_ptr[i + 1]; ++t) {
      int Ie = p_col[t];
      if (Ie >= I.ncm) continue;
      double u = p_val[t] * a;
      for (int q = p_ptr[j]; q < p_ptr[j + 1]; ++q)
        atomicAdd(&Ac[(long long)Ie * nc + p_col[q]], u * p_val[q]);
    }
    return;
  }
  if (!fe) {
    int Ib = primal[i];
    for (int q = p_ptr[j]; q < p_ptr[j + 1]; ++q)
      atomicAdd(&Ac[(long long)Ib * nc + p_col[q]], a * p_val[q]);
  } else {
    for (int t = p_ptr[i]; t < p_ptr[i + 1]; ++t) {
      int Ib = p_col[t];
      double u = p_val[t] * a;
      for (int q = p_ptr[j]; q < p_ptr[j + 1]; ++q)
        atomicAdd(&Ac[(long long)Ib * nc + p_col[q]], u * p_val[q]);
    }
  }
}

// nonzero pattern of each dense coarse row (warp per row)
__global__ void k_ac_count(const Inst* inst, int B, const int* off_nc, long long nct, CoarseSys cs,
                           int* cnt) {
  long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= nct) return;
  int ii = find_segment(off_nc, B + 1, w);
  const Inst& I = inst[ii];
  int r = (int)(w - I.nc_off);
  const double* row = cs.Ac + cs.ac_off[ii] + (long long)r * I.nc;
  int c = 0;
  for (int j = lane; j < I.nc; j += 32) c += (row[j] != 0.0 && j != r);
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[w] = c;
}

__global__ void k_ac_cols(const Inst* inst, int B, const int* off_nc, long long nct, CoarseSys cs,
                          const int* ptr, int* cols) {
  long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nct) return;
  int ii = find_segment(off_nc, B + 1, w);
  const Inst& I = inst[ii];
  int r = (int)(w - I.nc_off);
  const double* row = cs.Ac + cs.ac_off[ii] + (long long)r * I.nc;
  int o = ptr[w];
  for (int j = 0; j < I.nc; ++j)
    if (row[j] != 0.0 && j != r) cols[o++] = j;
}

// reverse Cuthill-McKee per instance, one warp each: BFS from a node of
// minimum degree (lowest index on ties), each node's unvisited neighbours
// appended in order of (degree, index), components in turn, then reversed.
// The warp gathers a node's new neighbours with a ballot and orders them with
// a bitonic sort in shared memory.
constexpr int RCM_DEG_MAX = 2048;   // neighbours of one coarse node

__global__ void k_rcm(const Inst* inst, int B, const int* ptr, const int* cols, CoarseSys cs,
                      int* visited, int* queue, int* err) {
  __shared__ long long key[RCM_DEG_MAX];
  int ii = blockIdx.x;
  if (ii >= B) return;
  const int lane = threadIdx.x;
  const Inst& I = inst[ii];
  const int n = I.nc, o = I.nc_off;
  const int* rp = ptr + o;
  int* vis = visited + o;
  int* qu = queue + o;
  int* perm = cs.perm + o;
  for (int i = lane; i < n; i += 32) vis[i] = 0;
  __syncwarp();
  int head = 0, tail = 0;
  while (tail < n) {
    // unvisited node of minimum (degree, index)
    long long best = 0x7fffffffffffffffLL;
    for (int i = lane; i < n; i += 32)
      if (!vis[i]) best = min(best, ((long long)(rp[i + 1] - rp[i]) << 32) | i);
    for (int s = 16; s; s >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, s));
    int start = (int)(best & 0xffffffff);
    if (lane == 0) {
      vis[start] = 1;
      qu[tail] = start;
    }
    ++tail;
    __syncwarp();
    while (head < tail) {
      int u = qu[head++];
      int cnt = 0;
      for (int p0 = rp[u]; p0 < rp[u + 1]; p0 += 32) {
        int p = p0 + lane;
        int v = p < rp[u + 1] ? cols[p] : -1;
        bool fresh = v >= 0 && !vis[v];
        unsigned m = __ballot_sync(0xffffffffu, fresh);
        if (fresh) {
          int at = cnt + __popc(m & ((1u << lane) - 1));
          if (at < RCM_DEG_MAX) key[at] = ((long long)(rp[v + 1] - rp[v]) << 32) | v;
          vis[v] = 1;
        }
        cnt += __popc(m);
      }
      if (cnt > RCM_DEG_MAX) {
        if (lane == 0) atomicCAS(err, 0, DERR_CAPACITY);
        return;
      }
      __syncwarp();
      int m = 1;
      while (m < cnt) m <<= 1;
      for (int i = cnt + lane; i < m; i += 32) key[i] = 0x7fffffffffffffffLL;
      __syncwarp();
      for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < m; i += 32) {
            int l = i ^ j;
            if (l > i) {
              bool up = (i & k) == 0;
              if ((key[i] > key[l]) == up) { long long t = key[i]; key[i] = key[l]; key[l] = t; }
            }
          }
          __syncwarp();
        }
      for (int i = lane; i < cnt; i += 32) qu[tail + i] = (int)(key[i] & 0xffffffff);
      tail += cnt;
      __syncwarp();
    }
  }
  for (int k = lane; k < n; k += 32) perm[k] = qu[n - 1 - k];
}

// lower / upper bandwidth of each instance's dense A_c under the ordering, from
// the same entries the band fill stores (thread per coarse row)
__global__ void k_bandwidth(const Inst* inst, int B, const int* off_nc, long long nct,
                            CoarseSys cs, const int* ip_all, int* kl_out, int* ku_out) {
  long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nct) return;
  int ii = find_segment(off_nc, B + 1, w);
  const Inst& I = inst[ii];
  int r = (int)(w - I.nc_off);
  const double* row = cs.Ac + cs.ac_off[ii] + (long long)r * I.nc;
  const int* ip = ip_all + I.nc_off;
  int kl = 0, ku = 0, i = ip[r];
  for (int c = 0; c < I.nc; ++c) {
    if (row[c] == 0.0) continue;
    int d = i - ip[c];
    kl = max(kl, d);
    ku = max(ku, -d);
  }
  atomicMax(&kl_out[ii], kl);
  atomicMax(&ku_out[ii], ku);
}

// only (nullable): instances to fill
__global__ void k_band_fill(const Inst* inst, int B, const int* off_nc, long long nct,
                            CoarseSys cs, const int* ip_all, const int* only) {
  long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nct) return;
  int ii = find_segment(off_nc, B + 1, w);
  if (only && !only[ii]) return;
  const Inst& I = inst[ii];
  int r = (int)(w - I.nc_off);
  int kl = cs.kl[ii], ku = cs.ku[ii], ldab = 2 * kl + ku + 1;
  const double* row = cs.Ac + cs.ac_off[ii] + (long long)r * I.nc;
  double* AB = cs.band + cs.band_off[ii];
  const int* ip = ip_all + I.nc_off;
  int i = ip[r];
  for (int c = 0; c < I.nc; ++c) {
    double v = row[c];
    if (v == 0.0 && c != r) continue;
    int j = ip[c];
    AB[(long long)(kl + ku + i - j) + (long long)ldab * j] = v;
  }
}

__global__ void k_inverse_perm(const Inst* inst, int B, const int* off_nc, long long nct,
                               CoarseSys cs, int* ip_all) {
  long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nct) return;
  int ii = find_segment(off_nc, B + 1, w);
  const Inst& I = inst[ii];
  int k = (int)(w - I.nc_off);
  ip_all[I.nc_off + cs.perm[w]] = k;
}

__device__ inline int wrap(int x, int k) { return x >= k ? x - k : x; }

// values of the row (and column) entering a factorisation ring that each
// thread loads one step ahead
constexpr int LU_PF = 4;

constexpr int LDL_T = 512;       // threads of the band LDL^T (ring in shared memory)
constexpr int LU_SMEM_T = 256;   // threads of the band LU with its ring in shared memory

constexpr int LU_EXTRA = 32;      // narrow LU ring: columns of fill past the upper band
constexpr double LU_TAU = 0.1;    // narrow LU ring: threshold of the pivot choice
// a pivot at most this fraction of the largest entry of its row (as assembled)
// is numerically zero: the rounding the elimination leaves in that row, a few
// eps times its scale, is then within three decimal digits of the pivot

// Symmetric positive definite coarse systems (R^FE = P^T: A_c = P^T A P):
// band LDL^T without pivoting, about a quarter of the band LU's work.  The
// active lower triangle (rows and columns j..j+kl) lives in a shared-memory
// ring of K = kl + 1 rows and columns, element (i, c) at slot
// (i mod K, c mod K).  The factors are written in the band LU's layout, so
// the solves need no second code path: unit lower multipliers
// L'(i,j) = S(i,j) / d_j, upper row U(j,c) = S(c,j) (= d_j L'(c,j)), pivot
// rows ipiv[j] = j.  A non-positive or non-finite pivot sets failed[ii]; the
// host then refactors that instance with the band LU.  A ring too large for
// shared memory lives in a global slice (gws + gslot[ii] gstride; the
// column below the pivot stays in shared memory).
__global__ void __launch_bounds__(1024) k_band_ldl(const Inst* inst, int B, CoarseSys cs, const int* only, int* failed,
                           double* gws, const int* gslot, long long gstride) {
  extern __shared__ double dyn[];
  int ii = blockIdx.x;
  if (!only[ii]) return;
  const Inst& I = inst[ii];
  const int n = I.nc, kl = cs.kl[ii], ku = cs.ku[ii], kv = kl + ku, ldab = 2 * kl + ku + 1;
  const int K = kl + 1, T = blockDim.x;
  const int nw = T >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* AB = cs.band + cs.band_off[ii];
  int* ipiv = cs.ipiv + I.nc_off;
  double* S = gws ? gws + (long long)gslot[ii] * gstride : dyn;
  double* colj = gws ? dyn : S + (long long)K * K;   // column j below the pivot
  __shared__ double s_inv;
#define BEL(i, c) AB[(long long)(kv + (i) - (c)) + (long long)ldab * (c)]
  for (int e = threadIdx.x; e < K * K; e += T) {
    int i = e / K, c = e - i * K;
    S[e] = (i < n && c <= i && i - c <= kl) ? BEL(i, c) : 0.0;
  }
  __syncthreads();
  // the row entering the ring at the end of step j (row j + K, columns
  // j + 1 .. j + K) is still as assembled: loaded when the step starts
  const bool pf = K <= LU_PF * T;
  for (int j = 0; j < n; ++j) {
    const int km = min(kl, n - 1 - j);
    const int js = j % K, base = wrap(js + 1, K);
    const int inew = j + K;
    double pr[LU_PF];
    if (pf) {
#pragma unroll
      for (int q = 0; q < LU_PF; ++q) {
        const int c = inew - kl + threadIdx.x + q * T;
        pr[q] = (inew < n && c <= inew) ? BEL(inew, c) : 0.0;
      }
    }
    const double d = S[js * K + js];
    const long long db = __double_as_longlong(d);   // positive and finite, tested on the bits
    if (!(db > 0 && db < 0x7ff0000000000000LL)) {
      if (threadIdx.x == 0) failed[ii] = 1;
      return;
    }
    if (threadIdx.x == 0) s_inv = 1.0 / d;   // one division per step, not one per thread
    for (int t = threadIdx.x; t < km; t += T) colj[t] = S[wrap(base + t, K) * K + js];
    __syncthreads();
    const double inv = s_inv;
    // S(i, c) -= L'(i, j) S(c, j) for j < c <= i <= j + km: a warp per row
    for (int r = w; r < km; r += nw) {
      double* row = S + wrap(base + r, K) * K;
      const double lr = colj[r] * inv;
      for (int q = lane; q <= r; q += 32) row[wrap(base + q, K)] -= lr * colj[q];
    }
    // column j of the factors back to the band: pivot, multipliers, and the
    // upper row U(j, c) = S(c, j) stored in column c (from colj: no ring
    // reads, so this overlaps the update)
    for (int t = threadIdx.x; t <= km; t += T) {
      if (t == 0) {
        BEL(j, j) = d;
        ipiv[j] = j;
      } else {
        BEL(j + t, j) = colj[t - 1] * inv;
        BEL(j, j + t) = colj[t - 1];
      }
    }
    __syncthreads();
    // row j + K of the original matrix takes row j's slot
    if (pf) {
#pragma unroll
      for (int q = 0; q < LU_PF; ++q) {
        const int c = inew - kl + threadIdx.x + q * T;
        if (inew < n && c <= inew) S[js * K + c % K] = pr[q];
      }
    } else if (inew < n) {
      for (int c = inew - kl + threadIdx.x; c <= inew; c += T) S[js * K + c % K] = BEL(inew, c);
    }
    __syncthreads();
  }
#undef BEL
  if (threadIdx.x == 0) cs.bad[ii] = 0;
}

// Inverses of the diagonal blocks of factors without row interchanges, for
// the blocked band solve: block b covers band positions [b NB, b NB + NB),
// L_bb^-1 (unit lower) and U_bb^-1 (U = D L^T as stored), column-major, the
// identity beyond n.  One warp per (block, triangle); lane c forms column c
// of the inverse by substitution in shared memory.
constexpr int BINV_WARPS = 4;

__global__ void k_band_binv(const Inst* inst, int B, CoarseSys cs) {
  constexpr int NB = COARSE_NB, LD = NB + 1;
  extern __shared__ double dyn[];
  const int ii = blockIdx.x;
  if (!cs.nopiv[ii]) return;
  const Inst& I = inst[ii];
  const int n = I.nc, kl = cs.kl[ii], ku = cs.ku[ii], kv = kl + ku, ldab = 2 * kl + ku + 1;
  const double* AB = cs.band + cs.band_off[ii];
  double* out = cs.binv + cs.binv_off[ii];
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  double* M = dyn + (long long)w * 2 * NB * LD;
  double* X = M + NB * LD;
  const int nb = (n + NB - 1) / NB;
  for (int task = w; task < 2 * nb; task += BINV_WARPS) {
    const int b = task >> 1, j0 = b * NB, m = min(NB, n - j0);
    const bool upper = task & 1;
    for (int i = 0; i < NB; ++i) {   // lane c loads column c of the block
      double v = i == c ? 1.0 : 0.0;
      if (i < m && c < m) {
        const int d = i - c;
        if (upper ? (d <= 0 && -d <= ku) : (d > 0 && d <= kl))
          v = AB[(long long)(kv + d) + (long long)ldab * (j0 + c)];
      }
      M[i * LD + c] = v;
    }
    __syncwarp();
    if (!upper) {
      for (int i = 0; i < NB; ++i) {
        double s = i == c ? 1.0 : 0.0;
        if (i > c)
          for (int k = c; k < i; ++k) s -= M[i * LD + k] * X[k * LD + c];
        X[i * LD + c] = s;
      }
    } else {
      for (int i = NB - 1; i >= 0; --i) {
        double s = 0.0;
        if (i <= c) {
          s = i == c ? 1.0 : 0.0;
          for (int k = i + 1; k <= c; ++k) s -= M[i * LD + k] * X[k * LD + c];
          s /= M[i * LD + i];
        }
        X[i * LD + c] = s;
      }
    }
    __syncwarp();
    double* o = out + (long long)b * 2 * NB * NB + (upper ? NB * NB : 0);
    for (int cc = 0; cc < NB; ++cc) o[cc * NB + c] = X[c * LD + cc];
    __syncwarp();
  }
}

// Band LU (LAPACK gbtf2 steps) on the active block only: rows j..j+kl and a
// ring of K2 columns from j on, element (i, c) at (i mod (kl+1), c mod K2), in
// shared memory or, when it does not fit, in a per-CTA slice of global memory
// (`gws`, `gstride` doubles per CTA).  Each finished pivot row and multiplier
// column goes back to the band; row j + kl + 1 and column j + K2 enter the
// ring in their place.
//
// With K2 = kl + ku + 1 (extra < 0) the ring holds every fill that partial
// pivoting can cause.  With K2 = ku + 1 + extra the factorisation pivots by
// threshold -- the diagonal stays unless it is below tau times the column's
// largest entry -- and an instance whose row interchanges would spread fill
// beyond the ring sets failed[ii] and leaves its band to be refactored with
// the full ring.
//
// The system is numerically singular (cs.bad) when the chosen pivot is at most
// SING_EPS times the largest entry of its row as assembled (rows keep their
// scale in `sc` through the interchanges); an exactly zero column is the
// extreme case.  A coarse node whose truncated basis function is a single
// cell inside its own primal block has an R^FV column that sums to zero.
//
// The row and the column that enter the ring at the end of step j are still
// as assembled, so each thread loads its share of them (up to LU_PF values
// of each) when step j starts, and they arrive while the step eliminates;
// the entering row's scale is reduced per warp into `scw` and combined by
// thread 0 when the next step chooses its pivot.
__global__ void __launch_bounds__(1024) k_band_lu_act(const Inst* inst, int B, CoarseSys cs, const int* only, int* err,
                              double* gws, long long gstride, int extra, double tau, int* failed) {
  extern __shared__ double dyn[];
  int ii = blockIdx.x;
  if (!only[ii]) return;
  const Inst& I = inst[ii];
  const int n = I.nc, kl = cs.kl[ii], ku = cs.ku[ii], kv = kl + ku, ldab = 2 * kl + ku + 1;
  const int K1 = kl + 1, K2 = extra < 0 ? kv + 1 : min(kv + 1, ku + 1 + extra);
  const int T = blockDim.x;
  const int nw = T >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* S = gws ? gws + (long long)blockIdx.x * gstride : dyn;
  double* lj = gws ? dyn : dyn + (long long)K1 * K2;   // multipliers of column j
  double* ur = lj + K1;                                // pivot row j
  double* sc = ur + kv + 1;                            // scale of the row in each slot
  double* AB = cs.band + cs.band_off[ii];
  // the entering row spans columns j+1 .. j+kl+ku+1 (its scale), the ring
  // takes the first K2 of them; prefetch when every thread holds its share
  const int RW = kl + ku + 1;
  const bool pf = RW <= LU_PF * T && kl <= LU_PF * T;
  __shared__ double scw[32];
  int* ipiv = cs.ipiv + I.nc_off;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_jp, s_ju, s_bad, s_badcol;
  __shared__ double s_piv, s_inv;
#define BEL(i, c) AB[(long long)(kv + (i) - (c)) + (long long)ldab * (c)]
#define SEL(rs, c) S[(long long)(rs) * K2 + (c)]
#define INBAND(i, c) ((i) < n && (c) < n && (c) - (i) <= ku && (i) - (c) <= kl)
  if (threadIdx.x == 0) { s_ju = 0; s_bad = 0; s_badcol = -1; }
  for (int e = threadIdx.x; e < K1 * K2; e += T) {
    int i = e / K2, c = e - i * K2;
    S[e] = INBAND(i, c) ? BEL(i, c) : 0.0;
  }
  for (int i = w; i < K1; i += nw) {   // rows 0..kl sit in slots 0..kl
    double m = 0.0;
    if (i < n)
      for (int c = max(0, i - kl) + lane; c <= min(n - 1, i + ku); c += 32) m = fmax(m, fabs(BEL(i, c)));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sc[i] = m;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int km = min(kl, n - 1 - j);
    const int jr = j % K1, jc = j % K2;
    const int inew = j + K1, cnew = j + K2;
    // entering row inew (columns j+1..) and column cnew (rows j+1..j+kl)
    double prow[LU_PF], pcol[LU_PF];
    if (pf) {
#pragma unroll
      for (int q = 0; q < LU_PF; ++q) {
        const int cc = 1 + threadIdx.x + q * T, t = 1 + threadIdx.x + q * T;
        prow[q] = (cc <= RW && INBAND(inew, j + cc)) ? BEL(inew, j + cc) : 0.0;
        pcol[q] = (t < K1 && INBAND(j + t, cnew)) ? BEL(j + t, cnew) : 0.0;
      }
    }
    double best = -1.0;
    int bi = 0;
    for (int t = threadIdx.x; t <= km; t += T) {
      double v = fabs(SEL(wrap(jr + t, K1), jc));
      if (v > best) { best = v; bi = t; }
    }
    for (int o = 16; o; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[w] = best; si[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (pf && j > 0) {   // scale of the row that entered slot (j-1) % K1 at the last step
        double m = 0.0;
        for (int q = 0; q < nw; ++q) m = fmax(m, scw[q]);
        sc[(j - 1) % K1] = m;
      }
      double b0 = -1.0;
      int i0 = 0;
      for (int q = 0; q < nw; ++q)
        if (sv[q] > b0 || (sv[q] == b0 && si[q] < i0)) { b0 = sv[q]; i0 = si[q]; }
      if (fabs(SEL(jr, jc)) >= tau * b0) i0 = 0;   // threshold: keep the diagonal
      s_jp = i0;
      ipiv[j] = j + i0;
      const double p0 = SEL(wrap(jr + i0, K1), jc);
      if (!(b0 > 0.0) || !isfinite(b0) || !(fabs(p0) > SING_EPS * sc[wrap(jr + i0, K1)])) {
        s_bad = 1;
        s_badcol = j;
      } else {
        s_piv = p0;
        s_inv = 1.0 / p0;   // one division per step, not one per thread
      }
      s_ju = max(s_ju, min(j + ku + i0, n - 1));
      if (s_ju - j + 1 > K2) s_bad = 2;   // fill beyond the ring
    }
    __syncthreads();
    if (s_bad) break;
    const int jp = s_jp, ju = s_ju, wd = ju - j;
    const double piv = s_piv, inv = s_inv;
    if (jp != 0) {
      const int pr = wrap(jr + jp, K1);
      for (int cc = threadIdx.x; cc <= wd; cc += T) {
        int c = wrap(jc + cc, K2);
        double t = SEL(jr, c);
        SEL(jr, c) = SEL(pr, c);
        SEL(pr, c) = t;
      }
      if (threadIdx.x == 0) {
        double t = sc[jr];
        sc[jr] = sc[pr];
        sc[pr] = t;
      }
      __syncthreads();
    }
    for (int t = 1 + threadIdx.x; t <= km; t += T) lj[t] = SEL(wrap(jr + t, K1), jc) * inv;
    for (int cc = 1 + threadIdx.x; cc <= wd; cc += T) ur[cc] = SEL(jr, wrap(jc + cc, K2));
    __syncthreads();
    // rank-1 update.  Ring in shared memory: a thread per (column, group of
    // rows), the column's ring slot and pivot-row value in registers; the
    // thread walks its rows one ring row (K2 doubles) at a time, the ring's
    // wrap split out of the walk, two rows per pass.  Adjacent threads take
    // adjacent columns.
    if (gws) {
      // ring in global memory: a warp per row, lanes along the pivot row,
      // four independent loads in flight per lane
      for (int t = 1 + w; t <= km; t += nw) {
        const int rs = wrap(jr + t, K1);
        const double l = lj[t];
        for (int c0 = 1 + lane; c0 <= wd; c0 += 128) {
          double v[4];
          int cs_[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            int cc = c0 + 32 * u;
            cs_[u] = cc <= wd ? wrap(jc + cc, K2) : -1;
            v[u] = cs_[u] >= 0 ? SEL(rs, cs_[u]) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (cs_[u] >= 0) SEL(rs, cs_[u]) = v[u] - l * ur[c0 + 32 * u];
        }
      }
    } else if (wd > 0 && km > 0) {
      const int G = wd >= T ? 1 : T / wd;   // row groups
      const int per = (km + G - 1) / G;
      for (int e = threadIdx.x; e < G * wd; e += T) {
        const int g = e / wd, cc = 1 + e - g * wd;
        const int t1 = min(km, (g + 1) * per);
        const double u = ur[cc];
        const int c = wrap(jc + cc, K2);
        for (int t = 1 + g * per; t <= t1;) {
          const int rs = wrap(jr + t, K1);
          const int run = min(t1 - t + 1, K1 - rs);   // rows before the ring wraps
          double* q = S + (long long)rs * K2 + c;
          const double* l = lj + t;
          int k = 0;
          for (; k + 2 <= run; k += 2, q += 2 * K2) {
            const double a0 = q[0], a1 = q[K2];
            q[0] = a0 - l[k] * u;
            q[K2] = a1 - l[k + 1] * u;
          }
          for (; k < run; ++k, q += K2) q[0] -= l[k] * u;
          t += run;
        }
      }
    }
    // finished pivot row and multipliers back to the band (temporaries only)
    for (int cc = threadIdx.x; cc <= wd; cc += T) BEL(j, j + cc) = cc == 0 ? piv : ur[cc];
    for (int t = 1 + threadIdx.x; t <= km; t += T) BEL(j + t, j) = lj[t];
    __syncthreads();
    // column slot jc becomes column j + K2 (still original in the band: no
    // step so far reached it), row slot jr becomes row j + K1
    if (pf) {
      double m = 0.0;
#pragma unroll
      for (int q = 0; q < LU_PF; ++q) {
        const int cc = 1 + threadIdx.x + q * T, t = 1 + threadIdx.x + q * T;
        if (t < K1) SEL(wrap(jr + t, K1), jc) = pcol[q];
        if (cc <= K2) SEL(jr, wrap(jc + cc, K2)) = prow[q];
        m = fmax(m, fabs(prow[q]));
      }
      for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) scw[w] = m;
    } else {
      for (int t = 1 + threadIdx.x; t < K1; t += T) {
        int i = j + t;
        SEL(wrap(jr + t, K1), jc) = INBAND(i, cnew) ? BEL(i, cnew) : 0.0;
      }
      for (int cc = 1 + threadIdx.x; cc <= K2; cc += T) {
        int c = j + cc;
        SEL(jr, wrap(jc + cc, K2)) = INBAND(inew, c) ? BEL(inew, c) : 0.0;
      }
      if (w == nw - 1) {   // scale of the entering row, still as assembled in the band
        double m = 0.0;
        if (inew < n)
          for (int c = inew - kl + lane; c <= min(n - 1, inew + ku); c += 32) m = fmax(m, fabs(BEL(inew, c)));
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) sc[jr] = m;
      }
    }
    __syncthreads();
  }
#undef INBAND
#undef SEL
#undef BEL
  if (threadIdx.x == 0) {
    if (s_bad == 2) {
      failed[ii] = 1;
    } else {
      cs.bad[ii] = s_bad ? s_badcol + 1 : 0;
    }
  }
}

}  // namespace

// mode < 0: each instance's own restriction; 0: R^FV for all; 1: R^FE for all
// reuse: the system was built before and the fine operator kept its pattern
// (a time-step update): A_c is summed again and refactored with the same
// ordering, bandwidths and band layout
int build_coarse_system(Batch& b, CoarseSys& cs, int mode, CoarseHost& ch, bool reuse,
                        const int* p_ptr, const int* p_col, const double* p_val) {
  const int T = 256;
  cudaStream_t st = b.stream;
  long long nct = b.tot_nc;
  int B = b.B;
  long long tot = 0;
  for (int i = 0; i < B; ++i) tot += (long long)b.h[i].nc * b.h[i].nc;
  if (!reuse) {
    // dense A_c per instance
    ch.ac_off.assign(B, 0);
    long long o = 0;
    for (int i = 0; i < B; ++i) {
      ch.ac_off[i] = o;
      o += (long long)b.h[i].nc * b.h[i].nc;
    }
    FAMS_TRY(b.alloc((void**)&cs.Ac, sizeof(double) * (tot + 1)));
    FAMS_TRY(b.alloc((void**)&cs.ac_off, sizeof(long long) * B));
    FAMS_TRY(b.alloc((void**)&cs.kl, sizeof(int) * B));
    FAMS_TRY(b.alloc((void**)&cs.ku, sizeof(int) * B));
    FAMS_TRY(b.alloc((void**)&cs.band_off, sizeof(long long) * B));
    FAMS_TRY(b.alloc((void**)&cs.ipiv, sizeof(int) * (nct + 1)));
    FAMS_TRY(b.alloc((void**)&cs.perm, sizeof(int) * (nct + 1)));
    FAMS_TRY(b.alloc((void**)&cs.bad, sizeof(int) * B));
    FAMS_TRY(b.alloc((void**)&cs.nopiv, sizeof(int) * B));
    FAMS_TRY(b.alloc((void**)&cs.binv_off, sizeof(long long) * B));
    FAMS_CUDA(cudaMemcpyAsync(cs.ac_off, ch.ac_off.data(), sizeof(long long) * B,
                              cudaMemcpyHostToDevice, st));
  }
  FAMS_CUDA(cudaMemsetAsync(cs.Ac, 0, sizeof(double) * (tot + 1), st));
  if (b.tot_nnz > 0)
    fams::note_launch(), k_rap<<<grid_for(b.tot_nnz, T), T, 0, st>>>(b.d_inst, B, b.off_row, b.tot_nnz, b.rowptr, b.col,
                                                b.val, b.tot_row, b.primal, p_ptr, p_col,
                                                p_val, cs, mode);
  int* ip = nullptr;
  FAMS_TRY(b.scratch((void**)&ip, sizeof(int) * (nct + 1)));
  if (!reuse) {
    // pattern, RCM, band sizes
    int *cnt = nullptr, *ptr = nullptr, *cols = nullptr, *vis = nullptr, *que = nullptr;
    FAMS_TRY(b.scratch((void**)&cnt, sizeof(int) * (nct + 1)));
    FAMS_TRY(b.scratch((void**)&ptr, sizeof(int) * (nct + 1)));
    FAMS_TRY(b.scratch((void**)&vis, sizeof(int) * (nct + 1)));
    FAMS_TRY(b.scratch((void**)&que, sizeof(int) * (nct + 1)));
    fams::note_launch(), k_ac_count<<<grid_for(nct * 32, T), T, 0, st>>>(b.d_inst, B, b.off_nc, nct, cs, cnt);
    long long nnzc = 0;
    FAMS_TRY(exclusive_scan(b, cnt, ptr, nct, &nnzc));
    FAMS_TRY(b.scratch((void**)&cols, sizeof(int) * (nnzc + 1)));
    fams::note_launch(), k_ac_cols<<<grid_for(nct, 64), 64, 0, st>>>(b.d_inst, B, b.off_nc, nct, cs, ptr, cols);
    int *dkl = nullptr, *dku = nullptr;
    FAMS_TRY(b.scratch((void**)&dkl, sizeof(int) * B));
    FAMS_TRY(b.scratch((void**)&dku, sizeof(int) * B));
    FAMS_CUDA(cudaMemsetAsync(dkl, 0, sizeof(int) * B, st));
    FAMS_CUDA(cudaMemsetAsync(dku, 0, sizeof(int) * B, st));
    fams::note_launch(), k_rcm<<<B, 32, 0, st>>>(b.d_inst, B, ptr, cols, cs, vis, que, b.d_err);
    fams::note_launch(), k_inverse_perm<<<grid_for(nct, T), T, 0, st>>>(b.d_inst, B, b.off_nc, nct, cs, ip);
    fams::note_launch(), k_bandwidth<<<grid_for(nct, 64), 64, 0, st>>>(b.d_inst, B, b.off_nc, nct, cs, ip, dkl, dku);
    FAMS_CUDA(cudaGetLastError());
    ch.kl.assign(B, 0);
    ch.ku.assign(B, 0);
    FAMS_CUDA(cudaMemcpyAsync(ch.kl.data(), dkl, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(ch.ku.data(), dku, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
    ch.band_off.assign(B, 0);
    long long bt = 0;
    for (int i = 0; i < B; ++i) {
      ch.band_off[i] = bt;
      bt += (long long)(2 * ch.kl[i] + ch.ku[i] + 1) * b.h[i].nc;
    }
    ch.band_tot = bt;
    FAMS_TRY(b.alloc((void**)&cs.band, sizeof(double) * (bt + 1)));
    FAMS_CUDA(cudaMemcpyAsync(cs.kl, ch.kl.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
    FAMS_CUDA(cudaMemcpyAsync(cs.ku, ch.ku.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
    FAMS_CUDA(cudaMemcpyAsync(cs.band_off, ch.band_off.data(), sizeof(long long) * B,
                              cudaMemcpyHostToDevice, st));
  } else {
    fams::note_launch(), k_inverse_perm<<<grid_for(nct, T), T, 0, st>>>(b.d_inst, B, b.off_nc, nct, cs, ip);
  }
  FAMS_CUDA(cudaMemsetAsync(cs.band, 0, sizeof(double) * (ch.band_tot + 1), st));
  fams::note_launch(), k_band_fill<<<grid_for(nct, 64), 64, 0, st>>>(b.d_inst, B, b.off_nc, nct, cs, ip,
                                                                   nullptr);
  // a single instance whose coarse system the one-CTA iteration cannot hold
  // (a band wider than its shared-memory chunks) goes to the whole GPU when
  // the caller left the choice to the library (grid_solve = 0)
  if (!reuse && mode < 0 && B == 1 && b.h[0].grid_solve == 0 && !whole_gpu(b) &&
      !one_cta_fits(b, b.h[0].nc, ch.kl[0], ch.ku[0],
                    b.h[0].krylov == FAMS_KRYLOV_GMRES ? b.h[0].restart : 0)) {
    b.h[0].grid_solve = 1;
    FAMS_CUDA(cudaMemcpyAsync(b.d_inst, b.h.data(), sizeof(Inst), cudaMemcpyHostToDevice, st));
  }
  if (whole_gpu(b)) {
    // one large instance: band LU with partial pivoting on every SM (its
    // iteration solves with A_c^-1 formed from these factors)
    FAMS_TRY(band_lu_grid(b, cs, ch));
    if (!reuse) {
      ch.binv_off.assign(B, 0);
      FAMS_TRY(b.alloc((void**)&cs.binv, sizeof(double)));
      FAMS_CUDA(cudaMemcpyAsync(cs.binv_off, ch.binv_off.data(), sizeof(long long) * B,
                                cudaMemcpyHostToDevice, st));
    }
    return b.check_err("coarse LU");
  }
  // factorisation: LDL^T for the symmetric positive definite (R^FE) systems
  // whose active triangle fits in shared memory, band LU for the others and
  // for any LDL^T that meets a non-positive pivot
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  max_smem -= 1024;   // static shared memory of the kernels
  // (rings too large for shared memory in global slices: LDL^T on a global
  // ring has half the band LU's work and no pivot search)
  std::vector<int> spd(B, 0), lu(B, 0), ldl_ok(B, 0), spd_s(B, 0), spd_g(B, 0), gslot(B, -1);
  size_t ldl_smem = 0, ldl_gsmem = 0;
  long long gstride = 0;
  int ng = 0;
  for (int i = 0; i < B; ++i) {
    bool fe = mode == 1 || (mode < 0 && b.h[i].restriction == FAMS_R_FE);
    const size_t K = (size_t)ch.kl[i] + 1;
    size_t need = sizeof(double) * (K * K + K);
    if (fe && ch.kl[i] == ch.ku[i]) {
      spd[i] = 1;
      if (need <= (size_t)max_smem) {
        spd_s[i] = 1;
        ldl_smem = std::max(ldl_smem, need);
      } else {
        spd_g[i] = 1;
        gslot[i] = ng++;
        gstride = std::max(gstride, (long long)(K * K));
        ldl_gsmem = std::max(ldl_gsmem, sizeof(double) * K);
      }
    } else {
      lu[i] = 1;
    }
  }
  int *d_spd = nullptr, *d_lu = nullptr, *d_spdg = nullptr, *d_gslot = nullptr;
  FAMS_TRY(b.scratch((void**)&d_spd, sizeof(int) * B));
  FAMS_TRY(b.scratch((void**)&d_lu, sizeof(int) * B));
  FAMS_CUDA(cudaMemcpyAsync(d_spd, spd_s.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
  FAMS_CUDA(cudaMemsetAsync(d_lu, 0, sizeof(int) * B, st));
  FAMS_CUDA(cudaMemsetAsync(cs.bad, 0, sizeof(int) * B, st));
  if (ldl_smem > 0 || ng > 0) {
    FAMS_CUDA(cudaFuncSetAttribute(k_band_ldl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   max_smem));
    if (ldl_smem > 0)
      fams::note_launch(), k_band_ldl<<<B, LDL_T, ldl_smem, st>>>(b.d_inst, B, cs, d_spd, d_lu,
                                                               nullptr, nullptr, 0);
    if (ng > 0) {
      double* gws = nullptr;
      FAMS_TRY(b.scratch((void**)&d_spdg, sizeof(int) * B));
      FAMS_TRY(b.scratch((void**)&d_gslot, sizeof(int) * B));
      FAMS_TRY(b.scratch((void**)&gws, sizeof(double) * (size_t)gstride * ng));
      FAMS_CUDA(cudaMemcpyAsync(d_spdg, spd_g.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
      FAMS_CUDA(cudaMemcpyAsync(d_gslot, gslot.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
      fams::note_launch(), k_band_ldl<<<B, 1024, ldl_gsmem, st>>>(b.d_inst, B, cs, d_spdg, d_lu,
                                                                 gws, d_gslot, gstride);
    }
    FAMS_CUDA(cudaGetLastError());
    std::vector<int> failed(B, 0);
    FAMS_CUDA(cudaMemcpyAsync(failed.data(), d_lu, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
    bool any = false;
    for (int i = 0; i < B; ++i) any |= failed[i] != 0;
    if (any) {   // back to the assembled matrix for the band LU
      for (int i = 0; i < B; ++i)
        if (failed[i])
          FAMS_CUDA(cudaMemsetAsync(cs.band + ch.band_off[i], 0,
                                    sizeof(double) * (2 * ch.kl[i] + ch.ku[i] + 1) * b.h[i].nc, st));
      fams::note_launch(), k_band_fill<<<grid_for(nct, 64), 64, 0, st>>>(b.d_inst, B, b.off_nc, nct,
                                                                         cs, ip, d_lu);
    }
    for (int i = 0; i < B; ++i) {
      lu[i] |= failed[i];
      ldl_ok[i] = spd[i] && !failed[i];
    }
  }
  // band LU on the active block.  R^FE systems whose LDL^T failed first try
  // a narrow ring (threshold pivoting, fill up to LU_EXTRA columns past the
  // upper band) in shared memory; then the full ring of partial pivoting for
  // the R^FV systems and for the instances that did not fit the narrow ring
  // or pivoted beyond it: in shared memory where it fits, else in global
  // scratch
  FAMS_CUDA(cudaFuncSetAttribute(k_band_lu_act, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem));
  size_t temps = 0;
  for (int i = 0; i < B; ++i)   // multipliers, pivot row and row scales of the widest band
    if (lu[i]) temps = std::max(temps, sizeof(double) * (size_t)(3 * ch.kl[i] + ch.ku[i] + 3));
  {
    std::vector<int> lu_n(B, 0);
    size_t act_n = 0;
    for (int i = 0; i < B; ++i) {
      // R^FV systems (high contrast, often pivoting across the whole lower
      // band) fail the narrow ring too often to gain from it: full ring first
      const bool fe = mode == 1 || (mode < 0 && b.h[i].restriction == FAMS_R_FE);
      if (!lu[i] || !fe) continue;
      size_t k2 = (size_t)std::min(ch.kl[i] + ch.ku[i] + 1, ch.ku[i] + 1 + LU_EXTRA);
      size_t act = (size_t)(ch.kl[i] + 1) * k2;
      if (sizeof(double) * act + temps <= (size_t)max_smem) {
        lu_n[i] = 1;
        act_n = std::max(act_n, act);
      }
    }
    if (act_n > 0) {
      int *d_n = nullptr, *d_f = nullptr;
      FAMS_TRY(b.scratch((void**)&d_n, sizeof(int) * B));
      FAMS_TRY(b.scratch((void**)&d_f, sizeof(int) * B));
      FAMS_CUDA(cudaMemcpyAsync(d_n, lu_n.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
      FAMS_CUDA(cudaMemsetAsync(d_f, 0, sizeof(int) * B, st));
      fams::note_launch(), k_band_lu_act<<<B, LU_SMEM_T, sizeof(double) * act_n + temps, st>>>(
          b.d_inst, B, cs, d_n, b.d_err, nullptr, 0, LU_EXTRA, LU_TAU, d_f);
      FAMS_CUDA(cudaGetLastError());
      std::vector<int> failed(B, 0);
      FAMS_CUDA(cudaMemcpyAsync(failed.data(), d_f, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
      FAMS_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int i = 0; i < B; ++i) {
        if (lu_n[i] && !failed[i]) lu[i] = 0;   // done
        if (failed[i]) {
          any = true;
          FAMS_CUDA(cudaMemsetAsync(cs.band + ch.band_off[i], 0,
                                    sizeof(double) * (2 * ch.kl[i] + ch.ku[i] + 1) * b.h[i].nc, st));
        }
      }
      if (any) {
        FAMS_CUDA(cudaMemcpyAsync(d_f, failed.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
        fams::note_launch(), k_band_fill<<<grid_for(nct, 64), 64, 0, st>>>(b.d_inst, B, b.off_nc, nct,
                                                                           cs, ip, d_f);
      }
    }
  }
  std::vector<int> lu_s(B, 0), lu_g(B, 0);
  size_t act_s = 0, act_g = 0;
  for (int i = 0; i < B; ++i) {
    if (!lu[i]) continue;
    size_t act = (size_t)(ch.kl[i] + 1) * (size_t)(ch.kl[i] + ch.ku[i] + 1);
    if (sizeof(double) * act + temps <= (size_t)max_smem) {
      lu_s[i] = 1;
      act_s = std::max(act_s, act);
    } else {
      lu_g[i] = 1;
      act_g = std::max(act_g, act);
    }
  }
  // the shared-memory and the global-memory passes factor disjoint sets of
  // instances: when both run, the global one goes on a second stream so that
  // the two overlap (each keeps only a few CTAs busy)
  int* d_lg = nullptr;
  double* gws = nullptr;
  if (act_g > 0) {
    FAMS_TRY(b.scratch((void**)&d_lg, sizeof(int) * B));
    FAMS_TRY(b.scratch((void**)&gws, sizeof(double) * act_g * (size_t)B));
    FAMS_CUDA(cudaMemcpyAsync(d_lg, lu_g.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
  }
  if (act_s > 0) FAMS_CUDA(cudaMemcpyAsync(d_lu, lu_s.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
  cudaStream_t gst = st;
  if (act_s > 0 && act_g > 0) {
    if (!b.aux) {
      FAMS_CUDA(cudaStreamCreateWithFlags(&b.aux, cudaStreamNonBlocking));
      FAMS_CUDA(cudaEventCreateWithFlags(&b.aux_ev, cudaEventDisableTiming));
      FAMS_CUDA(cudaEventCreateWithFlags(&b.aux_done, cudaEventDisableTiming));
    }
    FAMS_CUDA(cudaEventRecord(b.aux_ev, st));
    FAMS_CUDA(cudaStreamWaitEvent(b.aux, b.aux_ev, 0));
    gst = b.aux;
  }
  if (act_s > 0)
    fams::note_launch(), k_band_lu_act<<<B, LU_SMEM_T, sizeof(double) * act_s + temps, st>>>(
        b.d_inst, B, cs, d_lu, b.d_err, nullptr, 0, -1, 1.0, nullptr);
  if (act_g > 0)
    fams::note_launch(), k_band_lu_act<<<B, 1024, temps, gst>>>(b.d_inst, B, cs, d_lg, b.d_err, gws,
                                                                  (long long)act_g, -1, 1.0, nullptr);
  FAMS_CUDA(cudaGetLastError());
  if (gst != st) {
    FAMS_CUDA(cudaEventRecord(b.aux_done, gst));
    FAMS_CUDA(cudaStreamWaitEvent(st, b.aux_done, 0));
  }
  // inverse diagonal blocks of the LDL^T factors (room for every instance that
  // tries LDL^T, which the same bandwidths decide again on a refactorisation)
  if (!reuse) {
    ch.binv_off.assign(B, 0);
    long long tot_binv = 0;
    for (int i = 0; i < B; ++i) {
      ch.binv_off[i] = tot_binv;
      if (spd[i])
        tot_binv += (long long)((b.h[i].nc + COARSE_NB - 1) / COARSE_NB) * 2 * COARSE_NB * COARSE_NB;
    }
    FAMS_TRY(b.alloc((void**)&cs.binv, sizeof(double) * (tot_binv + 1)));
    FAMS_CUDA(cudaMemcpyAsync(cs.binv_off, ch.binv_off.data(), sizeof(long long) * B,
                              cudaMemcpyHostToDevice, st));
  }
  FAMS_CUDA(cudaMemcpyAsync(cs.nopiv, ldl_ok.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
  bool any_ldl = false;
  for (int i = 0; i < B; ++i) any_ldl |= ldl_ok[i] != 0;
  if (any_ldl) {
    const size_t sm = sizeof(double) * BINV_WARPS * 2 * COARSE_NB * (COARSE_NB + 1);
    FAMS_CUDA(cudaFuncSetAttribute(k_band_binv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    fams::note_launch(), k_band_binv<<<B, 32 * BINV_WARPS, sm, st>>>(b.d_inst, B, cs);
    FAMS_CUDA(cudaGetLastError());
  }
  ch.bad.assign(B, 0);
  FAMS_CUDA(cudaMemcpyAsync(ch.bad.data(), cs.bad, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaStreamSynchronize(st));
  return b.check_err("coarse LU");
}

int phase_coarse_op(Batch& b, int mode) {
  return build_coarse_system(b, b.cs[0], mode, b.csh[0], false, b.p_ptr, b.p_col, b.p_val);
}

}  // namespace fams
