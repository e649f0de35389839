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

#include <cuda_bf16.h>

#include "band_solve.cuh"
#include "batch.cuh"

namespace fams {

namespace {

constexpr int SOLVE_T = 512;
constexpr int ROWS_ILP = 4;
constexpr int BAND_BUF = 3072;   // doubles per staged chunk of band columns (24 KiB)
constexpr int SWEEP_RING = 1024; // level positions of recent sweep results kept in shared memory
// Rows of the triangular sweeps are copied into shared memory STAGE_D - 1
// levels ahead of their use (asynchronous copies, no registers held):
// threads 0..STAGE_W-1 take the first STAGE_W rows of a level, the other
// threads the rest of a wider level with plain loads.  Per staged row:
// STAGE_V values in the sweep's arithmetic (PK factor entries, right-hand
// side, reciprocal diagonal), the FP64 part of the output the U sweep adds
// to, and STAGE_I integers (PK neighbour positions, entry count, first CSR
// entry of L or the row of U).
// Ring and stages fit in the band buffer, so two CTAs per SM still leave
// about 90 KB of L1 to the sparse products: deeper staging (3 or 4 levels)
// took the SM's L1 (or the second CTA) and was slower overall.
constexpr int STAGE_D = 2;
constexpr int STAGE_W = 256;
constexpr int STAGE_V = PK + 2;
constexpr int STAGE_I = PK + 2;
constexpr int STAGE_SLOTS = STAGE_D * STAGE_W;
static_assert(SOLVE_T > STAGE_W, "threads beyond the staged rows take the rest of a level");
// shared memory behind the coarse vectors: the coarse solve's two band
// chunks, or during the sweeps the ring followed by the staged rows
constexpr size_t SWEEP_BYTES = SWEEP_RING * sizeof(double) +
    (size_t)STAGE_SLOTS * ((STAGE_V + 1) * sizeof(double) + STAGE_I * sizeof(int));
constexpr size_t BUF_BYTES =
    SWEEP_BYTES > 2 * BAND_BUF * sizeof(double) ? SWEEP_BYTES : 2 * BAND_BUF * sizeof(double);
static_assert(BUF_BYTES % sizeof(double) == 0, "the buffer is counted in doubles");
constexpr int BUF_DOUBLES = (int)(BUF_BYTES / sizeof(double));

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

__global__ void k_round(long long n, const double* src, float* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

__global__ void k_round_bf16(long long n, const double* src, __nv_bfloat16* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __double2bfloat16(src[i]);
}

__global__ void k_make_q(long long n, const double* rhs, const double* qD, double* q) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (rhs ? rhs[i] : 0.0) + qD[i];
}

struct SolveArgs {
  const Inst* inst;
  const int* active;   // per instance: 1 to solve (null: every instance)
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
  // the sub-block smoothing stage: ILU(0) of A without its cross-medium
  // entries, in the pattern of A and in level order (null: no instance has it)
  const double* Fb;
  const double* pk_lvb;
  const double* pk_uvb;
  const double* pk_udb;
  double* ylev;
  double* xlev;    // level order: the part of the two-stage output the U sweep adds to
  long long ntot;  // rows of the batch (stride of the PK arrays)
  double tol;
  // FP32 copies and work vectors of the mixed-precision inner stages
  const float* p_val32;
  const float* pt_val32;
  const __nv_bfloat16* p_val16;    // BF16 storage of P and P^T (fams_opts.bf16_p)
  const __nv_bfloat16* pt_val16;
  const float* F32;
  const float* pk_lv32;
  const float* pk_uv32;
  const float* pk_ud32;
  double* xs;     // iterate saved before an FP32 cycle
  float* yf;
  float* ylevf;
};

// the arrays of one arithmetic: FP64 throughout, or the FP32 copies
template <class T> struct Prec;
template <> struct Prec<double> {
  static __device__ const double* F(const SolveArgs& a, int set = 0) { return set ? a.Fb : a.F; }
  static __device__ const double* lv(const SolveArgs& a, int set = 0) { return set ? a.pk_lvb : a.pk_lv; }
  static __device__ const double* uv(const SolveArgs& a, int set = 0) { return set ? a.pk_uvb : a.pk_uv; }
  static __device__ const double* ud(const SolveArgs& a, int set = 0) { return set ? a.pk_udb : a.pk_ud; }
  static __device__ double* y(const SolveArgs& a) { return a.y; }
  static __device__ double* ylev(const SolveArgs& a) { return a.ylev; }
};
template <> struct Prec<float> {
  // (the sub-block stage runs in FP64 only: set 1 is never asked for here)
  static __device__ const float* F(const SolveArgs& a, int = 0) { return a.F32; }
  static __device__ const float* lv(const SolveArgs& a, int = 0) { return a.pk_lv32; }
  static __device__ const float* uv(const SolveArgs& a, int = 0) { return a.pk_uv32; }
  static __device__ const float* ud(const SolveArgs& a, int = 0) { return a.pk_ud32; }
  static __device__ float* y(const SolveArgs& a) { return a.yf; }
  static __device__ float* ylev(const SolveArgs& a) { return a.ylevf; }
};

// where the restriction and prolongation read P's values: FP64, the FP32
// copies, or their BF16 storage (widened to FP32 on load)
template <class TP> struct PVals;
template <> struct PVals<double> {
  static __device__ const double* pv(const SolveArgs& a) { return a.p_val; }
  static __device__ const double* ptv(const SolveArgs& a) { return a.pt_val; }
};
template <> struct PVals<float> {
  static __device__ const float* pv(const SolveArgs& a) { return a.p_val32; }
  static __device__ const float* ptv(const SolveArgs& a) { return a.pt_val32; }
};
template <> struct PVals<__nv_bfloat16> {
  static __device__ const __nv_bfloat16* pv(const SolveArgs& a) { return a.p_val16; }
  static __device__ const __nv_bfloat16* ptv(const SolveArgs& a) { return a.pt_val16; }
};

// y[i] = b[i] - sum_p val[p] v[col[p]] in FP64 for the instance's rows, four
// rows per thread in flight; y (and ylev, in level order) are stored in the
// arithmetic TO of their consumer.  Returns this thread's sum of y^2 when
// `norm`.
template <class TO>
__device__ inline double rows_residual(const SolveArgs& a, int ro, int n, const double* b,
                                       const double* v, TO* y, bool norm, TO* ylev = nullptr) {
  const double* val = a.val;
  double acc = 0;
  const int NT = blockDim.x;
  for (int i0 = ro + threadIdx.x; i0 < ro + n; i0 += ROWS_ILP * NT) {
    int rs[ROWS_ILP], re[ROWS_ILP];
    double s[ROWS_ILP];
    int m = 0;
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * NT;
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
        if (p < re[k]) s[k] -= val[p] * v[a.col[p]];
      }
    }
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * NT;
      if (i < ro + n) {
        y[i] = (TO)s[k];
        if (ylev) ylev[a.pk_pos[i]] = (TO)s[k];
        if (norm) acc += s[k] * s[k];
      }
    }
  }
  return acc;
}

// Band solve of factors without row interchanges (LDL^T, stored as unit L and
// U = D L^T) in blocks of COARSE_NB band positions: a block's unknowns come
// from its precomputed inverse diagonal block (a small dense product instead
// of COARSE_NB dependent steps), then the rows the block couples to are
// updated.  Forward with L, then backward with U.  Every thread takes part;
// partial sums are combined in a fixed order.  part: 4 (COARSE_NB + kl)
// doubles of shared memory.
__device__ void coarse_solve_blocked(const double* AB, const double* binv, int n, int kl, int ku,
                                     double* yb, double* part) {
  constexpr int NB = COARSE_NB;
  const int kv = kl + ku, ldab = 2 * kl + ku + 1;
  const int T = blockDim.x, tid = threadIdx.x;
  const int nb = (n + NB - 1) / NB;
  double* pd = part;            // 4 x NB partial sums of the diagonal block
  double* pr = part + 4 * NB;   // 4 x (coupled rows) partial sums
  for (int s = 0; s < 2 * nb; ++s) {
    const bool fwd = s < nb;
    const int b = fwd ? s : 2 * nb - 1 - s;
    const int j0 = b * NB, m = min(NB, n - j0);
    const double* X = binv + (long long)b * 2 * NB * NB + (fwd ? 0 : NB * NB);
    if (tid < 4 * NB) {
      // eight independent loads in flight, then the products
      const int i = tid & (NB - 1), q = tid / NB;
      double xv[8], yv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = 8 * q + u;
        const bool ok = i < m && c < m && (fwd ? c <= i : c >= i);
        xv[u] = ok ? X[c * NB + i] : 0.0;
        yv[u] = ok ? yb[j0 + c] : 0.0;
      }
      double acc = 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += xv[u] * yv[u];
      pd[q * NB + i] = acc;
    }
    __syncthreads();
    if (tid < m) yb[j0 + tid] = (pd[tid] + pd[NB + tid]) + (pd[2 * NB + tid] + pd[3 * NB + tid]);
    __syncthreads();
    // rows coupled to the block: below it within kl (forward), above it within ku (backward)
    const int r0 = fwd ? j0 + NB : max(0, j0 - ku);
    const int r1 = fwd ? min(n, j0 + m + kl) : j0;
    const int nr = max(0, r1 - r0);
    for (int e = tid; e < 4 * nr; e += T) {
      const int q = e / nr, i = r0 + e - q * nr;
      double av[8], yv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = j0 + 8 * q + u, d = i - c;
        const bool ok = c < j0 + m && (fwd ? d <= kl : -d <= ku);
        av[u] = ok ? AB[(long long)(kv + d) + (long long)ldab * c] : 0.0;
        yv[u] = ok ? yb[c] : 0.0;
      }
      double acc = 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += av[u] * yv[u];
      pr[e] = acc;
    }
    __syncthreads();
    for (int t = tid; t < nr; t += T)
      yb[r0 + t] -= (pr[t] + pr[nr + t]) + (pr[2 * nr + t] + pr[3 * nr + t]);
    __syncthreads();
  }
}

// Asynchronous global -> shared copies of 4 or 8 bytes (cp.async): each
// thread waits for its own groups only and reads only what it copied itself.
template <int BYTES>
__device__ inline void cp_async(void* dst, const void* src) {
  static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte copies");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Staged rows of a triangular sweep in shared memory, [field][slot], slot =
// stage * STAGE_W + thread.  x: the FP64 output part (U); v: PK factor
// entries, then right-hand side and reciprocal diagonal (U); c: PK neighbour
// positions, then entry count and first CSR entry (L) or row (U).
template <class T>
struct Stage {
  double* x;
  T* v;
  int* c;
};
template <class T>
__device__ inline Stage<T> stage_of(double* buf) {
  char* p = reinterpret_cast<char*>(buf) + SWEEP_RING * sizeof(double);
  char* pv = p + (size_t)STAGE_SLOTS * sizeof(double);
  return Stage<T>{reinterpret_cast<double*>(p), reinterpret_cast<T*>(pv),
                  reinterpret_cast<int*>(pv + (size_t)STAGE_V * STAGE_SLOTS * sizeof(T))};
}

// Copies this thread's row of the level at positions [lo, hi) (none: lo ==
// hi) into stage slot `stage` and commits one group (empty without a row).
// Every address depends only on the level position t, so the copies of a
// whole level are coalesced.
template <class T, bool LOWER>
__device__ inline void stage_rows(const SolveArgs& a, int lo, int hi, int set, const Stage<T>& sg,
                                  int stage) {
  const int tid = threadIdx.x;
  const int t = lo + tid;
  if (tid < STAGE_W && t < hi) {
    const int sl = stage * STAGE_W + tid;
    const int* pc = LOWER ? a.pk_lc : a.pk_uc;
    const T* pv = LOWER ? Prec<T>::lv(a, set) : Prec<T>::uv(a, set);
#pragma unroll
    for (int k = 0; k < PK; ++k) {
      cp_async<4>(sg.c + k * STAGE_SLOTS + sl, pc + (long long)k * a.ntot + t);
      cp_async<sizeof(T)>(sg.v + k * STAGE_SLOTS + sl, pv + (long long)k * a.ntot + t);
    }
    cp_async<sizeof(T)>(sg.v + PK * STAGE_SLOTS + sl, Prec<T>::ylev(a) + t);
    if (LOWER) {
      cp_async<4>(sg.c + PK * STAGE_SLOTS + sl, a.pk_nl + t);
      cp_async<4>(sg.c + (PK + 1) * STAGE_SLOTS + sl, a.pk_lp + t);
    } else {
      cp_async<4>(sg.c + PK * STAGE_SLOTS + sl, a.pk_nu + t);
      cp_async<4>(sg.c + (PK + 1) * STAGE_SLOTS + sl, a.lev_rows + t);
      cp_async<sizeof(T)>(sg.v + (PK + 1) * STAGE_SLOTS + sl, Prec<T>::ud(a, set) + t);
      cp_async<8>(sg.x + sl, a.xlev + t);
    }
  }
  cp_commit();
}

// shared-memory layout of the solve kernels (doubles): the coarse vector in
// band order, the coarse correction in coarse order, BUF_DOUBLES for the
// band chunks or the sweeps; the GMRES kernel adds its small dense arrays
// after them
struct SolveSmem {
  double* yb;
  double* ecs;
  double* buf;
  int* pbuf;
};

// SM cycles per phase, kept by thread 0 in shared memory: cyc[0..5] the six
// phases, cyc[6] the time stamp of the last mark (no registers held across
// the phases)
constexpr int NCYC = 7;
__device__ inline void stamp(long long* cyc) {
  if (threadIdx.x == 0) cyc[6] = clock64();
}
__device__ inline void mark(long long* cyc, int k) {
  if (threadIdx.x == 0) {
    const long long now = clock64();
    cyc[k] += now - cyc[6];
    cyc[6] = now;
  }
}

// Steps 5-7 of Table 1 on a residual r, in the arithmetic T of the vectors
// (the coarse solve is FP64 in both; SM cycles of the phases are added to
// cyc by thread 0):
//   dp = P A_c^-1 R r;  y = r - A dp (also in level order);
//   out = (base + dp) + (LU)^-1 y   (base null: out = dp + (LU)^-1 y)
// base + dp is kept in level order (xlev) for the U sweep.
// out may alias base; r, dp and out must not alias y, ylev or xlev.
template <class T, class TP = T>
__device__ __forceinline__ void two_stage(const SolveArgs& a, const Inst& I, int ii, const double* r,
                                          double* dp, double* out, const double* base,
                                          const SolveSmem& S, long long* cyc) {
  const int n = I.n, ro = I.row_off, nc = I.nc, co = I.nc_off;
  const double* AB = a.cs.band + a.cs.band_off[ii];
  const int* ipiv = a.cs.ipiv + co;
  const int* perm = a.cs.perm + co;
  const int kl = a.cs.kl[ii], ku = a.cs.ku[ii];
  const int* lp = a.lev_ptr + a.lev_off[ii];
  const int nlev = I.nlev;
  const int NT = blockDim.x;
  const TP* ptv = PVals<TP>::ptv(a);
  const TP* pv = PVals<TP>::pv(a);
  T* y = Prec<T>::y(a);
  T* ylev = Prec<T>::ylev(a);
  stamp(cyc);
  // step 5: coarse right-hand side R r, in band order: one warp per coarse
  // row (a row of P^T or a primal block holds hundreds of cells), lanes
  // along the row, then a fixed butterfly sum
  {
    const int lane = threadIdx.x & 31, nw = NT >> 5;
    for (int k = threadIdx.x >> 5; k < nc; k += nw) {
      const int c = co + perm[k];
      T s = 0;
      // MSMIX: P^T rows for the matrix coarse nodes, indicators for the fracture ones
      if (I.restriction == FAMS_R_FE || (I.restriction == FAMS_R_MIX && perm[k] < I.ncm)) {
        for (int p = a.pt_ptr[c] + lane; p < a.pt_ptr[c + 1]; p += 32) s += (T)ptv[p] * (T)r[a.pt_col[p]];
      } else {
        for (int p = a.blk_ptr[c] + lane; p < a.blk_ptr[c + 1]; p += 32) s += (T)r[a.blk_cell[p]];
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        S.yb[k] = (double)s;
        a.crhs[c] = (double)s;
      }
    }
  }
  __syncthreads();
  mark(cyc, 1);
  if (a.cs.nopiv[ii] && 4 * (COARSE_NB + kl) <= 2 * BAND_BUF)
    coarse_solve_blocked(AB, a.cs.binv + a.cs.binv_off[ii], nc, kl, ku, S.yb, S.buf);
  else
    band::coarse_solve(AB, ipiv, nc, kl, ku, S.yb, S.buf, S.pbuf, BAND_BUF);
  for (int k = threadIdx.x; k < nc; k += NT) {
    S.ecs[perm[k]] = S.yb[k];
    a.csol[co + perm[k]] = S.yb[k];
  }
  __syncthreads();
  mark(cyc, 2);
  // dp1 = P e_c (arithmetic T, stored FP64); base + dp1 in level order
  double* xlev = a.xlev;
  for (int i0 = ro + threadIdx.x; i0 < ro + n; i0 += ROWS_ILP * NT) {
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * NT;
      if (i < ro + n) {
        T s = 0;
        for (int p = a.p_ptr[i]; p < a.p_ptr[i + 1]; ++p) s += (T)pv[p] * (T)S.ecs[a.p_col[p]];
        dp[i] = (double)s;
        xlev[a.pk_pos[i]] = (base ? base[i] : 0.0) + (double)s;
      }
    }
  }
  __syncthreads();
  // step 6: r1 = r - A dp1 in FP64 (the difference of two nearly equal
  // vectors), stored in y (natural order) and ylev (level order) in T
  rows_residual<T>(a, ro, n, r, dp, y, false, ylev);
  __syncthreads();
  mark(cyc, 3);
  // step 7, L sweep: y_i = r1_i - sum_{j<i} L_ij y_j, by level position t.
  // Results also go to a shared-memory ring of the last SWEEP_RING
  // positions: a neighbour from a recent level is read there, older ones
  // from ylev.  The current level writes positions [lp[l], lp[l+1]), so a
  // position tc is still in the ring while tc >= lp[l+1] - SWEEP_RING.
  // Rows are staged STAGE_D - 1 levels ahead (stage_rows); the staging and
  // the ring use the band buffer, idle during the sweeps.
  // Pass 1 (instances with the sub-block smoothing stage): the same sweeps
  // with the media blocks' factors on r2 = r - A (dp1 + dp2), added to out.
  T* ring = reinterpret_cast<T*>(S.buf);
  const Stage<T> sg = stage_of<T>(S.buf);
  const int tid = threadIdx.x;
  const int npass = I.subblock ? 2 : 1;
  for (int pass = 0; pass < npass; ++pass) {
    if (pass == 1) {
      for (int i = ro + tid; i < ro + n; i += NT) dp[i] += y[i];
      __syncthreads();
      rows_residual<T>(a, ro, n, r, dp, y, false, ylev);
      __syncthreads();
    }
    const T* Fs = Prec<T>::F(a, pass);
    const T* uds = Prec<T>::ud(a, pass);
    // level bounds in registers: lw[k] = lp[l + k] (clamped to lp[nlev]),
    // the next one loaded a level ahead
    int lw[STAGE_D + 1];
#pragma unroll
    for (int k = 0; k <= STAGE_D; ++k) lw[k] = lp[min(k, nlev)];
#pragma unroll
    for (int j = 0; j < STAGE_D - 1; ++j) stage_rows<T, true>(a, lw[j], lw[j + 1], pass, sg, j);
    for (int l = 0; l < nlev; ++l) {
      const int lnext = lp[min(l + STAGE_D + 1, nlev)];
      stage_rows<T, true>(a, lw[STAGE_D - 1], lw[STAGE_D], pass, sg, (l + STAGE_D - 1) % STAGE_D);
      cp_wait<STAGE_D - 1>();
      const int lo = lw[0], hi = lw[1];
      const int lim = hi - SWEEP_RING;
      auto yv = [&](int tc) { return tc >= lim ? ring[tc & (SWEEP_RING - 1)] : ylev[tc]; };
      if (tid < STAGE_W) {
        const int t = lo + tid;
        if (t < hi) {
          const int sl = (l % STAGE_D) * STAGE_W + tid;
          const int cnt = sg.c[PK * STAGE_SLOTS + sl];
          T s = sg.v[PK * STAGE_SLOTS + sl];
#pragma unroll
          for (int k = 0; k < PK; ++k)
            if (k < cnt) s -= sg.v[k * STAGE_SLOTS + sl] * yv(sg.c[k * STAGE_SLOTS + sl]);
          if (cnt > PK) {
            const int p0 = sg.c[(PK + 1) * STAGE_SLOTS + sl];
            for (int p = p0 + PK; p < p0 + cnt; ++p) s -= Fs[p] * yv(a.pk_pos[a.col[p]]);
          }
          ring[t & (SWEEP_RING - 1)] = s;
          ylev[t] = s;
        }
      } else {
        for (int t = lo + tid; t < hi; t += NT - STAGE_W) {
          int i = a.lev_rows[t];
          T s = ylev[t];
          for (int p = a.rowptr[i]; p < a.diag[i]; ++p) s -= Fs[p] * yv(a.pk_pos[a.col[p]]);
          ring[t & (SWEEP_RING - 1)] = s;
          ylev[t] = s;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < STAGE_D; ++k) lw[k] = lw[k + 1];
      lw[STAGE_D] = lnext;
    }
    mark(cyc, 4);
    // U sweep and step 8: out = xlev + dp2 with xlev = base + dp1 (pass 1:
    // xlev = pass 0's output).  The ring now holds the upper neighbours,
    // valid while tc < lp[l] + SWEEP_RING.  Iteration j = nlev - 1 - l uses
    // stage j % STAGE_D.
    const bool keep = pass + 1 < npass;   // pass 0's output is pass 1's xlev
    // uw[k] = lp[l + 1 - k] (clamped to lp[0]) for the current level l
    int uw[STAGE_D + 1];
#pragma unroll
    for (int k = 0; k <= STAGE_D; ++k) uw[k] = lp[max(nlev - k, 0)];
#pragma unroll
    for (int j = 0; j < STAGE_D - 1; ++j) stage_rows<T, false>(a, uw[j + 1], uw[j], pass, sg, j);
    for (int l = nlev - 1, j = 0; l >= 0; --l, ++j) {
      const int unext = lp[max(l - STAGE_D, 0)];
      stage_rows<T, false>(a, uw[STAGE_D], uw[STAGE_D - 1], pass, sg, (j + STAGE_D - 1) % STAGE_D);
      cp_wait<STAGE_D - 1>();
      const int lo = uw[1], hi = uw[0];
      const int lim = lo + SWEEP_RING;
      auto yv = [&](int tc) { return tc < lim ? ring[tc & (SWEEP_RING - 1)] : ylev[tc]; };
      if (tid < STAGE_W) {
        const int t = lo + tid;
        if (t < hi) {
          const int sl = (j % STAGE_D) * STAGE_W + tid;
          const int cnt = sg.c[PK * STAGE_SLOTS + sl];
          const int i = sg.c[(PK + 1) * STAGE_SLOTS + sl];
          T s = sg.v[PK * STAGE_SLOTS + sl];
#pragma unroll
          for (int k = 0; k < PK; ++k)
            if (k < cnt) s -= sg.v[k * STAGE_SLOTS + sl] * yv(sg.c[k * STAGE_SLOTS + sl]);
          if (cnt > PK) {
            const int d = a.diag[i];
            for (int p = d + 1 + PK; p <= d + cnt; ++p) s -= Fs[p] * yv(a.pk_pos[a.col[p]]);
          }
          const T xi = s * sg.v[(PK + 1) * STAGE_SLOTS + sl];   // reciprocal of U's diagonal
          const double o = sg.x[sl] + (double)xi;
          ring[t & (SWEEP_RING - 1)] = xi;
          ylev[t] = xi;
          y[i] = xi;
          out[i] = o;
          if (keep) xlev[t] = o;
        }
      } else {
        for (int t = lo + tid; t < hi; t += NT - STAGE_W) {
          int i = a.lev_rows[t];
          int d = a.diag[i];
          T s = ylev[t];
          for (int p = d + 1; p < a.rowptr[i + 1]; ++p) s -= Fs[p] * yv(a.pk_pos[a.col[p]]);
          const T xi = s * uds[t];
          const double o = xlev[t] + (double)xi;
          ring[t & (SWEEP_RING - 1)] = xi;
          ylev[t] = xi;
          y[i] = xi;
          out[i] = o;
          if (keep) xlev[t] = o;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < STAGE_D; ++k) uw[k] = uw[k + 1];
      uw[STAGE_D] = unext;
    }
  }
  mark(cyc, 5);
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

// The Table 1 loop.  FP64: every step in FP64.  Mixed precision: the
// residual and the iterate stay FP64, the two-stage step runs on the residual
// rounded to FP32 with the FP32 copies of P, A and the ILU(0) factors (the
// coarse solve stays FP64), and its correction is added to the FP64 iterate
// -- iterative refinement with the two-stage step as the inner solver.  A
// sweep that does not reduce the FP64 residual switches the instance to FP64
// sweeps for the rest of the solve.
__global__ void __launch_bounds__(SOLVE_T, 2) k_solve(SolveArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ int s_done;
  __shared__ int pbuf[2 * band::CH_MAX];
  int ii = blockIdx.x;
  const Inst& I = a.inst[ii];
  if (I.krylov != FAMS_KRYLOV_NONE || (a.active && !a.active[ii])) return;
  const int n = I.n, ro = I.row_off;
  const SolveSmem S = solve_smem(sm, I.nc, pbuf);
  const int NT = blockDim.x;
  bool use32 = I.precision == FAMS_MIXED;
  // ||q||
  double acc = 0.0;
  for (int i = ro + threadIdx.x; i < ro + n; i += NT) acc += a.q[i] * a.q[i];
  double qn = sqrt(block_sum(acc, red));
  if (!(qn > 0.0)) qn = 1.0;
  int it = 0;
  double rel = 0.0, prev = INFINITY;
  // SM cycles per phase (thread 0, between barriers): residual, restriction,
  // band solve, prolongation + r1, L sweep, U sweep
  __shared__ long long cyc[NCYC];
  if (threadIdx.x < NCYC) cyc[threadIdx.x] = 0;
  __syncthreads();
  for (;;) {
    stamp(cyc);
    // step 3: r = q - A p (FP64)
    acc = rows_residual<double>(a, ro, n, a.q, a.x, a.r, true);
    rel = sqrt(block_sum(acc, red)) / qn;
    if (use32 && !(rel < prev)) use32 = false;   // FP32 no longer makes progress
    prev = rel;
    if (threadIdx.x == 0) {
      a.hist[(long long)ii * a.hist_len + it] = rel;
      s_done = (rel <= a.tol || it >= I.max_iter || !isfinite(rel) || a.cs.bad[ii]);
    }
    __syncthreads();
    mark(cyc, 0);
    if (s_done) break;
    // steps 5-8: p = p + dp1 + dp2
    if (!use32)
      two_stage<double>(a, I, ii, a.r, a.dp, a.x, a.x, S, cyc);
    else
      if (I.bf16_p)
        two_stage<float, __nv_bfloat16>(a, I, ii, a.r, a.dp, a.x, a.x, S, cyc);
      else
        two_stage<float>(a, I, ii, a.r, a.dp, a.x, a.x, S, cyc);
    ++it;
  }
  write_stats(a, ii, it, rel, qn, cyc);
}

// GMRES helpers on the vectors of one instance (rows [ro, ro + n)); every
// reduction has a fixed order, so results do not depend on the batch

// y = A v (FP64); returns this thread's sum of y^2
__device__ inline double rows_apply(const SolveArgs& a, int ro, int n, const double* v, double* y) {
  const double* val = a.val;
  double acc = 0;
  const int NT = blockDim.x;
  for (int i0 = ro + threadIdx.x; i0 < ro + n; i0 += ROWS_ILP * NT) {
    int rs[ROWS_ILP], re[ROWS_ILP];
    double s[ROWS_ILP];
    int m = 0;
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * NT;
      bool ok = i < ro + n;
      rs[k] = ok ? a.rowptr[i] : 0;
      re[k] = ok ? a.rowptr[i + 1] : 0;
      s[k] = 0;
      m = max(m, re[k] - rs[k]);
    }
    for (int e = 0; e < m; ++e) {
#pragma unroll
      for (int k = 0; k < ROWS_ILP; ++k) {
        int p = rs[k] + e;
        if (p < re[k]) s[k] += val[p] * v[a.col[p]];
      }
    }
#pragma unroll
    for (int k = 0; k < ROWS_ILP; ++k) {
      int i = i0 + k * NT;
      if (i < ro + n) {
        y[i] = s[k];
        acc += s[k] * s[k];
      }
    }
  }
  return acc;
}

constexpr double MIXED_MIN_GAIN = 0.1;   // FP32 cycle: least FP64 residual reduction kept

// shared state of one GMRES CTA
struct GmresSmem {
  double* H;     // (m+1) x m Hessenberg matrix, column k at H + k (m+1)
  double* g;     // m+1 rotated right-hand side
  double* cs;    // m Givens cosines
  double* sn;    // m Givens sines
  double* yv;    // m least-squares solution
  double* red;   // block_sum scratch
  int* done;
};

// One GMRES(m) cycle from the residual in a.r (norm beta), ending with
// x += M^-1 V y.  `it` counts preconditioner applications.
//
// mixed = true: flexible GMRES with the two-stage step's restriction,
// prolongation and ILU(0) sweeps in FP32 (two_stage<float>).  The basis V,
// w = A z, the Gram-Schmidt passes, r1 = r - A dp1 and the coarse solve stay
// FP64, and each output z_k is kept in FP64 (Z), so that A Z = V H holds in
// FP64 whatever the FP32 rounding did to the preconditioner; the cycle ends
// with x += Z y (no further preconditioner application).  Rounding z_k or r1
// to FP32 would cost the high-contrast instances their convergence: with
// k_f / k_m up to 1e8, A applied to an FP32 rounding error of z is as large
// as A z itself.
template <bool mixed>
__device__ void gmres_cycle(const SolveArgs& a, const Inst& I, int ii, double* V, double* Z,
                            double beta, double qn, int& it, const SolveSmem& S,
                            const GmresSmem& G, long long* cyc) {
  const int n = I.n, ro = I.row_off, m = I.restart;
  const long long ld = a.ntot;
  const int NT = blockDim.x;
  // V_0 = r / beta, g = beta e_1
  stamp(cyc);
  for (int i = ro + threadIdx.x; i < ro + n; i += NT) V[i] = a.r[i] / beta;
  for (int k = threadIdx.x; k <= m; k += NT) G.g[k] = k == 0 ? beta : 0.0;
  __syncthreads();
  mark(cyc, 0);
  int k = 0;
  for (;;) {
    // z = M^-1 V_k, w = A z (in V_{k+1})
    double* Vk = V + (long long)k * ld;
    double* w = V + (long long)(k + 1) * ld;
    double acc;
    if constexpr (mixed) {
      double* Zk = Z + (long long)k * ld;
      if (I.bf16_p)
        two_stage<float, __nv_bfloat16>(a, I, ii, Vk, a.dp, Zk, nullptr, S, cyc);
      else
        two_stage<float>(a, I, ii, Vk, a.dp, Zk, nullptr, S, cyc);
      stamp(cyc);
      acc = rows_apply(a, ro, n, Zk, w);
    } else {
      two_stage<double>(a, I, ii, Vk, a.dp, a.r, nullptr, S, cyc);
      stamp(cyc);
      acc = rows_apply(a, ro, n, a.r, w);
    }
    (void)acc;
    // modified Gram-Schmidt, as in the oracle: for i = 0..k, h_i = V_i . w,
    // then w -= h_i V_i.  Pass i applies the previous projection and forms
    // the next dot product in one sweep over the rows, so each step costs
    // 2 (k+1) n FMAs and k + 2 block reductions.
    double* Hk = G.H + (long long)k * (m + 1);
    double hprev = 0.0;
    for (int i = 0; i <= k + 1; ++i) {
      const double* Vp = i > 0 ? V + (long long)(i - 1) * ld : nullptr;
      const double* Vi = i <= k ? V + (long long)i * ld : nullptr;
      // ROWS_ILP rows per thread in flight: all loads first (the compiler
      // cannot prove that w does not alias the basis vectors, so it would not
      // move a row's loads above the previous row's store), then the
      // arithmetic in the same row order as one row at a time
      double s = 0.0;
      for (int r0 = ro + threadIdx.x; r0 < ro + n; r0 += ROWS_ILP * NT) {
        double wv[ROWS_ILP], pv[ROWS_ILP], iv[ROWS_ILP];
#pragma unroll
        for (int u = 0; u < ROWS_ILP; ++u) {
          const int r = r0 + u * NT;
          const bool ok = r < ro + n;
          wv[u] = ok ? w[r] : 0.0;
          pv[u] = ok && Vp ? Vp[r] : 0.0;
          iv[u] = ok && Vi ? Vi[r] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < ROWS_ILP; ++u) {
          const int r = r0 + u * NT;
          if (r < ro + n) {
            double wr = wv[u];
            if (Vp) {
              wr -= hprev * pv[u];
              w[r] = wr;
            }
            s += Vi ? iv[u] * wr : wr * wr;
          }
        }
      }
      double h = block_sum(s, G.red);
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
      for (int i = ro + threadIdx.x; i < ro + n; i += NT) w[i] *= inv;
    }
    __syncthreads();
    // Givens rotations on column k and the right-hand side g
    if (threadIdx.x == 0) {
      Hk[k + 1] = hn;
      for (int i = 0; i < k; ++i) {
        double t = G.cs[i] * Hk[i] + G.sn[i] * Hk[i + 1];
        Hk[i + 1] = -G.sn[i] * Hk[i] + G.cs[i] * Hk[i + 1];
        Hk[i] = t;
      }
      double d = hypot(Hk[k], Hk[k + 1]);
      G.cs[k] = Hk[k] / d;
      G.sn[k] = Hk[k + 1] / d;
      Hk[k] = d;
      Hk[k + 1] = 0.0;
      G.g[k + 1] = -G.sn[k] * G.g[k];
      G.g[k] = G.cs[k] * G.g[k];
      double est = fabs(G.g[k + 1]) / qn;
      a.hist[(long long)ii * a.hist_len + it + 1] = est;
      *G.done = (est <= a.tol || k + 1 >= m || it + 1 >= I.max_iter || !isfinite(est));
    }
    __syncthreads();
    mark(cyc, 0);
    ++k;
    ++it;
    if (*G.done) break;
  }
  // y = H^-1 g (upper triangular k x k)
  stamp(cyc);
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = G.g[i];
      for (int j = i + 1; j < k; ++j) s -= G.H[(long long)j * (m + 1) + i] * G.yv[j];
      G.yv[i] = s / G.H[(long long)i * (m + 1) + i];
    }
  }
  __syncthreads();
  if constexpr (mixed) {
    // x += Z y
    for (int i = ro + threadIdx.x; i < ro + n; i += NT) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += G.yv[j] * Z[(long long)j * ld + i];
      a.x[i] += s;
    }
    __syncthreads();
    mark(cyc, 0);
  } else {
    // u = V y (in V_k), x += M^-1 u
    double* u = V + (long long)k * ld;
    for (int i = ro + threadIdx.x; i < ro + n; i += NT) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += G.yv[j] * V[(long long)j * ld + i];
      u[i] = s;
    }
    __syncthreads();
    mark(cyc, 0);
    two_stage<double>(a, I, ii, u, a.dp, a.x, a.x, S, cyc);
  }
}

// GMRES(m) with the two-stage step as right preconditioner (Sec. 4.5, 4.6;
// Saad's right-preconditioned GMRES, Givens rotations).  The Arnoldi vectors
// are orthogonalised by modified Gram-Schmidt, each projection fused with
// the next dot product in one pass over the rows.  Iterations count preconditioner applications; the history
// holds the least-squares residual estimate inside a cycle and the true
// residual at each cycle's end.
//
// Mixed precision: flexible GMRES with the two-stage step in FP32 (see
// gmres_cycle).  A cycle that does not cut the FP64 residual by
// MIXED_MIN_GAIN marks FP32 as too coarse for this instance: the cycle is
// undone if the residual grew, and the instance continues with the FP64
// two-stage step.
__global__ void __launch_bounds__(SOLVE_T, 2) k_gmres(SolveArgs a, double* kry, double* kryz) {
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ int s_done;
  __shared__ int pbuf[2 * band::CH_MAX];
  int ii = blockIdx.x;
  const Inst& I = a.inst[ii];
  if (I.krylov != FAMS_KRYLOV_GMRES || (a.active && !a.active[ii])) return;
  const int n = I.n, ro = I.row_off, m = I.restart;
  const SolveSmem S = solve_smem(sm, I.nc, pbuf);
  GmresSmem G;
  G.H = sm + 2 * I.nc + BUF_DOUBLES;
  G.g = G.H + (m + 1) * m;
  G.cs = G.g + (m + 1);
  G.sn = G.cs + m;
  G.yv = G.sn + m;
  G.red = red;
  G.done = &s_done;
  const int NT = blockDim.x;
  bool use32 = I.precision == FAMS_MIXED;
  double acc = 0.0;
  for (int i = ro + threadIdx.x; i < ro + n; i += NT) acc += a.q[i] * a.q[i];
  double qn = sqrt(block_sum(acc, red));
  if (!(qn > 0.0)) qn = 1.0;
  __shared__ long long cyc[NCYC];
  if (threadIdx.x < NCYC) cyc[threadIdx.x] = 0;
  __syncthreads();
  stamp(cyc);
  int it = 0;
  acc = rows_residual<double>(a, ro, n, a.q, a.x, a.r, true);
  double beta = sqrt(block_sum(acc, red));
  double rel = beta / qn;
  if (threadIdx.x == 0) a.hist[(long long)ii * a.hist_len] = rel;
  mark(cyc, 0);
  for (;;) {
    if (threadIdx.x == 0)
      s_done = (rel <= a.tol || it >= I.max_iter || !isfinite(rel) || a.cs.bad[ii] || !(beta > 0.0));
    __syncthreads();
    if (s_done) break;
    if (use32) {
      for (int i = ro + threadIdx.x; i < ro + n; i += NT) a.xs[i] = a.x[i];
      __syncthreads();
      gmres_cycle<true>(a, I, ii, kry, kryz, beta, qn, it, S, G, cyc);
    } else {
      gmres_cycle<false>(a, I, ii, kry, nullptr, beta, qn, it, S, G, cyc);
    }
    stamp(cyc);
    acc = rows_residual<double>(a, ro, n, a.q, a.x, a.r, true);
    double beta1 = sqrt(block_sum(acc, red));
    if (use32 && !(beta1 <= MIXED_MIN_GAIN * beta)) {
      use32 = false;
      if (!(beta1 < beta)) {   // undo the cycle
        for (int i = ro + threadIdx.x; i < ro + n; i += NT) a.x[i] = a.xs[i];
        __syncthreads();
        acc = rows_residual<double>(a, ro, n, a.q, a.x, a.r, true);
        beta1 = sqrt(block_sum(acc, red));
      }
    }
    beta = beta1;
    rel = beta / qn;
    if (threadIdx.x == 0) a.hist[(long long)ii * a.hist_len + it] = rel;
    mark(cyc, 0);
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
  // GMRES bases: (restart + 1) vectors V indexed like the batch rows, and for
  // the mixed-precision instances the restart vectors Z of flexible GMRES
  int mr = 0, mrz = 0;
  bool mixed = false;
  for (auto& I : b.h) {
    bool m32 = I.precision == FAMS_MIXED;
    mixed |= m32;
    mr = std::max(mr, I.restart);
    if (m32 && I.krylov == FAMS_KRYLOV_GMRES) mrz = std::max(mrz, I.restart);
  }
  if (mr > 0)
    FAMS_TRY(b.alloc((void**)&b.krylov, sizeof(double) * (size_t)(mr + 1) * (size_t)(n + 1)));
  if (mrz > 0)
    FAMS_TRY(b.alloc((void**)&b.krylov_z, sizeof(double) * (size_t)mrz * (size_t)(n + 1)));
  if (mixed) {
    const long long n1 = n + 1, nnz = b.tot_nnz, pn = b.tot_pnnz;
    FAMS_TRY(b.alloc((void**)&b.ilu32, sizeof(float) * (nnz + 1)));
    FAMS_TRY(b.alloc((void**)&b.p_val32, sizeof(float) * (pn + 1)));
    FAMS_TRY(b.alloc((void**)&b.pt_val32, sizeof(float) * (pn + 1)));
    bool bf = false;
    for (auto& I : b.h) bf = bf || I.bf16_p;
    if (bf) {
      FAMS_TRY(b.alloc((void**)&b.p_val16, sizeof(unsigned short) * (pn + 1)));
      FAMS_TRY(b.alloc((void**)&b.pt_val16, sizeof(unsigned short) * (pn + 1)));
    }
    FAMS_TRY(b.alloc((void**)&b.pk_lv32, sizeof(float) * PK * n1));
    FAMS_TRY(b.alloc((void**)&b.pk_uv32, sizeof(float) * PK * n1));
    FAMS_TRY(b.alloc((void**)&b.pk_ud32, sizeof(float) * n1));
    for (float** v : {&b.yf, &b.ylevf})
      FAMS_TRY(b.alloc((void**)v, sizeof(float) * n1));
    FAMS_TRY(b.alloc((void**)&b.xs, sizeof(double) * n1));
    auto round = [&](const double* src, float* dst, long long cnt) {
      if (cnt > 0) fams::note_launch(), k_round<<<grid_for(cnt, 256), 256, 0, b.stream>>>(cnt, src, dst);
    };
    round(b.ilu, b.ilu32, nnz);
    round(b.p_val, b.p_val32, pn);
    round(b.pt_val, b.pt_val32, pn);
    if (b.p_val16 && pn > 0) {
      fams::note_launch(), k_round_bf16<<<grid_for(pn, 256), 256, 0, b.stream>>>(
          pn, b.p_val, reinterpret_cast<__nv_bfloat16*>(b.p_val16));
      fams::note_launch(), k_round_bf16<<<grid_for(pn, 256), 256, 0, b.stream>>>(
          pn, b.pt_val, reinterpret_cast<__nv_bfloat16*>(b.pt_val16));
    }
    round(b.pk_lv, b.pk_lv32, PK * n1);
    round(b.pk_uv, b.pk_uv32, PK * n1);
    round(b.pk_ud, b.pk_ud32, n1);
    FAMS_CUDA(cudaGetLastError());
  }
  return FAMS_OK;
}

// FP32 copies of the operators after their FP64 values changed
int refresh_mixed(Batch& b) {
  if (!b.ilu32) return FAMS_OK;
  const long long n1 = b.tot_row + 1, nnz = b.tot_nnz;
  auto round = [&](const double* src, float* dst, long long cnt) {
    if (cnt > 0) fams::note_launch(), k_round<<<grid_for(cnt, 256), 256, 0, b.stream>>>(cnt, src, dst);
  };
  round(b.ilu, b.ilu32, nnz);
  round(b.pk_lv, b.pk_lv32, PK * n1);
  round(b.pk_uv, b.pk_uv32, PK * n1);
  round(b.pk_ud, b.pk_ud32, n1);
  round(b.p_val, b.p_val32, b.tot_pnnz);
  round(b.pt_val, b.pt_val32, b.tot_pnnz);
  if (b.p_val16 && b.tot_pnnz > 0) {
    fams::note_launch(), k_round_bf16<<<grid_for(b.tot_pnnz, 256), 256, 0, b.stream>>>(
        b.tot_pnnz, b.p_val, reinterpret_cast<__nv_bfloat16*>(b.p_val16));
    fams::note_launch(), k_round_bf16<<<grid_for(b.tot_pnnz, 256), 256, 0, b.stream>>>(
        b.tot_pnnz, b.pt_val, reinterpret_cast<__nv_bfloat16*>(b.pt_val16));
  }
  FAMS_CUDA(cudaGetLastError());
  return FAMS_OK;
}

int make_q(Batch& b, const double* rhs_dev) {
  long long n = b.tot_row;
  fams::note_launch(), k_make_q<<<grid_for(n, 256), 256, 0, b.stream>>>(n, rhs_dev, b.qD, b.q);
  FAMS_CUDA(cudaGetLastError());
  return FAMS_OK;
}

// whether the one-CTA iteration kernels hold a coarse system of nc unknowns
// and band kl + ku + 1 (the band chunks and the coarse vectors in shared
// memory), for an instance of GMRES restart m (0: the Table 1 loop)
bool one_cta_fits(const Batch& b, int nc, int kl, int ku, int m) {
  if (kl + ku + 1 > BAND_BUF) return false;
  size_t smem = sizeof(double) * (2 * (size_t)nc + BUF_DOUBLES);
  if (m > 0) smem += sizeof(double) * ((size_t)m * m + 5 * (size_t)m + 1);
  int max_smem = 0;
  if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device) !=
      cudaSuccess)
    return true;   // (the launch reports it)
  return (long long)smem + 3072 <= max_smem;
}

int run_solve(Batch& b, double tol, float* ms, const int* active) {
  if (solve_on_grid(b)) return run_solve_grid(b, tol, ms);
  SolveArgs a{};
  a.inst = b.d_inst;
  a.active = active;
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
  a.Fb = b.ilu_b; a.pk_lvb = b.pk_lv_b; a.pk_uvb = b.pk_uv_b; a.pk_udb = b.pk_ud_b;
  a.ylev = b.ylev; a.xlev = b.xlev;
  a.ntot = b.tot_row;
  a.tol = tol;
  a.p_val32 = b.p_val32; a.pt_val32 = b.pt_val32; a.F32 = b.ilu32;
  a.p_val16 = reinterpret_cast<const __nv_bfloat16*>(b.p_val16);
  a.pt_val16 = reinterpret_cast<const __nv_bfloat16*>(b.pt_val16);
  a.pk_lv32 = b.pk_lv32; a.pk_uv32 = b.pk_uv32; a.pk_ud32 = b.pk_ud32;
  a.xs = b.xs; a.yf = b.yf; a.ylevf = b.ylevf;
  int maxnc = 0;
  for (auto& I : b.h) maxnc = std::max(maxnc, I.nc);
  for (int i = 0; i < b.B; ++i)
    if (b.csh[0].kl[i] + b.csh[0].ku[i] + 1 > BAND_BUF) {
      set_error("coarse band wider than the staged band buffer");
      return FAMS_ECAPACITY;
    }
  size_t smem = sizeof(double) * (2 * (size_t)maxnc + BUF_DOUBLES);
  int mr = 0, nrich = 0, ngm = 0;
  for (auto& I : b.h) {
    mr = std::max(mr, I.restart);
    (I.krylov == FAMS_KRYLOV_NONE ? nrich : ngm)++;
  }
  size_t smem_g = smem + sizeof(double) * ((size_t)mr * mr + 5 * (size_t)mr + 1);
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  if ((long long)(mr > 0 ? smem_g : smem) + 3072 > max_smem) {
    set_error("coarse system too large for the shared-memory coarse solve");
    return FAMS_ECAPACITY;
  }
  for (const void* k : {(const void*)k_solve, (const void*)k_gmres})
    FAMS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 3072));
  cudaEvent_t e0, e1;
  FAMS_CUDA(cudaEventCreate(&e0));
  FAMS_CUDA(cudaEventCreate(&e1));
  FAMS_CUDA(cudaEventRecord(e0, b.stream));
  // each kernel leaves the other kind of instance alone
  if (nrich > 0) fams::note_launch(), k_solve<<<b.B, SOLVE_T, smem, b.stream>>>(a);
  if (ngm > 0)
    fams::note_launch(), k_gmres<<<b.B, SOLVE_T, smem_g, b.stream>>>(a, b.krylov, b.krylov_z);
  FAMS_CUDA(cudaGetLastError());
  FAMS_CUDA(cudaEventRecord(e1, b.stream));
  if (b.prepare_flux) FAMS_TRY(flux_beside(b, e0));
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
//   q, x, r, dp, y, ylev, xlev   STATIC_ROWS each
//   crhs, csol             STATIC_COARSE each
//   stat                   STATIC_STAT (STAT_W used)
//   hist                   STATIC_HIST
namespace {
constexpr long long STATIC_ROWS = FAMS_STATIC_MAX_ROWS;
constexpr long long STATIC_COARSE = FAMS_STATIC_MAX_COARSE;
constexpr long long STATIC_STAT = 32;
constexpr long long STATIC_HIST = (long long)FAMS_STATIC_MAX_ITER + 1;
constexpr long long STATIC_DOUBLES = 7 * STATIC_ROWS + 2 * STATIC_COARSE + STATIC_STAT + STATIC_HIST;
static_assert(STATIC_ROWS % 32 == 0 && STATIC_COARSE % 32 == 0 && STATIC_STAT % 32 == 0,
              "parts of the static work array must stay 256-byte aligned");
static_assert(STATIC_STAT >= STAT_W, "status words do not fit");
}  // namespace

// In host code this name only stands for the device array: its device address
// comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_solve_static_work[STATIC_DOUBLES];

namespace {
// device address of the work array in the current device's context, looked
// up on every call (a cheap host query): a cached address would go stale when
// the context is recreated (cudaDeviceReset) and the module loads elsewhere
int static_work(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_solve_static_work);
  if (e != cudaSuccess || !p) {
    set_error(std::string("cudaGetSymbolAddress of the static work array: ") +
              cudaGetErrorString(e));
    return FAMS_ECUDA;
  }
  *out = static_cast<double*>(p);
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
  size_t smem = sizeof(double) * (2 * (size_t)I.nc + BUF_DOUBLES);
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  if ((long long)smem + 3072 > max_smem) {
    set_error("coarse system too large for the shared-memory coarse solve");
    return FAMS_ECAPACITY;
  }
  double* w = nullptr;
  FAMS_TRY(static_work(&w));
  double* q = w;
  double* xs = w + STATIC_ROWS;
  double* dp = w + 3 * STATIC_ROWS;
  double* stat = w + 7 * STATIC_ROWS + 2 * STATIC_COARSE;

  SolveArgs a{};
  a.inst = b.d_inst;
  a.cs = b.cs[0];
  a.rowptr = b.rowptr; a.col = b.col; a.val = b.val; a.diag = b.diag;
  a.p_ptr = b.p_ptr; a.p_col = b.p_col; a.p_val = b.p_val;
  a.pt_ptr = b.pt_ptr; a.pt_col = b.pt_col; a.pt_val = b.pt_val;
  a.blk_ptr = b.blk_ptr; a.blk_cell = b.blk_cell;
  a.F = b.ilu; a.lev_off = b.lev_off; a.lev_ptr = b.lev_ptr; a.lev_rows = b.lev_rows;
  a.q = q; a.x = xs; a.r = w + 2 * STATIC_ROWS; a.dp = dp; a.y = w + 4 * STATIC_ROWS;
  a.ylev = w + 5 * STATIC_ROWS;
  a.xlev = w + 6 * STATIC_ROWS;
  a.crhs = w + 7 * STATIC_ROWS; a.csol = w + 7 * STATIC_ROWS + STATIC_COARSE;
  a.stat = stat;
  a.hist = stat + STATIC_STAT; a.hist_len = STATIC_HIST;
  a.pk_pos = b.pk_pos; a.pk_nl = b.pk_nl; a.pk_lp = b.pk_lp; a.pk_lc = b.pk_lc; a.pk_lv = b.pk_lv;
  a.pk_nu = b.pk_nu; a.pk_uc = b.pk_uc; a.pk_uv = b.pk_uv; a.pk_ud = b.pk_ud;
  a.Fb = b.ilu_b; a.pk_lvb = b.pk_lv_b; a.pk_uvb = b.pk_uv_b; a.pk_udb = b.pk_ud_b;
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
                                 max_smem - 3072));
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
