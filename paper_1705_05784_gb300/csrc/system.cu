// Fine-scale EDFM system A p = q (Sec. 2, Eqs. 1-8) in CSR with sorted
// columns: two-point matrix stencil (harmonic face transmissibilities),
// matrix-fracture connections T = CI k_m, fracture-fracture links, Dirichlet
// faces through half-cell transmissibilities, well perforations (a
// rate-controlled well is one more row with sum_i beta_i (p^w - p_i) = Q_w; a
// pressure-controlled well's perforations enter like Dirichlet half-cells).
// Row order [matrix; fracture; well].
#include <cstring>

#include "batch.cuh"

namespace fams {

namespace {

__device__ inline double face_T(double ki, double kj, double area, double h) {
  return area / (h / (2.0 * ki) + h / (2.0 * kj));
}

__global__ void k_nnc_mcell(const Inst* inst, int B, const int* off_row, long long nnc,
                            const int* nrow_m, int* mcell) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnc) return;
  int r = nrow_m[k];
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  mcell[k] = I.m_off + (r - I.row_off);
}

__global__ void k_ff_bcell(const Inst* inst, int B, const int* off_row, long long nff,
                           const int* ffb, int* bcell) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nff) return;
  int r = ffb[k];
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  bcell[k] = I.fc_off + (r - I.row_off - I.nm);
}

// perforations: global matrix cell -> global row, global rate well -> its
// row, productivity index -> beta = PI k of the cell (Sec. 2: lambda^m = k)
__global__ void k_perf_rows(const Inst* inst, int B, const int* off_m, long long np,
                            const double* perm, int* prow, int* pwrow, double* beta) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int gm = prow[k];
  const Inst& I = inst[find_segment(off_m, B + 1, gm)];
  prow[k] = I.row_off + (gm - I.m_off);
  if (pwrow[k] >= 0) pwrow[k] = I.row_off + I.nm + I.nf + (pwrow[k] - I.w_off);
  beta[k] *= perm[gm];
}

struct WellArgs {
  const int* mperf_ptr;   // null: no wells in the batch
  const int* mperf_idx;
  const int* prow;
  const int* pwrow;
  const double* beta;
  const double* bhp;
  const int* wrange;
  const double* rate;
};

__global__ void k_row_count(const Inst* inst, int B, const int* off_row, long long nrow,
                            const int* nnc_t_ptr, const int* nnc_first, const int* ffr_ptr,
                            const int* ff_first, WellArgs w, int* cnt) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  int loc = (int)(r - I.row_off);
  int c = 1;
  if (loc < I.nm) {
    int x = loc % I.nx, y = (loc / I.nx) % I.ny, z = loc / (I.nx * I.ny);
    c += (x > 0) + (x < I.nx - 1) + (y > 0) + (y < I.ny - 1);
    if (I.dim == 3) c += (z > 0) + (z < I.nz - 1);
    int gm = I.m_off + loc;
    c += nnc_t_ptr[gm + 1] - nnc_t_ptr[gm];
    if (w.mperf_ptr)
      for (int q = w.mperf_ptr[gm]; q < w.mperf_ptr[gm + 1]; ++q) c += w.pwrow[w.mperf_idx[q]] >= 0;
  } else if (loc < I.nm + I.nf) {
    int gc = I.fc_off + (loc - I.nm);
    c += nnc_first[gc + 1] - nnc_first[gc];
    c += ffr_ptr[gc + 1] - ffr_ptr[gc];
    c += ff_first[gc + 1] - ff_first[gc];
  } else {
    const int gw = I.w_off + (loc - I.nm - I.nf);
    c += w.wrange[2 * gw + 1] - w.wrange[2 * gw];
  }
  cnt[r] = c;
}

__global__ void k_row_fill(const Inst* inst, int B, const int* off_row, long long nrow,
                           const double* perm, const int* nnc_t_ptr, const int* nnc_t_fc,
                           const double* nnc_t_T, const int* nnc_first, const int* nrow_m,
                           const double* nT, const int* ffr_ptr, const int* ffr_a,
                           const double* ffr_T, const int* ff_first, const int* ffb,
                           const double* ffT, WellArgs w, const int* rowptr, int* col,
                           double* val, int* diag, double* TD, double* qD) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  int loc = (int)(r - I.row_off);
  int p = rowptr[r];
  double sumT = 0.0, td = 0.0, qd = 0.0;
  int dpos = -1;
  if (loc < I.nm) {
    int nx = I.nx, ny = I.ny, nz = I.nz;
    int x = loc % nx, y = (loc / nx) % ny, z = loc / (nx * ny);
    const double* k = perm + I.m_off;
    double ki = k[loc];
    double ax = I.dy * I.dz, ay = I.dx * I.dz, az = I.dx * I.dy;
    // columns in ascending order
    if (I.dim == 3 && z > 0) {
      double t = face_T(k[loc - nx * ny], ki, az, I.dz);
      col[p] = (int)r - nx * ny; val[p++] = -t; sumT += t;
    }
    if (y > 0) {
      double t = face_T(k[loc - nx], ki, ay, I.dy);
      col[p] = (int)r - nx; val[p++] = -t; sumT += t;
    }
    if (x > 0) {
      double t = face_T(k[loc - 1], ki, ax, I.dx);
      col[p] = (int)r - 1; val[p++] = -t; sumT += t;
    }
    dpos = p++;
    if (x < nx - 1) {
      double t = face_T(ki, k[loc + 1], ax, I.dx);
      col[p] = (int)r + 1; val[p++] = -t; sumT += t;
    }
    if (y < ny - 1) {
      double t = face_T(ki, k[loc + nx], ay, I.dy);
      col[p] = (int)r + nx; val[p++] = -t; sumT += t;
    }
    if (I.dim == 3 && z < nz - 1) {
      double t = face_T(ki, k[loc + nx * ny], az, I.dz);
      col[p] = (int)r + nx * ny; val[p++] = -t; sumT += t;
    }
    int gm = I.m_off + loc;
    for (int q = nnc_t_ptr[gm]; q < nnc_t_ptr[gm + 1]; ++q) {
      int gc = nnc_t_fc[q];
      double t = nnc_t_T[q];
      col[p] = I.row_off + I.nm + (gc - I.fc_off); val[p++] = -t; sumT += t;
    }
    // perforations: a rate well's row (after every fracture row), or a
    // pressure well's Dirichlet-like term
    if (w.mperf_ptr)
      for (int q = w.mperf_ptr[gm]; q < w.mperf_ptr[gm + 1]; ++q) {
        const int k = w.mperf_idx[q];
        const double t = w.beta[k];
        if (w.pwrow[k] >= 0) {
          col[p] = w.pwrow[k]; val[p++] = -t; sumT += t;
        } else {
          td += t;
          qd += t * w.bhp[k];
        }
      }
    // Dirichlet faces: T_D = 2 k A / h
    const int on[6] = {x == 0, x == nx - 1, y == 0, y == ny - 1, I.dim == 3 && z == 0,
                       I.dim == 3 && z == nz - 1};
    const double ar[6] = {ax, ax, ay, ay, az, az};
    const double hh[6] = {I.dx, I.dx, I.dy, I.dy, I.dz, I.dz};
    for (int f = 0; f < 6; ++f) {
      if (on[f] && ((I.bc_mask >> f) & 1)) {
        double t = 2.0 * ki * ar[f] / hh[f];
        td += t;
        qd += t * I.bc_val[f];
      }
    }
  } else if (loc < I.nm + I.nf) {
    int gc = I.fc_off + (loc - I.nm);
    for (int q = nnc_first[gc]; q < nnc_first[gc + 1]; ++q) {
      double t = nT[q];
      col[p] = nrow_m[q]; val[p++] = -t; sumT += t;
    }
    for (int q = ffr_ptr[gc]; q < ffr_ptr[gc + 1]; ++q) {
      double t = ffr_T[q];
      col[p] = I.row_off + I.nm + (ffr_a[q] - I.fc_off); val[p++] = -t; sumT += t;
    }
    dpos = p++;
    for (int q = ff_first[gc]; q < ff_first[gc + 1]; ++q) {
      double t = ffT[q];
      col[p] = ffb[q]; val[p++] = -t; sumT += t;
    }
  } else {
    // a rate-controlled well: its perforated cells (ascending), then the
    // diagonal; its total rate is the row's source
    const int gw = I.w_off + (loc - I.nm - I.nf);
    for (int k = w.wrange[2 * gw]; k < w.wrange[2 * gw + 1]; ++k) {
      const double t = w.beta[k];
      col[p] = w.prow[k]; val[p++] = -t; sumT += t;
    }
    dpos = p++;
    qd = w.rate[gw];
  }
  col[dpos] = (int)r;
  val[dpos] = sumT + td;
  diag[r] = dpos;
  TD[r] = td;
  qD[r] = qd;
}

// time-step update (the harmonic mean of the two cells' mobility scales on
// every connection, the cell's scale on a Dirichlet half-cell): the rows of A
// and their Dirichlet terms, with q keeping its sources
__device__ inline double hmean(double a, double b) { return 2.0 * a * b / (a + b); }

__global__ void k_update_rows(long long nrow, const int* rowptr, const int* col, const int* diag,
                              const double* val0, const double* TD0, const double* qD0,
                              const double* mob, double* val, double* TD, double* qD, double* q) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const double sr = mob[r];
  double dsum = 0.0;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
    int c = col[p];
    if (c == r) continue;
    double v = val0[p] * hmean(sr, mob[c]);
    val[p] = v;
    dsum -= v;
  }
  const double td = TD0[r] * sr, qd = qD0[r] * sr;
  val[diag[r]] = dsum + td;
  q[r] += qd - qD[r];
  TD[r] = td;
  qD[r] = qd;
}

__global__ void k_update_conn(long long nnc, const int* row_m, const int* row_f, const double* T0,
                              long long nff, const int* fa, const int* fb, const double* F0,
                              const double* mob, double* T, double* FT) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnc) T[k] = T0[k] * hmean(mob[row_m[k]], mob[row_f[k]]);
  else if (k < nnc + nff) {
    long long e = k - nnc;
    FT[e] = F0[e] * hmean(mob[fa[e]], mob[fb[e]]);
  }
}

__global__ void k_fill(long long n, double v, double* x) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

}  // namespace

// scale[i]: n_matrix + n_frac mobility scales of instance i relative to the
// setup-time values (null: 1 everywhere, i.e. back to them)
int phase_update(Batch& b, const double* const* scale) {
  const int T = 256;
  cudaStream_t st = b.stream;
  const long long n = b.tot_row, nnz = b.tot_nnz, nnc = b.tot_nnc, nff = b.tot_ff;
  auto keep = [&](double** dst, const double* src, long long cnt) -> int {
    FAMS_TRY(b.alloc((void**)dst, sizeof(double) * (cnt + 1)));
    if (cnt > 0) FAMS_CUDA(cudaMemcpyAsync(*dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
    return FAMS_OK;
  };
  if (!b.mob) {
    FAMS_TRY(b.alloc((void**)&b.mob, sizeof(double) * (n + 1)));
    FAMS_TRY(keep(&b.val0, b.val, nnz));
    FAMS_TRY(keep(&b.TD0, b.TD, n));
    FAMS_TRY(keep(&b.qD0, b.qD, n));
    FAMS_TRY(keep(&b.nnc_T0, b.nnc_T, nnc));
    FAMS_TRY(keep(&b.ff_T0, b.ff_T, nff));
  }
  if (n > 0) fams::note_launch(), k_fill<<<grid_for(n, T), T, 0, st>>>(n, 1.0, b.mob);
  for (int i = 0; i < b.B; ++i)
    if (scale && scale[i])
      FAMS_CUDA(cudaMemcpyAsync(b.mob + b.h[i].row_off, scale[i],
                                sizeof(double) * (b.h[i].nm + b.h[i].nf), cudaMemcpyDefault, st));
  if (n > 0)
    fams::note_launch(), k_update_rows<<<grid_for(n, T), T, 0, st>>>(
        n, b.rowptr, b.col, b.diag, b.val0, b.TD0, b.qD0, b.mob, b.val, b.TD, b.qD, b.q);
  if (nnc + nff > 0)
    fams::note_launch(), k_update_conn<<<grid_for(nnc + nff, T), T, 0, st>>>(
        nnc, b.nnc_row_m, b.nnc_row_f, b.nnc_T0, nff, b.ff_a, b.ff_b, b.ff_T0, b.mob, b.nnc_T,
        b.ff_T);
  FAMS_CUDA(cudaGetLastError());
  // P stays; R A P, its factors, ILU(0) and the FP32 copies follow A
  FAMS_TRY(build_coarse_system(b, b.cs[0], -1, b.csh[0], true, b.p_ptr, b.p_col, b.p_val));
  b.fv_ready = false;
  b.ainv_ready = false;
  FAMS_TRY(ilu_refactor(b));
  FAMS_TRY(refresh_mixed(b));
  FAMS_CUDA(cudaStreamSynchronize(st));
  b.free_tmp();
  return b.check_err("time-step update");
}

namespace {

void release_coarse(Batch& b, CoarseSys& cs, CoarseHost& ch) {
  b.release(cs.Ac); b.release(cs.ac_off); b.release(cs.band); b.release(cs.band_off);
  b.release(cs.kl); b.release(cs.ku); b.release(cs.ipiv); b.release(cs.perm); b.release(cs.bad);
  b.release(cs.nopiv); b.release(cs.binv); b.release(cs.binv_off);
  ch = CoarseHost{};
}

// The time-step update, then the adaptive basis update (Sec. 3.1: basis
// functions recomputed only where the fine-scale properties change beyond a
// threshold): a row is marked when its mobility scale moved by more than a
// factor 1 + eps from the scale its basis row was last computed with; the
// dual blocks holding a marked row, and those reading a row solved again in
// an earlier stage, are solved again from the updated operator; P, P^T, R A P
// and its factors follow when any block was.  ILU(0) depends on A only and
// stays as the update left it.
// adaptive update: rows whose mobility scale moved by more than a factor
// 1 + eps from the scale their basis row was last computed with (eps < 0:
// every row)
__global__ void k_mark_moved(long long n, const double* mob, const double* ref, double eps,
                             int* marked) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = mob[i], r = ref ? ref[i] : 1.0;
  marked[i] = eps < 0.0 || s > (1.0 + eps) * r || s < r / (1.0 + eps);
}

__global__ void k_ref_update(long long n, const int* rec, const double* mob, double* ref) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && rec[i]) ref[i] = mob[i];
}

__global__ void k_any(long long n, const int* v, int* out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && v[i]) *out = 1;
}

}  // namespace

int phase_update_basis(Batch& b, const double* const* scale, double eps, int* rebuilt) {
  const int T = 256;
  cudaStream_t st = b.stream;
  const long long n = b.tot_row;
  if (rebuilt) *rebuilt = 0;
  FAMS_TRY(phase_update(b, scale));
  if (n == 0) return FAMS_OK;
  if (!b.mob_basis) {   // the scales the current basis rows were computed with: the setup's
    FAMS_TRY(b.alloc((void**)&b.mob_basis, sizeof(double) * (n + 1)));
    fams::note_launch(), k_fill<<<grid_for(n, T), T, 0, st>>>(n, 1.0, b.mob_basis);
  }
  int *marked = nullptr, *rec = nullptr, *any = nullptr;
  FAMS_TRY(b.scratch((void**)&marked, sizeof(int) * (n + 1)));
  FAMS_TRY(b.scratch((void**)&rec, sizeof(int) * (n + 1)));
  FAMS_TRY(b.scratch((void**)&any, sizeof(int)));
  FAMS_CUDA(cudaMemsetAsync(rec, 0, sizeof(int) * (n + 1), st));
  FAMS_CUDA(cudaMemsetAsync(any, 0, sizeof(int), st));
  fams::note_launch(), k_mark_moved<<<grid_for(n, T), T, 0, st>>>(n, b.mob, b.mob_basis, eps, marked);
  fams::note_launch(), k_any<<<grid_for(n, T), T, 0, st>>>(n, marked, any);
  int hany = 0;
  FAMS_CUDA(cudaMemcpyAsync(&hany, any, sizeof(int), cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaStreamSynchronize(st));
  if (!hany) {
    b.free_tmp();
    return FAMS_OK;
  }
  // the new P replaces the old once the stages have read the old rows
  int *op = b.p_ptr, *oc = b.p_col, *opt = b.pt_ptr, *otc = b.pt_col;
  double *ov = b.p_val, *otv = b.pt_val;
  int *ofp = b.pf_ptr, *ofc = b.pf_col;
  double* ofv = b.pf_val;
  const bool oalias = b.pf_alias;
  int solved = 0;
  FAMS_TRY(phase_basis(b, marked, rec, &solved));
  b.release(op); b.release(oc); b.release(ov);
  b.release(opt); b.release(otc); b.release(otv);
  if (!oalias) { b.release(ofp); b.release(ofc); b.release(ofv); }
  fams::note_launch(), k_ref_update<<<grid_for(n, T), T, 0, st>>>(n, rec, b.mob, b.mob_basis);
  if (solved > 0) {
    release_coarse(b, b.cs[0], b.csh[0]);
    FAMS_TRY(phase_coarse_op(b, -1));
    if (b.fv_built) release_coarse(b, b.cs[1], b.csh[1]);
    b.fv_built = false;
    b.fv_ready = false;
    b.ainv_ready = false;
    if (b.p_val32) {   // FP32 copies of P and P^T at the new size
      b.release(b.p_val32);
      b.release(b.pt_val32);
      FAMS_TRY(b.alloc((void**)&b.p_val32, sizeof(float) * (b.tot_pnnz + 1)));
      FAMS_TRY(b.alloc((void**)&b.pt_val32, sizeof(float) * (b.tot_pnnz + 1)));
      if (b.p_val16) {
        b.release(b.p_val16);
        b.release(b.pt_val16);
        FAMS_TRY(b.alloc((void**)&b.p_val16, sizeof(unsigned short) * (b.tot_pnnz + 1)));
        FAMS_TRY(b.alloc((void**)&b.pt_val16, sizeof(unsigned short) * (b.tot_pnnz + 1)));
      }
      FAMS_TRY(refresh_mixed(b));
    }
  }
  FAMS_CUDA(cudaStreamSynchronize(st));
  b.free_tmp();
  FAMS_TRY(b.check_err("basis update"));
  if (rebuilt) *rebuilt = solved;
  return FAMS_OK;
}

int phase_system(Batch& b) {
  const int T = 256;
  cudaStream_t st = b.stream;
  long long nnc = b.tot_nnc, nff = b.tot_ff, nfc = b.tot_fc, nrow = b.tot_row;
  // matrix-cell view of the matrix-fracture connections, sorted by fracture cell
  int* mcell = nullptr;
  FAMS_TRY(b.scratch((void**)&mcell, sizeof(int) * (nnc + 1)));
  if (nnc > 0)
    fams::note_launch(), k_nnc_mcell<<<grid_for(nnc, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nnc, b.nnc_row_m,
                                                mcell);
  int *nnc_t_ptr = nullptr, *nnc_t_fc = nullptr;
  double* nnc_t_T = nullptr;
  FAMS_TRY(transpose(b, b.nnc_first, mcell, b.nnc_T, (int)nfc, (int)b.tot_m, nnc, &nnc_t_ptr,
                     &nnc_t_fc, &nnc_t_T, false));
  // fracture-fracture links seen from their higher cell
  int* bcell = nullptr;
  FAMS_TRY(b.scratch((void**)&bcell, sizeof(int) * (nff + 1)));
  if (nff > 0)
    fams::note_launch(), k_ff_bcell<<<grid_for(nff, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nff, b.ff_b, bcell);
  int *ffr_ptr = nullptr, *ffr_a = nullptr;
  double* ffr_T = nullptr;
  FAMS_TRY(transpose(b, b.ff_first, bcell, b.ff_T, (int)nfc, (int)nfc, nff, &ffr_ptr, &ffr_a,
                     &ffr_T, false));
  // ffr_a: for each higher cell, the lower cells (fracture-cell index) in order
  if (b.tot_perf > 0)
    fams::note_launch(), k_perf_rows<<<grid_for(b.tot_perf, T), T, 0, st>>>(
        b.d_inst, b.B, b.off_m, b.tot_perf, b.perm, b.perf_row, b.perf_wrow, b.perf_beta);
  const WellArgs wa{b.tot_perf > 0 ? b.mperf_ptr : nullptr, b.mperf_idx, b.perf_row, b.perf_wrow,
                    b.perf_beta, b.perf_bhp, b.wperf_range, b.w_rate};
  int* cnt = nullptr;
  FAMS_TRY(b.scratch((void**)&cnt, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.alloc((void**)&b.rowptr, sizeof(int) * (nrow + 1)));
  if (nrow > 0)
    fams::note_launch(), k_row_count<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, nnc_t_ptr,
                                                 b.nnc_first, ffr_ptr, b.ff_first, wa, cnt);
  long long nnz = 0;
  FAMS_TRY(exclusive_scan(b, cnt, b.rowptr, nrow, &nnz));
  b.tot_nnz = nnz;
  FAMS_TRY(b.alloc((void**)&b.col, sizeof(int) * (nnz + 1)));
  FAMS_TRY(b.alloc((void**)&b.val, sizeof(double) * (nnz + 1)));
  FAMS_TRY(b.alloc((void**)&b.diag, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.alloc((void**)&b.TD, sizeof(double) * (nrow + 1)));
  FAMS_TRY(b.alloc((void**)&b.qD, sizeof(double) * (nrow + 1)));
  if (nrow > 0)
    fams::note_launch(), k_row_fill<<<grid_for(nrow, T), T, 0, st>>>(
        b.d_inst, b.B, b.off_row, nrow, b.perm, nnc_t_ptr, nnc_t_fc, nnc_t_T, b.nnc_first,
        b.nnc_row_m, b.nnc_T, ffr_ptr, ffr_a, ffr_T, b.ff_first, b.ff_b, b.ff_T, wa, b.rowptr,
        b.col, b.val, b.diag, b.TD, b.qD);
  FAMS_CUDA(cudaGetLastError());
  // row pointers at the instance boundaries (off_row: B + 1 row offsets)
  std::vector<int> hp;
  FAMS_TRY(take_ints(b, b.rowptr, b.off_row, b.B + 1, hp));
  for (int i = 0; i < b.B; ++i) {
    Inst& I = b.h[i];
    I.nnz_off = hp[i];
    I.nnz = hp[i + 1] - hp[i];
  }
  FAMS_TRY(b.upload_inst());
  return b.check_err("fine system");
}

}  // namespace fams
