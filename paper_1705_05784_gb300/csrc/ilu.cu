// ILU(0) smoother of the complete fine matrix (Sec. 3.2: M_S from an ILU(0)
// decomposition of A), natural order (matrix cells, then fracture cells), no
// pivoting, restricted to the pattern of A.
//
// Rows are grouped into dependency levels: a row's level is one more than the
// highest level among the rows it depends on (its strictly lower entries).
// For the natural-order stencil rows that is x + y + z; fracture rows follow
// in one sequential pass per instance.  Rows of one level are independent, so
// the factorisation and the triangular sweeps process a level in parallel and
// give the same result as the row-by-row definition.
#include <algorithm>

#include "batch.cuh"

namespace fams {

namespace {

__global__ void k_lev_matrix(const Inst* inst, int B, const int* off_row, long long nrow,
                             int* level) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  int loc = (int)(r - I.row_off);
  if (loc >= I.nm) return;
  int x = loc % I.nx, y = (loc / I.nx) % I.ny, z = loc / (I.nx * I.ny);
  level[r] = x + y + z;
}

constexpr int LEV_WIN = 8192;   // fracture rows whose levels stay in shared memory

// Fracture rows of one instance in order, one warp: lanes take a row's lower
// entries (matrix levels from the cell index, fracture levels from shared
// memory for the first LEV_WIN fracture rows), row bounds fetched 32 rows at
// a time.
__global__ void k_lev_frac(const Inst* inst, int B, const int* rowptr, const int* col,
                           const int* diag, int* level, int* nlev) {
  __shared__ int win[LEV_WIN];
  const Inst& I = inst[blockIdx.x];
  int lane = threadIdx.x;
  int mx = I.nm > 0 ? (I.nx - 1) + (I.ny - 1) + (I.dim == 3 ? I.nz - 1 : 0) : -1;
  int f0 = I.row_off + I.nm, end = I.row_off + I.n;
  for (int r0 = f0; r0 < end; r0 += 32) {
    int rr = r0 + lane;
    int ra = rr < end ? rowptr[rr] : 0, rd = rr < end ? diag[rr] : 0;
    int nr = min(32, end - r0);
    for (int j = 0; j < nr; ++j) {
      int a = __shfl_sync(0xffffffffu, ra, j), d = __shfl_sync(0xffffffffu, rd, j);
      int l = 0;
      for (int p = a + lane; p < d; p += 32) {
        int c = col[p];
        int loc = c - I.row_off, lc;
        if (loc < I.nm) {
          lc = loc % I.nx + (loc / I.nx) % I.ny + loc / (I.nx * I.ny);
        } else {
          lc = c - f0 < LEV_WIN ? win[c - f0] : level[c];
        }
        l = max(l, lc + 1);
      }
      for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, o));
      if (lane == 0) {
        level[r0 + j] = l;
        if (r0 + j - f0 < LEV_WIN) win[r0 + j - f0] = l;
      }
      __syncwarp();
      mx = max(mx, l);
    }
  }
  if (lane == 0) nlev[blockIdx.x] = mx + 1;
}

__global__ void k_lev_count(const Inst* inst, int B, const int* off_row, long long nrow,
                            const int* level, const int* lev_off, int* cnt) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  int ii = find_segment(off_row, B + 1, r);
  atomicAdd(&cnt[lev_off[ii] + level[r]], 1);
}

__global__ void k_lev_place(const Inst* inst, int B, const int* off_row, long long nrow,
                            const int* level, const int* lev_off, const int* lev_ptr, int* cursor,
                            int* rows) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  int ii = find_segment(off_row, B + 1, r);
  int s = lev_off[ii] + level[r];
  rows[lev_ptr[s] + atomicAdd(&cursor[s], 1)] = (int)r;
}

// IKJ ILU(0), one CTA per instance, level by level
__global__ void k_ilu_factor(const Inst* inst, int B, const int* rowptr, const int* col,
                             const int* diag, const int* lev_off, const int* lev_ptr,
                             const int* rows, double* F, int* err) {
  int ii = blockIdx.x;
  const Inst& I = inst[ii];
  const int* lp = lev_ptr + lev_off[ii];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int l = 0; l < I.nlev; ++l) {
    for (int t = lp[l] + threadIdx.x; t < lp[l + 1]; t += blockDim.x) {
      int i = rows[t];
      int e = rowptr[i + 1], d = diag[i];
      for (int p = rowptr[i]; p < d; ++p) {
        int k = col[p];
        double lik = F[p] / F[diag[k]];
        F[p] = lik;
        int u = p + 1;
        for (int q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
          int j = col[q];
          while (u < e && col[u] < j) ++u;
          if (u < e && col[u] == j) F[u] -= lik * F[q];
        }
      }
      double piv = F[d];
      if (!(piv != 0.0) || !isfinite(piv)) bad = 1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicCAS(err, 0, DERR_BREAKDOWN);
}

// A without its cross-medium entries (matrix, fracture and well blocks), in
// A's pattern: the sub-block smoothing stage's matrix
__global__ void k_block_vals(const Inst* inst, int B, const int* off_row, long long nrow,
                             const int* rowptr, const int* col, const double* val, double* out) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  auto med = [&](long long g) {
    const long long loc = g - I.row_off;
    return loc < I.nm ? 0 : (loc < I.nm + I.nf ? 1 : 2);
  };
  const int mr = med(r);
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) out[p] = med(col[p]) == mr ? val[p] : 0.0;
}

__global__ void k_pos(long long nrow, const int* rows, int* pos) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nrow) pos[rows[t]] = (int)t;
}

// level-ordered structure-of-arrays copy of the factors (position t); the
// first PK neighbours of each triangle are stored by their level positions,
// so the sweeps can find recent results in shared memory
__global__ void k_pack(long long nrow, const int* rows, const int* rowptr, const int* col,
                       const int* diag, const double* F, const int* pos, int* nl, int* lp, int* lc,
                       double* lv, int* nu, int* uc, double* uv, double* ud) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrow) return;
  int i = rows[t];
  int a = rowptr[i], d = diag[i], e = rowptr[i + 1];
  nl[t] = d - a;
  lp[t] = a;
  nu[t] = e - d - 1;
  ud[t] = 1.0 / F[d];   // reciprocal: the sweep multiplies
  for (int k = 0; k < PK; ++k) {
    long long o = (long long)k * nrow + t;
    lc[o] = (a + k < d) ? pos[col[a + k]] : 0;
    lv[o] = (a + k < d) ? F[a + k] : 0.0;
    uc[o] = (d + 1 + k < e) ? pos[col[d + 1 + k]] : 0;
    uv[o] = (d + 1 + k < e) ? F[d + 1 + k] : 0.0;
  }
}

}  // namespace

// the factors of the sub-block stage (when an instance asks for it): A's
// values without the cross-medium entries, factored on A's levels, packed
// beside the main factors
static int block_factors(Batch& b, bool alloc) {
  const int T = 256;
  cudaStream_t st = b.stream;
  const long long nrow = b.tot_row, n1 = nrow + 1;
  bool any = false;
  for (auto& I : b.h) any = any || I.subblock;
  if (!any) return FAMS_OK;
  if (alloc) {
    FAMS_TRY(b.alloc((void**)&b.ilu_b, sizeof(double) * (b.tot_nnz + 1)));
    FAMS_TRY(b.alloc((void**)&b.pk_lv_b, sizeof(double) * PK * n1));
    FAMS_TRY(b.alloc((void**)&b.pk_uv_b, sizeof(double) * PK * n1));
    FAMS_TRY(b.alloc((void**)&b.pk_ud_b, sizeof(double) * n1));
  }
  if (nrow == 0) return FAMS_OK;
  fams::note_launch(), k_block_vals<<<grid_for(nrow, T), T, 0, st>>>(
      b.d_inst, b.B, b.off_row, nrow, b.rowptr, b.col, b.val, b.ilu_b);
  if (whole_gpu(b)) {
    FAMS_TRY(ilu_factor_grid(b, b.ilu_b));
  } else {
    fams::note_launch(), k_ilu_factor<<<b.B, 512, 0, st>>>(b.d_inst, b.B, b.rowptr, b.col, b.diag,
                                                            b.lev_off, b.lev_ptr, b.lev_rows,
                                                            b.ilu_b, b.d_err);
  }
  FAMS_CUDA(cudaGetLastError());
  FAMS_TRY(b.check_err("ILU(0) of the media blocks"));
  fams::note_launch(), k_pack<<<grid_for(nrow, T), T, 0, st>>>(
      nrow, b.lev_rows, b.rowptr, b.col, b.diag, b.ilu_b, b.pk_pos, b.pk_nl, b.pk_lp, b.pk_lc,
      b.pk_lv_b, b.pk_nu, b.pk_uc, b.pk_uv_b, b.pk_ud_b);
  FAMS_CUDA(cudaGetLastError());
  return FAMS_OK;
}

int phase_ilu(Batch& b) {
  const int T = 256;
  cudaStream_t st = b.stream;
  long long nrow = b.tot_row;
  int B = b.B;
  int *level = nullptr, *dnlev = nullptr;
  FAMS_TRY(b.scratch((void**)&level, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&dnlev, sizeof(int) * B));
  fams::note_launch(), k_lev_matrix<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, B, b.off_row, nrow, level);
  fams::note_launch(), k_lev_frac<<<B, 32, 0, st>>>(b.d_inst, B, b.rowptr, b.col, b.diag, level, dnlev);
  std::vector<int> nlev(B);
  FAMS_CUDA(cudaMemcpyAsync(nlev.data(), dnlev, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaStreamSynchronize(st));
  std::vector<int> loff(B + 1, 0);
  for (int i = 0; i < B; ++i) {
    b.h[i].nlev = nlev[i];
    loff[i + 1] = loff[i] + nlev[i] + 1;
  }
  FAMS_TRY(b.upload_inst());
  int tl = loff[B];
  int *cnt = nullptr, *cursor = nullptr;
  FAMS_TRY(b.alloc((void**)&b.lev_off, sizeof(int) * (B + 1)));
  FAMS_TRY(b.alloc((void**)&b.lev_ptr, sizeof(int) * (tl + 1)));
  FAMS_TRY(b.alloc((void**)&b.lev_rows, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&cnt, sizeof(int) * (tl + 1)));
  FAMS_TRY(b.scratch((void**)&cursor, sizeof(int) * (tl + 1)));
  FAMS_CUDA(cudaMemcpyAsync(b.lev_off, loff.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st));
  FAMS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (tl + 1), st));
  FAMS_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (tl + 1), st));
  fams::note_launch(), k_lev_count<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, B, b.off_row, nrow, level, b.lev_off, cnt);
  FAMS_TRY(exclusive_scan(b, cnt, b.lev_ptr, tl, nullptr));
  fams::note_launch(), k_lev_place<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, B, b.off_row, nrow, level, b.lev_off,
                                               b.lev_ptr, cursor, b.lev_rows);
  // rows of a level in ascending order (independent rows: only for locality)
  FAMS_TRY(sort_segments(b, b.lev_ptr, tl, b.lev_rows, nullptr, false));
  FAMS_TRY(b.alloc((void**)&b.ilu, sizeof(double) * (b.tot_nnz + 1)));
  FAMS_CUDA(cudaMemcpyAsync(b.ilu, b.val, sizeof(double) * b.tot_nnz, cudaMemcpyDeviceToDevice, st));
  if (whole_gpu(b)) {
    FAMS_TRY(ilu_factor_grid(b, b.ilu));
  } else {
    fams::note_launch(), k_ilu_factor<<<B, 512, 0, st>>>(b.d_inst, B, b.rowptr, b.col, b.diag,
                                                          b.lev_off, b.lev_ptr, b.lev_rows, b.ilu,
                                                          b.d_err);
  }
  FAMS_CUDA(cudaGetLastError());
  FAMS_TRY(b.check_err("ILU(0)"));
  long long n1 = nrow + 1;
  FAMS_TRY(b.alloc((void**)&b.pk_pos, sizeof(int) * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_nl, sizeof(int) * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_lp, sizeof(int) * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_nu, sizeof(int) * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_lc, sizeof(int) * PK * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_uc, sizeof(int) * PK * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_lv, sizeof(double) * PK * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_uv, sizeof(double) * PK * n1));
  FAMS_TRY(b.alloc((void**)&b.pk_ud, sizeof(double) * n1));
  FAMS_TRY(b.alloc((void**)&b.ylev, sizeof(double) * n1));
  FAMS_TRY(b.alloc((void**)&b.xlev, sizeof(double) * n1));
  if (nrow > 0) {
    fams::note_launch(), k_pos<<<grid_for(nrow, T), T, 0, st>>>(nrow, b.lev_rows, b.pk_pos);
    fams::note_launch(), k_pack<<<grid_for(nrow, T), T, 0, st>>>(
        nrow, b.lev_rows, b.rowptr, b.col, b.diag, b.ilu, b.pk_pos, b.pk_nl, b.pk_lp, b.pk_lc,
        b.pk_lv, b.pk_nu, b.pk_uc, b.pk_uv, b.pk_ud);
  }
  FAMS_CUDA(cudaGetLastError());
  return block_factors(b, true);
}

// new values, same pattern and levels (a time-step update)
int ilu_refactor(Batch& b) {
  const int T = 256;
  cudaStream_t st = b.stream;
  long long nrow = b.tot_row;
  FAMS_CUDA(cudaMemcpyAsync(b.ilu, b.val, sizeof(double) * b.tot_nnz, cudaMemcpyDeviceToDevice, st));
  if (whole_gpu(b)) {
    FAMS_TRY(ilu_factor_grid(b, b.ilu));
  } else {
    fams::note_launch(), k_ilu_factor<<<b.B, 512, 0, st>>>(b.d_inst, b.B, b.rowptr, b.col, b.diag,
                                                            b.lev_off, b.lev_ptr, b.lev_rows, b.ilu,
                                                            b.d_err);
  }
  FAMS_CUDA(cudaGetLastError());
  FAMS_TRY(b.check_err("ILU(0)"));
  if (nrow > 0)
    fams::note_launch(), k_pack<<<grid_for(nrow, T), T, 0, st>>>(
        nrow, b.lev_rows, b.rowptr, b.col, b.diag, b.ilu, b.pk_pos, b.pk_nl, b.pk_lp, b.pk_lc,
        b.pk_lv, b.pk_nu, b.pk_uc, b.pk_uv, b.pk_ud);
  FAMS_CUDA(cudaGetLastError());
  return block_factors(b, false);
}

}  // namespace fams
