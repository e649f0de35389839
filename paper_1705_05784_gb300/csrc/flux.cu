// Conservative fine-scale flux reconstruction after any iterate (Sec. 1 and
// Sec. 3.2: possible after an MSFV stage).
//   1. p' = x + P (R^FV A P)^-1 R^FV (q - A x)          (one FV stage)
//   2. every connection between two primal blocks carries T (p'_i - p'_j);
//   3. each primal block solves its own TPFA problem with those fluxes as
//      Neumann data (Dirichlet faces stay Dirichlet; a block without one is
//      pinned to p' at its coarse node) -> p~;
//   4. connections inside a block carry T (p~_i - p~_j).
// R^FV (q - A p') = 0 makes every local problem consistent, so the result is
// mass conservative cell by cell.
#include <algorithm>

#include "batch.cuh"

namespace fams {

namespace {

__device__ inline double block_sum_f(double v, double* red) {
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

// step 1 for one instance (one CTA)
__global__ void k_flux_stage(const Inst* inst, int ii, CoarseSys cs, const int* rowptr,
                             const int* col, const double* val, const int* blk_ptr,
                             const int* blk_cell, const int* p_ptr, const int* p_col,
                             const double* p_val, const double* q, const double* x, double* r,
                             double* pp) {
  extern __shared__ double sm[];
  const Inst& I = inst[ii];
  int n = I.n, ro = I.row_off, nc = I.nc, co = I.nc_off;
  double* yb = sm;
  double* ecs = sm + nc;
  for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
    double s = q[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) s -= val[p] * x[col[p] - ro];
    r[i] = s;
  }
  __syncthreads();
  const int* perm = cs.perm + co;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    int c = co + perm[k];
    double s = 0.0;
    for (int p = blk_ptr[c]; p < blk_ptr[c + 1]; ++p) s += r[blk_cell[p]];
    yb[k] = s;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const double* AB = cs.band + cs.band_off[ii];
    const int* ipiv = cs.ipiv + co;
    int kl = cs.kl[ii], ku = cs.ku[ii], kv = kl + ku, ldab = 2 * kl + ku + 1;
    int lane = threadIdx.x;
    for (int j = 0; j < nc; ++j) {
      int km = min(kl, nc - 1 - j);
      int pj = ipiv[j];
      if (lane == 0 && pj != j) { double t = yb[j]; yb[j] = yb[pj]; yb[pj] = t; }
      __syncwarp();
      double yj = yb[j];
      for (int t = 1 + lane; t <= km; t += 32)
        yb[j + t] -= AB[(long long)(kv + t) + (long long)ldab * j] * yj;
      __syncwarp();
    }
    for (int j = nc - 1; j >= 0; --j) {
      double yj = yb[j] / AB[(long long)kv + (long long)ldab * j];
      __syncwarp();
      if (lane == 0) yb[j] = yj;
      for (int i = max(0, j - kv) + lane; i < j; i += 32)
        yb[i] -= AB[(long long)(kv + i - j) + (long long)ldab * j] * yj;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nc; k += blockDim.x) ecs[perm[k]] = yb[k];
  __syncthreads();
  for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
    double s = 0.0;
    for (int p = p_ptr[i]; p < p_ptr[i + 1]; ++p) s += p_val[p] * ecs[p_col[p]];
    pp[i] = x[i - ro] + s;
  }
}

// steps 2-3: one CTA per primal block, dense Gaussian elimination with
// partial pivoting on the block's local TPFA matrix
__global__ void k_flux_local(const Inst* inst, int ii, const int* blk_list, const int* blk_ptr,
                             const int* blk_cell, const int* rowptr, const int* col,
                             const double* val, const double* TD, const double* qD,
                             const double* q, const int* primal, const int* node_cell,
                             const double* pp, double* pt, double* gwork, long long gstride,
                             int* err) {
  extern __shared__ double dsm[];
  const Inst& I = inst[ii];
  int c = I.nc_off + blk_list[blockIdx.x];
  int a = blk_ptr[c], m = blk_ptr[c + 1] - a;
  double* K = gwork ? gwork + (long long)blockIdx.x * gstride : dsm;
  double* rhs = K + (long long)m * m;
  __shared__ int s_hasD, s_piv, s_bad;
  if (threadIdx.x == 0) { s_hasD = 0; s_bad = 0; }
  for (long long t = threadIdx.x; t < (long long)m * m + m; t += blockDim.x) K[t] = 0.0;
  __syncthreads();
  int myblk = c - I.nc_off;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    int i = blk_cell[a + t];
    double b = q[i];  // sources + Dirichlet terms
    double d = TD[i];
    if (TD[i] > 0.0) s_hasD = 1;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int j = col[p];
      if (j == i) continue;
      double T = -val[p];
      if (primal[j] == myblk) {
        // position of j in the sorted member list
        int lo = 0, hi = m - 1, pos = -1;
        while (lo <= hi) {
          int mid = (lo + hi) >> 1;
          int v = blk_cell[a + mid];
          if (v == j) { pos = mid; break; }
          if (v < j) lo = mid + 1; else hi = mid - 1;
        }
        if (pos < 0) { atomicCAS(err, 0, DERR_INVAL); continue; }
        K[(long long)t * m + pos] -= T;
        d += T;
      } else {
        b -= T * (pp[i] - pp[j]);
      }
    }
    K[(long long)t * m + t] += d;
    rhs[t] = b;
  }
  __syncthreads();
  if (!s_hasD && threadIdx.x == 0) {
    int v = node_cell[c];
    int lo = 0, hi = m - 1, pos = 0;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int w = blk_cell[a + mid];
      if (w == v) { pos = mid; break; }
      if (w < v) lo = mid + 1; else hi = mid - 1;
    }
    for (int j = 0; j < m; ++j) K[(long long)pos * m + j] = 0.0;
    K[(long long)pos * m + pos] = 1.0;
    rhs[pos] = pp[v];
  }
  __syncthreads();
  // Gaussian elimination with partial pivoting
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      int pr = j;
      double best = fabs(K[(long long)j * m + j]);
      for (int i = j + 1; i < m; ++i) {
        double v = fabs(K[(long long)i * m + j]);
        if (v > best) { best = v; pr = i; }
      }
      if (!(best > 0.0)) s_bad = 1;
      s_piv = pr;
    }
    __syncthreads();
    if (s_bad) break;
    int pr = s_piv;
    if (pr != j) {
      for (int t = threadIdx.x; t <= m; t += blockDim.x) {
        if (t < m) {
          double u = K[(long long)j * m + t];
          K[(long long)j * m + t] = K[(long long)pr * m + t];
          K[(long long)pr * m + t] = u;
        } else {
          double u = rhs[j]; rhs[j] = rhs[pr]; rhs[pr] = u;
        }
      }
      __syncthreads();
    }
    double piv = K[(long long)j * m + j];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
      double f = K[(long long)i * m + j] / piv;
      K[(long long)i * m + j] = f;
      for (int t = j + 1; t < m; ++t) K[(long long)i * m + t] -= f * K[(long long)j * m + t];
      rhs[i] -= f * rhs[j];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicCAS(err, 0, DERR_BREAKDOWN);
    return;
  }
  if (threadIdx.x == 0) {
    for (int j = m - 1; j >= 0; --j) {
      double s = rhs[j];
      for (int t = j + 1; t < m; ++t) s -= K[(long long)j * m + t] * rhs[t];
      rhs[j] = s / K[(long long)j * m + j];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m; t += blockDim.x) pt[blk_cell[a + t]] = rhs[t];
}

// step 4: face and connection fluxes of one instance
__global__ void k_flux_faces(const Inst* inst, int ii, const double* perm, const int* primal,
                             const double* pp, const double* pt, double* face) {
  const Inst& I = inst[ii];
  int nx = I.nx, ny = I.ny, nz = I.dim == 3 ? I.nz : 1;
  long long nfx = (long long)(nx + 1) * ny * nz, nfy = (long long)nx * (ny + 1) * nz;
  long long nfz = I.dim == 3 ? (long long)nx * ny * (nz + 1) : 0;
  long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfx + nfy + nfz) return;
  const double* k = perm + I.m_off;
  int ro = I.row_off;
  int axis, i, j, l;
  long long g = f;
  if (g < nfx) { axis = 0; i = (int)(g % (nx + 1)); j = (int)((g / (nx + 1)) % ny); l = (int)(g / ((long long)(nx + 1) * ny)); }
  else if ((g -= nfx) < nfy) { axis = 1; i = (int)(g % nx); j = (int)((g / nx) % (ny + 1)); l = (int)(g / ((long long)nx * (ny + 1))); }
  else { g -= nfy; axis = 2; i = (int)(g % nx); j = (int)((g / nx) % ny); l = (int)(g / ((long long)nx * ny)); }
  int n_ax = axis == 0 ? nx : (axis == 1 ? ny : nz);
  int c_ax = axis == 0 ? i : (axis == 1 ? j : l);
  double area = axis == 0 ? I.dy * I.dz : (axis == 1 ? I.dx * I.dz : I.dx * I.dy);
  double h = axis == 0 ? I.dx : (axis == 1 ? I.dy : I.dz);
  long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
  long long hi_cell = (long long)i + (long long)nx * (j + (long long)ny * l);
  double out = 0.0;
  if (c_ax == 0 || c_ax == n_ax) {
    int fid = 2 * axis + (c_ax == n_ax ? 1 : 0);
    if ((I.bc_mask >> fid) & 1) {
      long long cell = (c_ax == 0) ? hi_cell : hi_cell - stride;
      double TDf = 2.0 * k[cell] * area / h;
      double pc = pt[ro + cell];
      out = (c_ax == 0) ? TDf * (I.bc_val[fid] - pc) : TDf * (pc - I.bc_val[fid]);
    }
  } else {
    long long lo_cell = hi_cell - stride;
    double T = area / (h / (2.0 * k[lo_cell]) + h / (2.0 * k[hi_cell]));
    bool same = primal[ro + lo_cell] == primal[ro + hi_cell];
    const double* p = same ? pt : pp;
    out = T * (p[ro + lo_cell] - p[ro + hi_cell]);
  }
  face[f] = out;
}

__global__ void k_flux_nnc(const Inst* inst, int ii, const int* nrow_m, const int* nrow_f,
                           const double* nT, const int* ffa, const int* ffb, const double* ffT,
                           const int* primal, const double* pp, const double* pt, double* out) {
  const Inst& I = inst[ii];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < I.nnc) {
    long long k = I.nnc_off + t;
    out[t] = nT[k] * (pp[nrow_m[k]] - pp[nrow_f[k]]);
  } else if (t < (long long)I.nnc + I.nff) {
    long long k = I.ff_off + (t - I.nnc);
    int a = ffa[k], b = ffb[k];
    const double* p = primal[a] == primal[b] ? pt : pp;
    out[t] = ffT[k] * (p[a] - p[b]);
  }
}

}  // namespace

int run_flux(Batch& b, int ii, const double* x_dev, double* face, double* nnc_out) {
  cudaStream_t st = b.stream;
  bool all_fv = true;
  for (auto& I : b.h) all_fv = all_fv && I.restriction == FAMS_R_FV;
  CoarseSys* cs = &b.cs[0];
  if (!all_fv) {
    if (!b.fv_ready) {
      FAMS_TRY(build_coarse_system(b, b.cs[1], 0, b.csh[1]));
      b.fv_ready = true;
    }
    cs = &b.cs[1];
  }
  const Inst& I = b.h[ii];
  const CoarseHost& chh = all_fv ? b.csh[0] : b.csh[1];
  if (chh.bad[ii]) {
    set_error("instance " + std::to_string(ii) + ": the finite-volume coarse system is "
              "numerically singular (zero pivot at LU step " + std::to_string(chh.bad[ii] - 1) +
              "); no conservative reconstruction");
    return FAMS_EBREAKDOWN;
  }
  double* pp = b.r;   // work vectors: r = residual, dp = p', y = p~
  double* pt = b.y;
  double* res = b.dp;
  size_t smem = sizeof(double) * 2 * (size_t)I.nc;
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  max_smem -= 1024;  // static shared memory of the kernels
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_local, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  fams::note_launch(), k_flux_stage<<<1, 512, smem, st>>>(b.d_inst, ii, *cs, b.rowptr, b.col, b.val, b.blk_ptr,
                                     b.blk_cell, b.p_ptr, b.p_col, b.p_val, b.q, x_dev, res, pp);
  FAMS_CUDA(cudaGetLastError());
  // local problems: split by size (shared memory or a bounded global workspace)
  std::vector<int> hp(I.nc + 1);
  FAMS_CUDA(cudaMemcpyAsync(hp.data(), b.blk_ptr + I.nc_off, sizeof(int) * (I.nc + 1),
                            cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaStreamSynchronize(st));
  std::vector<int> small, large;
  size_t small_smem = 0;
  long long big = 0;
  for (int c = 0; c < I.nc; ++c) {
    long long m = hp[c + 1] - hp[c];
    long long need = (m * m + m) * 8;
    if (need + 1024 <= max_smem) { small.push_back(c); small_smem = std::max(small_smem, (size_t)need); }
    else { large.push_back(c); big = std::max(big, m * m + m); }
  }
  int* lst = nullptr;
  FAMS_CUDA(cudaMalloc(&lst, sizeof(int) * (I.nc + 1)));
  double* work = nullptr;
  int status = FAMS_OK;
  if (!small.empty()) {
    cudaMemcpyAsync(lst, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice, st);
    fams::note_launch(), k_flux_local<<<(int)small.size(), 256, small_smem, st>>>(
        b.d_inst, ii, lst, b.blk_ptr, b.blk_cell, b.rowptr, b.col, b.val, b.TD, b.qD, b.q,
        b.primal, b.node_cell, pp, pt, nullptr, 0, b.d_err);
  }
  if (!large.empty()) {
    long long per = std::max(1LL, (1LL << 26) / std::max(big, 1LL));
    if (cudaMalloc(&work, sizeof(double) * big * std::min<long long>(per, large.size())) != cudaSuccess) {
      cudaFree(lst);
      set_error("flux workspace allocation failed");
      return FAMS_ENOMEM;
    }
    int* l2 = lst + small.size();
    cudaMemcpyAsync(l2, large.data(), sizeof(int) * large.size(), cudaMemcpyHostToDevice, st);
    for (size_t o = 0; o < large.size(); o += per) {
      int cnt = (int)std::min<long long>(per, (long long)(large.size() - o));
      fams::note_launch(), k_flux_local<<<cnt, 256, 0, st>>>(b.d_inst, ii, l2 + o, b.blk_ptr, b.blk_cell, b.rowptr,
                                        b.col, b.val, b.TD, b.qD, b.q, b.primal, b.node_cell, pp,
                                        pt, work, big, b.d_err);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) status = FAMS_ECUDA;
  long long nfaces = (long long)(I.nx + 1) * I.ny * (I.dim == 3 ? I.nz : 1) +
                     (long long)I.nx * (I.ny + 1) * (I.dim == 3 ? I.nz : 1) +
                     (I.dim == 3 ? (long long)I.nx * I.ny * (I.nz + 1) : 0);
  if (status == FAMS_OK) {
    fams::note_launch(), k_flux_faces<<<grid_for(nfaces, 256), 256, 0, st>>>(b.d_inst, ii, b.perm, b.primal, pp, pt,
                                                        face);
    long long nn = (long long)I.nnc + I.nff;
    if (nn > 0)
      fams::note_launch(), k_flux_nnc<<<grid_for(nn, 256), 256, 0, st>>>(b.d_inst, ii, b.nnc_row_m, b.nnc_row_f,
                                                    b.nnc_T, b.ff_a, b.ff_b, b.ff_T, b.primal, pp,
                                                    pt, nnc_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) status = FAMS_ECUDA;
  }
  cudaStreamSynchronize(st);
  cudaFree(lst);
  if (work) cudaFree(work);
  if (status != FAMS_OK) {
    set_error(std::string("flux kernels: ") + cudaGetErrorString(e));
    return status;
  }
  return b.check_err("flux reconstruction");
}

}  // namespace fams
