// Conservative fine-scale flux reconstruction after any iterate (Sec. 1 and
// Sec. 3.2: possible after an MSFV stage).
//   1. p' = x + P (R^FV A P)^-1 R^FV (q - A x)          (one FV stage)
//   2. every connection between two primal blocks carries T (p'_i - p'_j);
//   3. each primal block solves its own TPFA problem with those fluxes as
//      Neumann data (Dirichlet faces stay Dirichlet; a block without one is
//      pinned to p' at its coarse node) -> p~;
//   4. connections inside a block carry T (p~_i - p~_j).
// R^FV (q - A p') = 0 makes every local problem consistent, so the result is
// mass conservative cell by cell.  All requested instances are processed
// together: one CTA per instance for step 1, one CTA per primal block for
// step 3, one thread per face or connection for steps 2 and 4.
#include <algorithm>

#include "batch.cuh"

namespace fams {

namespace {

// step 1, one CTA per listed instance
__global__ void k_flux_stage(const Inst* inst, const int* list, CoarseSys cs, const int* rowptr,
                             const int* col, const double* val, const int* blk_ptr,
                             const int* blk_cell, const int* p_ptr, const int* p_col,
                             const double* p_val, const double* q, const double* x, double* r,
                             double* pp) {
  extern __shared__ double sm[];
  int ii = list[blockIdx.x];
  const Inst& I = inst[ii];
  int n = I.n, ro = I.row_off, nc = I.nc, co = I.nc_off;
  double* yb = sm;
  double* ecs = sm + nc;
  for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
    double s = q[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) s -= val[p] * x[col[p]];
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
    pp[i] = x[i] + s;
  }
}

// step 3: one CTA per listed primal block (global coarse index), dense
// Gaussian elimination with partial pivoting of the block's local TPFA matrix
__global__ void k_flux_local(const Inst* inst, int B, const int* off_nc, const int* blk_list,
                             const int* blk_ptr, const int* blk_cell, const int* rowptr,
                             const int* col, const double* val, const double* TD, const double* q,
                             const int* primal, const int* node_cell, const double* pp,
                             double* pt, double* gwork, long long gstride, int* err) {
  extern __shared__ double dsm[];
  int c = blk_list[blockIdx.x];
  const Inst& I = inst[find_segment(off_nc, B + 1, c)];
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

__device__ inline long long faces_of(const Inst& I) {
  long long nz = I.dim == 3 ? I.nz : 1;
  return (long long)(I.nx + 1) * I.ny * nz + (long long)I.nx * (I.ny + 1) * nz +
         (I.dim == 3 ? (long long)I.nx * I.ny * (nz + 1) : 0);
}

// steps 2 and 4 on the matrix faces of every listed instance: x faces
// ((nx+1) ny nz, x fastest), then y faces, then z faces; positive along +axis
__global__ void k_flux_faces(const Inst* inst, const int* list, int nlist, const long long* foff,
                             long long ftot, const double* perm, const int* primal,
                             const double* pp, const double* pt, double* face) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ftot) return;
  int li = 0, hi = nlist - 1;
  while (li < hi) {
    int mid = (li + hi + 1) >> 1;
    if (foff[mid] <= g) li = mid; else hi = mid - 1;
  }
  const Inst& I = inst[list[li]];
  long long f = g - foff[li];
  int nx = I.nx, ny = I.ny, nz = I.dim == 3 ? I.nz : 1;
  long long nfx = (long long)(nx + 1) * ny * nz, nfy = (long long)nx * (ny + 1) * nz;
  const double* k = perm + I.m_off;
  int ro = I.row_off;
  int axis, i, j, l;
  long long e = f;
  if (e < nfx) { axis = 0; i = (int)(e % (nx + 1)); j = (int)((e / (nx + 1)) % ny); l = (int)(e / ((long long)(nx + 1) * ny)); }
  else if ((e -= nfx) < nfy) { axis = 1; i = (int)(e % nx); j = (int)((e / nx) % (ny + 1)); l = (int)(e / ((long long)nx * (ny + 1))); }
  else { e -= nfy; axis = 2; i = (int)(e % nx); j = (int)((e / nx) % ny); l = (int)(e / ((long long)nx * ny)); }
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
  face[g] = out;
}

// steps 2 and 4 on the fracture connections: matrix-fracture (positive
// matrix -> fracture), then fracture-fracture (positive lower -> higher cell)
__global__ void k_flux_nnc(const Inst* inst, const int* list, int nlist, const long long* noff,
                           long long ntot, const int* nrow_m, const int* nrow_f, const double* nT,
                           const int* ffa, const int* ffb, const double* ffT, const int* primal,
                           const double* pp, const double* pt, double* out) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ntot) return;
  int li = 0, hi = nlist - 1;
  while (li < hi) {
    int mid = (li + hi + 1) >> 1;
    if (noff[mid] <= g) li = mid; else hi = mid - 1;
  }
  const Inst& I = inst[list[li]];
  long long t = g - noff[li];
  if (t < I.nnc) {
    long long k = I.nnc_off + t;
    out[g] = nT[k] * (pp[nrow_m[k]] - pp[nrow_f[k]]);
  } else {
    long long k = I.ff_off + (t - I.nnc);
    int a = ffa[k], b = ffb[k];
    const double* p = primal[a] == primal[b] ? pt : pp;
    out[g] = ffT[k] * (p[a] - p[b]);
  }
}

}  // namespace

// The R^FV coarse system of the reconstruction: the iteration's own when every
// instance iterates with R^FV, otherwise a second one built on first use.
int flux_prepare(Batch& b, const CoarseHost** ch) {
  bool all_fv = true;
  for (auto& I : b.h) all_fv = all_fv && I.restriction == FAMS_R_FV;
  if (all_fv) {
    *ch = &b.csh[0];
    return FAMS_OK;
  }
  if (!b.fv_ready) {
    FAMS_TRY(build_coarse_system(b, b.cs[1], 0, b.csh[1]));
    b.fv_ready = true;
    b.free_tmp();
  }
  *ch = &b.csh[1];
  return FAMS_OK;
}

// Flux of the listed instances.  x: concatenated iterates (global rows);
// face / nnc: concatenated outputs at foff / noff (per listed instance).
int run_flux(Batch& b, const std::vector<int>& list, const double* x, double* face,
             const std::vector<long long>& foff, double* nnc, const std::vector<long long>& noff) {
  cudaStream_t st = b.stream;
  const CoarseHost* chh = nullptr;
  FAMS_TRY(flux_prepare(b, &chh));
  CoarseSys* cs = (chh == &b.csh[0]) ? &b.cs[0] : &b.cs[1];
  int nl = (int)list.size();
  if (nl == 0) return FAMS_OK;
  double* pp = b.r;   // work vectors: r = p', y = p~, dp = residual
  double* pt = b.y;
  double* res = b.dp;
  int maxnc = 0;
  for (int ii : list) maxnc = std::max(maxnc, b.h[ii].nc);
  size_t smem = sizeof(double) * 2 * (size_t)maxnc;
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  max_smem -= 1024;  // static shared memory of the kernels
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_local, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  int* dlist = nullptr;
  FAMS_TRY(b.scratch((void**)&dlist, sizeof(int) * nl));
  FAMS_CUDA(cudaMemcpyAsync(dlist, list.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st));
  fams::note_launch(), k_flux_stage<<<nl, 512, smem, st>>>(
      b.d_inst, dlist, *cs, b.rowptr, b.col, b.val, b.blk_ptr, b.blk_cell, b.p_ptr, b.p_col,
      b.p_val, b.q, x, res, pp);
  FAMS_CUDA(cudaGetLastError());
  // local problems of every primal block of the listed instances, split by
  // size (shared memory or a bounded global workspace)
  std::vector<int> hp(b.tot_nc + 1);
  FAMS_CUDA(cudaMemcpyAsync(hp.data(), b.blk_ptr, sizeof(int) * (b.tot_nc + 1),
                            cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaStreamSynchronize(st));
  std::vector<int> small, large;
  size_t small_smem = 0;
  long long big = 0;
  for (int ii : list) {
    const Inst& I = b.h[ii];
    for (int c = I.nc_off; c < I.nc_off + I.nc; ++c) {
      long long m = hp[c + 1] - hp[c];
      long long need = (m * m + m) * 8;
      if (need <= max_smem) { small.push_back(c); small_smem = std::max(small_smem, (size_t)need); }
      else { large.push_back(c); big = std::max(big, m * m + m); }
    }
  }
  int* lst = nullptr;
  FAMS_TRY(b.scratch((void**)&lst, sizeof(int) * (small.size() + large.size() + 1)));
  if (!small.empty()) {
    FAMS_CUDA(cudaMemcpyAsync(lst, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice, st));
    fams::note_launch(), k_flux_local<<<(int)small.size(), 256, small_smem, st>>>(
        b.d_inst, b.B, b.off_nc, lst, b.blk_ptr, b.blk_cell, b.rowptr, b.col, b.val, b.TD, b.q,
        b.primal, b.node_cell, pp, pt, nullptr, 0, b.d_err);
  }
  if (!large.empty()) {
    long long per = std::max(1LL, (1LL << 26) / std::max(big, 1LL));
    double* work = nullptr;
    FAMS_TRY(b.scratch((void**)&work, sizeof(double) * big * std::min<long long>(per, large.size())));
    int* l2 = lst + small.size();
    FAMS_CUDA(cudaMemcpyAsync(l2, large.data(), sizeof(int) * large.size(), cudaMemcpyHostToDevice, st));
    for (size_t o = 0; o < large.size(); o += per) {
      int cnt = (int)std::min<long long>(per, (long long)(large.size() - o));
      fams::note_launch(), k_flux_local<<<cnt, 256, 0, st>>>(
          b.d_inst, b.B, b.off_nc, l2 + o, b.blk_ptr, b.blk_cell, b.rowptr, b.col, b.val, b.TD,
          b.q, b.primal, b.node_cell, pp, pt, work, big, b.d_err);
    }
  }
  FAMS_CUDA(cudaGetLastError());
  long long* dfo = nullptr;
  long long* dno = nullptr;
  FAMS_TRY(b.scratch((void**)&dfo, sizeof(long long) * (nl + 1)));
  FAMS_TRY(b.scratch((void**)&dno, sizeof(long long) * (nl + 1)));
  FAMS_CUDA(cudaMemcpyAsync(dfo, foff.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, st));
  FAMS_CUDA(cudaMemcpyAsync(dno, noff.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, st));
  if (foff[nl] > 0)
    fams::note_launch(), k_flux_faces<<<grid_for(foff[nl], 256), 256, 0, st>>>(
        b.d_inst, dlist, nl, dfo, foff[nl], b.perm, b.primal, pp, pt, face);
  if (noff[nl] > 0)
    fams::note_launch(), k_flux_nnc<<<grid_for(noff[nl], 256), 256, 0, st>>>(
        b.d_inst, dlist, nl, dno, noff[nl], b.nnc_row_m, b.nnc_row_f, b.nnc_T, b.ff_a, b.ff_b,
        b.ff_T, b.primal, pp, pt, nnc);
  FAMS_CUDA(cudaGetLastError());
  FAMS_CUDA(cudaStreamSynchronize(st));
  b.free_tmp();
  return b.check_err("flux reconstruction");
}

}  // namespace fams
