// Conservative fine-scale flux reconstruction after any iterate (Sec. 1 and
// Sec. 3.2: possible after an MSFV stage).
//   1. p' = x + P (R^FV A P)^-1 R^FV (q - A x)          (one FV stage; P here
//      holds the basis functions before truncation: a truncated basis
//      function can lie inside its own primal block, where its column of
//      R^FV A P vanishes)
//   2. every connection between two primal blocks carries T (p'_i - p'_j);
//   3. each primal block solves its own TPFA problem with those fluxes as
//      Neumann data (Dirichlet faces stay Dirichlet; a block without one is
//      pinned to p' at its coarse node) -> p~;
//   4. connections inside a block carry T (p~_i - p~_j).
// R^FV (q - A p') = 0 makes every local problem consistent, so the result is
// mass conservative cell by cell.  All requested instances are processed
// together: one CTA per instance for step 1, one warp (small blocks) or one
// CTA per primal block for step 3, one thread per face or connection for
// steps 2 and 4.
#include <algorithm>

#include "band_solve.cuh"
#include "batch.cuh"
#include "dense.cuh"

namespace fams {

namespace {

constexpr int LOCAL_CTA_WARPS = 4;            // warp-per-block launches: blocks per CTA
constexpr long long LOCAL_WARP_NEED = 1024;   // doubles: largest block solved by one warp
constexpr long long LOCAL_MID_NEED = 6144;    // doubles: largest block on a 128-thread CTA

// step 1, one CTA per listed instance
__global__ void k_flux_stage(const Inst* inst, const int* list, CoarseSys cs, const int* rowptr,
                             const int* col, const double* val, const int* blk_ptr,
                             const int* blk_cell, const int* p_ptr, const int* p_col,
                             const double* p_val, const double* q, const double* x, double* r,
                             double* pp, double* gws, long long gstride, int bb) {
  extern __shared__ double sm[];
  __shared__ int pbuf[2 * band::CH_MAX];
  int ii = list[blockIdx.x];
  const Inst& I = inst[ii];
  int n = I.n, ro = I.row_off, nc = I.nc, co = I.nc_off;
  // the two coarse vectors: shared memory, or global scratch when they do not
  // fit; then two chunks of bb doubles for the band solve's staged columns
  double* yb = gws ? gws + (long long)blockIdx.x * gstride : sm;
  double* ecs = yb + nc;
  double* bbuf = gws ? sm : sm + 2 * (long long)nc;
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
  // the R^FV band factors (gbtrs steps on four warps, the others staging
  // band columns)
  band::coarse_solve(cs.band + cs.band_off[ii], cs.ipiv + co, nc, cs.kl[ii], cs.ku[ii], yb, bbuf,
                     pbuf, bb);
  __syncthreads();
  for (int k = threadIdx.x; k < nc; k += blockDim.x) ecs[perm[k]] = yb[k];
  __syncthreads();
  for (int i = ro + threadIdx.x; i < ro + n; i += blockDim.x) {
    double s = 0.0;
    for (int p = p_ptr[i]; p < p_ptr[i + 1]; ++p) s += p_val[p] * ecs[p_col[p]];
    pp[i] = x[i] + s;
  }
}

// step 3: the local TPFA problem of one primal block (global coarse index)
// on a thread group: [K | rhs] with leading dimension m + 1 (then m doubles
// of pivot reciprocals), Neumann data
// from p' on the block boundary, pinned to p' at the block's coarse node when
// no Dirichlet face closes it; dense elimination without pivoting
struct LocalArgs {
  const Inst* inst;
  int B;
  const int* off_nc;
  const int* blk_list;
  long long nblk;
  const int* blk_ptr;
  const int* blk_cell;
  const int* rowptr;
  const int* col;
  const double* val;
  const double* TD;
  const double* q;
  const int* primal;
  const int* node_cell;
  const double* pp;
  double* pt;
  const int* bw;   // per primal block: lower and upper bandwidth in block order
  int* err;
};

// bandwidths of each primal block's local matrix in block order (cells in
// ascending index): one thread per block
__global__ void k_blk_band(const int* blk_ptr, const int* blk_cell, int nblk, const int* rowptr,
                           const int* col, const int* primal, int* bw) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nblk) return;
  const int a0 = blk_ptr[c], m = blk_ptr[c + 1] - a0;
  int bl = 0, bu = 0;
  for (int t = 0; t < m; ++t) {
    const int i = blk_cell[a0 + t];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int j = col[p];
      if (j == i || primal[j] != primal[i]) continue;
      int lo = 0, hi = m - 1, pos = -1;
      while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = blk_cell[a0 + mid];
        if (v == j) { pos = mid; break; }
        if (v < j) lo = mid + 1; else hi = mid - 1;
      }
      if (pos < 0) continue;
      bl = max(bl, t - pos);
      bu = max(bu, pos - t);
    }
  }
  bw[2 * c] = bl;
  bw[2 * c + 1] = bu;
}

template <class G>
__device__ void flux_local(const LocalArgs& a, int c, double* K, int* red) {
  const int gr = G::rank(), gs = G::size();
  const Inst& I = a.inst[find_segment(a.off_nc, a.B + 1, c)];
  const int a0 = a.blk_ptr[c], m = a.blk_ptr[c + 1] - a0;
  // band storage: W band entries, then the right-hand side
  const int bl = a.bw[2 * c], bu = a.bw[2 * c + 1], W = bl + bu + 1;
  const int ld = W + 1;
  (void)red;
  for (long long t = gr; t < (long long)m * ld; t += gs) K[t] = 0.0;
  G::sync();
  const int myblk = c - I.nc_off;
  bool hasD = false;
  for (int t = gr; t < m; t += gs) {
    int i = a.blk_cell[a0 + t];
    double* Kt = K + (long long)t * ld;
    double b = a.q[i];  // sources + Dirichlet terms
    double d = a.TD[i];
    if (a.TD[i] > 0.0) hasD = true;
    for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) {
      int j = a.col[p];
      if (j == i) continue;
      double T = -a.val[p];
      if (a.primal[j] == myblk) {
        int lo = 0, hi = m - 1, pos = -1;
        while (lo <= hi) {
          int mid = (lo + hi) >> 1;
          int v = a.blk_cell[a0 + mid];
          if (v == j) { pos = mid; break; }
          if (v < j) lo = mid + 1; else hi = mid - 1;
        }
        if (pos < 0 || t - pos > bl || pos - t > bu) { atomicCAS(a.err, 0, DERR_INVAL); continue; }
        Kt[pos - t + bl] -= T;
        d += T;
      } else {
        b -= T * (a.pp[i] - a.pp[j]);
      }
    }
    Kt[bl] += d;
    Kt[W] = b;
  }
  // pin the coarse node unless a Dirichlet face closes the block
  bool anyD = G::per_warp ? __any_sync(0xffffffffu, hasD) : __syncthreads_or(hasD);
  if (!anyD) {
    int v = a.node_cell[c];
    int lo = 0, hi = m - 1, pos = 0;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int w = a.blk_cell[a0 + mid];
      if (w == v) { pos = mid; break; }
      if (w < v) lo = mid + 1; else hi = mid - 1;
    }
    G::sync();
    double* Kp = K + (long long)pos * ld;
    for (int j = gr; j <= W; j += gs) Kp[j] = j == bl ? 1.0 : (j == W ? a.pp[v] : 0.0);
  }
  G::sync();
  if (!ge_solve<G>(K, ld, m, 1, bl, bu, K + (long long)m * ld)) {
    if (gr == 0) atomicCAS(a.err, 0, DERR_BREAKDOWN);
    return;
  }
  for (int t = gr; t < m; t += gs) a.pt[a.blk_cell[a0 + t]] = K[(long long)t * ld + W];
}

// primal blocks of the listed instances: one warp each (WarpGroup, several
// per CTA, `slice` doubles of shared memory each) or one CTA each (CtaGroup;
// in shared memory, or in `gwork` with `slice` doubles per CTA)
template <class G>
__global__ void k_flux_local(LocalArgs a, long long slice, double* gwork) {
  extern __shared__ double dsm[];
  __shared__ int red[32];
  const int sub = G::per_warp ? (threadIdx.x >> 5) : 0;
  const long long idx = (long long)blockIdx.x * (G::per_warp ? (blockDim.x >> 5) : 1) + sub;
  if (idx >= a.nblk) return;
  double* K = gwork ? gwork + (long long)blockIdx.x * slice : dsm + (long long)sub * slice;
  flux_local<G>(a, a.blk_list[idx], K, red);
}

__device__ inline long long faces_of(const Inst& I) {
  long long nz = I.dim == 3 ? I.nz : 1;
  return (long long)(I.nx + 1) * I.ny * nz + (long long)I.nx * (I.ny + 1) * nz +
         (I.dim == 3 ? (long long)I.nx * I.ny * (nz + 1) : 0);
}

// steps 2 and 4 on the matrix faces of every listed instance: x faces
// ((nx+1) ny nz, x fastest), then y faces, then z faces; positive along +axis
// mob (nullable): mobility scales of a time-step update, applied as the
// harmonic mean of the two cells' scales (a Dirichlet face: the cell's)
__global__ void k_flux_faces(const Inst* inst, const int* list, int nlist, const long long* foff,
                             long long ftot, const double* perm, const double* mob,
                             const int* primal, const double* pp, const double* pt, double* face) {
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
      if (mob) TDf *= mob[ro + cell];
      double pc = pt[ro + cell];
      out = (c_ax == 0) ? TDf * (I.bc_val[fid] - pc) : TDf * (pc - I.bc_val[fid]);
    }
  } else {
    long long lo_cell = hi_cell - stride;
    double T = area / (h / (2.0 * k[lo_cell]) + h / (2.0 * k[hi_cell]));
    if (mob) {
      double a = mob[ro + lo_cell], c = mob[ro + hi_cell];
      T *= 2.0 * a * c / (a + c);
    }
    bool same = primal[ro + lo_cell] == primal[ro + hi_cell];
    const double* p = same ? pt : pp;
    out = T * (p[ro + lo_cell] - p[ro + hi_cell]);
  }
  face[g] = out;
}

// perforations of the wells, for the flux output: global rows of the cell
// and of its rate well (-1: pressure well), beta = PI k, bottom-hole pressure
struct PerfArgs {
  const int* row;
  const int* wrow;
  const double* beta;
  const double* bhp;
  const double* mob;   // nullable: mobility scales of a time-step update
};

// steps 2 and 4 on the fracture connections: matrix-fracture (positive
// matrix -> fracture), then fracture-fracture (positive lower -> higher
// cell), then the well perforations (positive cell -> well: a rate well
// is its own primal block, so T (p'_cell - p'_well); a pressure well like a
// Dirichlet face, from the local solution)
__global__ void k_flux_nnc(const Inst* inst, const int* list, int nlist, const long long* noff,
                           long long ntot, const int* nrow_m, const int* nrow_f, const double* nT,
                           const int* ffa, const int* ffb, const double* ffT, PerfArgs pf,
                           const int* primal, const double* pp, const double* pt, double* out) {
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
  } else if (t < I.nnc + I.nff) {
    long long k = I.ff_off + (t - I.nnc);
    int a = ffa[k], b = ffb[k];
    const double* p = primal[a] == primal[b] ? pt : pp;
    out[g] = ffT[k] * (p[a] - p[b]);
  } else {
    const long long k = I.perf_off + (t - I.nnc - I.nff);
    const int c = pf.row[k], w = pf.wrow[k];
    double T = pf.beta[k];
    if (w >= 0) {
      if (pf.mob) T *= 2.0 * pf.mob[c] * pf.mob[w] / (pf.mob[c] + pf.mob[w]);
      out[g] = T * (pp[c] - pp[w]);
    } else {
      if (pf.mob) T *= pf.mob[c];
      out[g] = T * (pt[c] - pf.bhp[k]);
    }
  }
}

}  // namespace

// primal-block sizes and the bandwidths of their local problems, fixed after
// setup: computed once, kept on the host for the size classes
int local_bands(Batch& b) {
  if (!b.h_blk_ptr.empty()) return FAMS_OK;
  cudaStream_t st = b.stream;
  std::vector<int> hp(b.tot_nc + 1), hbw(2 * (b.tot_nc + 1), 0);
  FAMS_TRY(b.alloc((void**)&b.blk_bw, sizeof(int) * 2 * (b.tot_nc + 1)));
  if (b.tot_nc > 0)
    fams::note_launch(), k_blk_band<<<grid_for(b.tot_nc, 128), 128, 0, st>>>(
        b.blk_ptr, b.blk_cell, (int)b.tot_nc, b.rowptr, b.col, b.primal, b.blk_bw);
  FAMS_CUDA(cudaGetLastError());
  FAMS_CUDA(cudaMemcpyAsync(hp.data(), b.blk_ptr, sizeof(int) * (b.tot_nc + 1),
                            cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaMemcpyAsync(hbw.data(), b.blk_bw, sizeof(int) * 2 * b.tot_nc,
                            cudaMemcpyDeviceToHost, st));
  FAMS_CUDA(cudaStreamSynchronize(st));
  b.h_blk_bw.swap(hbw);
  b.h_blk_ptr.swap(hp);
  return FAMS_OK;
}

// The R^FV coarse system of the reconstruction, R^FV A P with the basis
// functions before truncation: the iteration's own when every instance
// iterates with R^FV and none truncates, otherwise a second one built on
// first use.
int flux_prepare(Batch& b, const CoarseHost** ch) {
  FAMS_TRY(local_bands(b));
  bool all_fv = b.pf_alias;
  for (auto& I : b.h) all_fv = all_fv && I.restriction == FAMS_R_FV;
  if (all_fv) {
    *ch = &b.csh[0];
    return FAMS_OK;
  }
  if (!b.fv_ready) {
    // built once; a time-step update (fv_built, !fv_ready) refactors it in place
    FAMS_TRY(build_coarse_system(b, b.cs[1], 0, b.csh[1], b.fv_built, b.pf_ptr, b.pf_col,
                                 b.pf_val));
    b.fv_ready = true;
    b.fv_built = true;
    b.free_tmp();
  }
  *ch = &b.csh[1];
  return FAMS_OK;
}

// flux_prepare on the side stream, started while the iteration kernels run on
// the context's stream: the R^FV system reads only A and P (complete at
// `ready`, recorded before the iteration), and its one-CTA-per-instance
// kernels take the SM slots of instances that converge early.  The context's
// stream then waits for it.  A failure here does not fail the solve: the
// system stays unbuilt and the reconstruction builds it (and reports the
// error) on its first call.
int flux_beside(Batch& b, cudaEvent_t ready) {
  // a whole-GPU context builds it on its own stream when first needed: its
  // cooperative kernels take every SM and never run beside another kernel
  if (whole_gpu(b)) return FAMS_OK;
  bool all_fv = b.pf_alias;
  for (auto& I : b.h) all_fv = all_fv && I.restriction == FAMS_R_FV;
  if ((all_fv || b.fv_ready) && !b.h_blk_ptr.empty()) return FAMS_OK;
  if (!b.side) {
    FAMS_CUDA(cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking));
    FAMS_CUDA(cudaEventCreateWithFlags(&b.side_done, cudaEventDisableTiming));
  }
  FAMS_CUDA(cudaStreamWaitEvent(b.side, ready, 0));
  std::vector<void*> keep;
  keep.swap(b.tmp);   // scratch of the running solve stays out of this build's frees
  std::swap(b.stream, b.side);
  const CoarseHost* ch = nullptr;
  int rc = flux_prepare(b, &ch);
  b.free_tmp();
  std::swap(b.stream, b.side);
  b.tmp.swap(keep);
  FAMS_CUDA(cudaEventRecord(b.side_done, b.side));
  FAMS_CUDA(cudaStreamWaitEvent(b.stream, b.side_done, 0));
  (void)rc;
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
  // band chunks of the staged band solve: at least one column of the
  // widest listed band
  int bb = 3072;
  for (int ii : list) bb = std::max(bb, chh->kl[ii] + chh->ku[ii] + 1);
  const size_t band_smem = sizeof(double) * 2 * (size_t)bb;
  size_t smem = sizeof(double) * 2 * (size_t)maxnc + band_smem;
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  max_smem -= 1024;  // static shared memory of the kernels
  if (band_smem > (size_t)max_smem) {
    set_error("reconstruction's coarse band too wide for the staged band solve");
    return FAMS_ECAPACITY;
  }
  double* gws = nullptr;   // coarse vectors in global memory when they do not fit beside
  if (smem > (size_t)max_smem) {
    FAMS_TRY(b.scratch((void**)&gws, sizeof(double) * 2 * (size_t)maxnc * (size_t)nl));
    smem = band_smem;
  }
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_local<CtaGroup>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  FAMS_CUDA(cudaFuncSetAttribute(k_flux_local<WarpGroup>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  int* dlist = nullptr;
  FAMS_TRY(b.scratch((void**)&dlist, sizeof(int) * nl));
  FAMS_CUDA(cudaMemcpyAsync(dlist, list.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st));
  fams::note_launch(), k_flux_stage<<<nl, 512, smem, st>>>(
      b.d_inst, dlist, *cs, b.rowptr, b.col, b.val, b.blk_ptr, b.blk_cell, b.pf_ptr, b.pf_col,
      b.pf_val, b.q, x, res, pp, gws, 2 * (long long)maxnc, bb);
  FAMS_CUDA(cudaGetLastError());
  // local problems of every primal block of the listed instances, by size
  // class (doubles of [K | rhs]): one warp, a 128-thread CTA, a 256-thread
  // CTA in shared memory, or a 512-thread CTA on a bounded global workspace
  const std::vector<int>& hp = b.h_blk_ptr;   // filled by flux_prepare
  const std::vector<int>& hbw = b.h_blk_bw;
  std::vector<int> cls[4];
  long long cmax[4] = {0, 0, 0, 0};
  for (int ii : list) {
    const Inst& I = b.h[ii];
    for (int c = I.nc_off; c < I.nc_off + I.nc; ++c) {
      long long m = hp[c + 1] - hp[c];
      // band and right-hand side of every row, pivot reciprocals
      long long need = m * ((long long)hbw[2 * c] + hbw[2 * c + 1] + 3);
      int q = need <= LOCAL_WARP_NEED ? 0 : need <= LOCAL_MID_NEED ? 1
            : need * 8 <= max_smem ? 2 : 3;
      cls[q].push_back(c);
      ++b.class_cnt[4 + q];
      cmax[q] = std::max(cmax[q], need);
    }
  }
  int* lst = nullptr;
  FAMS_TRY(b.scratch((void**)&lst, sizeof(int) * (b.tot_nc + 1)));
  LocalArgs la{b.d_inst, b.B, b.off_nc, nullptr, 0, b.blk_ptr, b.blk_cell, b.rowptr, b.col,
               b.val, b.TD, b.q, b.primal, b.node_cell, pp, pt, b.blk_bw, b.d_err};
  // disjoint size classes: lists and workspace on the main stream, then each
  // class on its own stream so that their tails overlap
  int* ls[4] = {nullptr, nullptr, nullptr, nullptr};
  long long lo = 0;
  for (int q = 0; q < 4; ++q) {
    if (cls[q].empty()) continue;
    ls[q] = lst + lo;
    lo += (long long)cls[q].size();
    FAMS_CUDA(cudaMemcpyAsync(ls[q], cls[q].data(), sizeof(int) * cls[q].size(),
                              cudaMemcpyHostToDevice, st));
  }
  const long long per3 = std::max(1LL, (1LL << 26) / std::max(cmax[3], 1LL));
  double* work = nullptr;
  if (!cls[3].empty())
    FAMS_TRY(b.scratch((void**)&work, sizeof(double) * cmax[3] *
                                          std::min(per3, (long long)cls[3].size())));
  cudaStream_t cst[4] = {st, st, st, st};
  FAMS_TRY(fork_streams(b, 3, cst + 1));
  for (int q = 0; q < 4; ++q) {
    if (cls[q].empty()) continue;
    long long cnt = (long long)cls[q].size();
    int* l = ls[q];
    cudaStream_t qs = cst[q];
    la.blk_list = l;
    la.nblk = cnt;
    if (q == 0) {
      long long slice = (cmax[0] + 3) & ~3LL;
      fams::note_launch(),
          k_flux_local<WarpGroup><<<(int)((cnt + LOCAL_CTA_WARPS - 1) / LOCAL_CTA_WARPS),
                                    32 * LOCAL_CTA_WARPS,
                                    sizeof(double) * slice * LOCAL_CTA_WARPS, qs>>>(la, slice,
                                                                                  nullptr);
    } else if (q < 3) {
      fams::note_launch(),
          k_flux_local<CtaGroup><<<(int)cnt, q == 1 ? 128 : 256, sizeof(double) * cmax[q], qs>>>(
              la, cmax[q], nullptr);
    } else {
      for (long long o = 0; o < cnt; o += per3) {
        la.blk_list = l + o;
        la.nblk = std::min(per3, cnt - o);
        fams::note_launch(),
            k_flux_local<CtaGroup><<<(int)la.nblk, 512, 0, qs>>>(la, cmax[3], work);
      }
    }
    FAMS_CUDA(cudaGetLastError());
  }
  FAMS_TRY(join_streams(b, 3));
  FAMS_CUDA(cudaGetLastError());
  long long* dfo = nullptr;
  long long* dno = nullptr;
  FAMS_TRY(b.scratch((void**)&dfo, sizeof(long long) * (nl + 1)));
  FAMS_TRY(b.scratch((void**)&dno, sizeof(long long) * (nl + 1)));
  FAMS_CUDA(cudaMemcpyAsync(dfo, foff.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, st));
  FAMS_CUDA(cudaMemcpyAsync(dno, noff.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, st));
  if (foff[nl] > 0)
    fams::note_launch(), k_flux_faces<<<grid_for(foff[nl], 256), 256, 0, st>>>(
        b.d_inst, dlist, nl, dfo, foff[nl], b.perm, b.mob, b.primal, pp, pt, face);
  if (noff[nl] > 0)
    fams::note_launch(), k_flux_nnc<<<grid_for(noff[nl], 256), 256, 0, st>>>(
        b.d_inst, dlist, nl, dno, noff[nl], b.nnc_row_m, b.nnc_row_f, b.nnc_T, b.ff_a, b.ff_b,
        b.ff_T, PerfArgs{b.perf_row, b.perf_wrow, b.perf_beta, b.perf_bhp, b.mob}, b.primal, pp,
        pt, nnc);
  FAMS_CUDA(cudaGetLastError());
  FAMS_CUDA(cudaStreamSynchronize(st));
  b.free_tmp();
  return b.check_err("flux reconstruction");
}

}  // namespace fams
