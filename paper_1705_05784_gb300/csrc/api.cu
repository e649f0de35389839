// C ABI of libfams (include/fams.h): argument checks, batch bookkeeping and
// the order of the setup phases.  Every computation of the method runs in the
// kernels of the other translation units.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>

#include "batch.cuh"

struct fams_ctx {
  fams::Batch b;
};

namespace fams {

constexpr uint64_t POOL_KEEP = 32ull << 30;   // least freed device memory the pool keeps

namespace {
thread_local std::string g_err;
std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};
}

void set_error(const std::string& msg) { g_err = msg; }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

int Batch::upload_inst() {
  std::vector<int> o(8 * (B + 1));
  for (int i = 0; i <= B; ++i) {
    bool last = i == B;
    const Inst* I = last ? nullptr : &h[i];
    o[0 * (B + 1) + i] = last ? (int)tot_m : I->m_off;
    o[1 * (B + 1) + i] = last ? (int)tot_fr : I->fr_off;
    o[2 * (B + 1) + i] = last ? (int)tot_fc : I->fc_off;
    o[3 * (B + 1) + i] = last ? (int)tot_s : I->s_off;
    o[4 * (B + 1) + i] = last ? (int)tot_row : I->row_off;
    o[5 * (B + 1) + i] = last ? (int)tot_pair : I->inter_off;
    o[6 * (B + 1) + i] = last ? (int)tot_nc : I->nc_off;
    o[7 * (B + 1) + i] = last ? (int)tot_net : I->net_off;
  }
  FAMS_CUDA(cudaMemcpyAsync(off_m, o.data(), sizeof(int) * 8 * (B + 1), cudaMemcpyHostToDevice, stream));
  FAMS_CUDA(cudaMemcpyAsync(d_inst, h.data(), sizeof(Inst) * B, cudaMemcpyHostToDevice, stream));
  FAMS_CUDA(cudaStreamSynchronize(stream));
  return FAMS_OK;
}

int Batch::check_err(const char* phase) {
  int w[3] = {0, 0, 0};
  FAMS_CUDA(cudaMemcpyAsync(w, d_err, sizeof(int) * 3, cudaMemcpyDeviceToHost, stream));
  FAMS_CUDA(cudaStreamSynchronize(stream));
  FAMS_CUDA(cudaGetLastError());
  int e = w[0];
  if (e == DERR_NONE) return FAMS_OK;
  FAMS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int) * 3, stream));
  std::string p(phase);
  if (w[1] > 0) p += " (instance " + std::to_string(w[1] - 1) + ", item " + std::to_string(w[2]) + ")";
  switch (e) {
    case DERR_BREAKDOWN: set_error(p + ": zero or non-finite pivot"); return FAMS_EBREAKDOWN;
    case DERR_CAPACITY: set_error(p + ": a local problem exceeds a compiled-in size limit"); return FAMS_ECAPACITY;
    case DERR_TIMEOUT: set_error(p + ": a bounded device wait gave up"); return FAMS_ETIMEOUT;
    case DERR_FLOATING: set_error(p + ": a dual block has no link to known basis values"); return FAMS_EINVAL;
    default: set_error(p + ": invalid input"); return FAMS_EINVAL;
  }
}

namespace {

int validate(const fams_grid& g, const fams_fracs* f, const fams_opts& o) {
  auto bad = [](const char* m) { set_error(m); return FAMS_EINVAL; };
  if (g.dim != 2 && g.dim != 3) return bad("grid.dim must be 2 or 3");
  if (g.nx < 1 || g.ny < 1 || g.nz < 1) return bad("grid sizes must be >= 1");
  if (g.dim == 2 && g.nz != 1) return bad("2D grids need nz = 1");
  if (!(g.dx > 0) || !(g.dy > 0) || !(g.dz > 0)) return bad("cell sizes must be > 0");
  int faces = g.dim == 3 ? 0x3f : 0x0f;
  if ((g.bc_mask & faces) == 0) return bad("at least one Dirichlet face is required");
  if ((long long)g.nx * g.ny * g.nz > 200000000LL) return bad("grid too large");
  if (f && f->n < 0) return bad("fracs.n < 0");
  if (f && f->n > 0 && (!f->xy || !f->kf)) return bad("fracture arrays missing");
  if (f && f->n > 0 && (!(f->aperture > 0) || !(f->h_f > 0))) return bad("aperture and h_f must be > 0");
  for (int a = 0; a < g.dim; ++a)
    if (o.coarsen[a] < 1) return bad("coarsening ratios must be >= 1");
  if (o.basis < 0 || o.basis > 3) return bad("basis must be 0..3");
  if (o.restriction != FAMS_R_FV && o.restriction != FAMS_R_FE && o.restriction != FAMS_R_MIX)
    return bad("restriction must be FAMS_R_FV, FAMS_R_FE or FAMS_R_MIX");
  if (!(o.alpha >= 0.0) || !(o.alpha < 1.0)) return bad("alpha must be in [0, 1)");
  if (o.max_iter < 0) return bad("max_iter must be >= 0");
  if (o.precision != FAMS_FP64 && o.precision != FAMS_MIXED)
    return bad("precision must be FAMS_FP64 or FAMS_MIXED");
  if (g.dim == 3 && o.frac_cz < 1) return bad("frac_cz must be >= 1");
  if (o.krylov != FAMS_KRYLOV_NONE && o.krylov != FAMS_KRYLOV_GMRES)
    return bad("krylov must be FAMS_KRYLOV_NONE or FAMS_KRYLOV_GMRES");
  if (o.krylov == FAMS_KRYLOV_GMRES && (o.restart < 1 || o.restart > FAMS_MAX_RESTART))
    return bad("GMRES restart must be in 1..FAMS_MAX_RESTART");
  if (o.prepare_flux != 0 && o.prepare_flux != 1) return bad("prepare_flux must be 0 or 1");
  if (o.merge_cap < 0) return bad("merge_cap must be >= 0");
  if (o.grid_solve < -1 || o.grid_solve > 1) return bad("grid_solve must be -1, 0 or 1");
  if (o.subblock != 0 && o.subblock != 1) return bad("subblock must be 0 or 1");
  if (o.subblock && o.precision != FAMS_FP64) return bad("subblock needs precision FAMS_FP64");
  if (o.bf16_p != 0 && o.bf16_p != 1) return bad("bf16_p must be 0 or 1");
  if (o.bf16_p && o.precision != FAMS_MIXED) return bad("bf16_p needs precision FAMS_MIXED");
  if (o.coarse_mode < 0 || o.coarse_mode > 2) return bad("coarse_mode must be 0, 1 or 2");
  return FAMS_OK;
}

// flags an entry that is not positive and finite (integer test on the bits:
// the sign bit makes negatives negative, NaN and infinity lie above the
// largest finite pattern)
__global__ void k_check_positive(const double* v, long long n, int* bad) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long b = __double_as_longlong(v[i]);
  if (!(b > 0 && b < 0x7ff0000000000000LL)) atomicExch(bad, 1);
}

// copy a small caller array (host or device memory) into host memory
int copy_to_host(void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return FAMS_OK;
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, src);
  if (e != cudaSuccess) {
    cudaGetLastError();
    at.type = cudaMemoryTypeUnregistered;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    FAMS_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return FAMS_OK;
}

// wells of the batch to host arrays in the perforation order of the flux
// output (per instance: rate wells' perforations, then pressure wells', each
// in input order), with their checks
struct HostWells {
  std::vector<int> inst, cell, wloc;   // wloc: rate-well index in the instance, -1 pressure
  std::vector<double> pi, bhp;
  std::vector<int> nw, nperf;          // per instance
  std::vector<double> rate;            // per rate well of the batch, in order
};

int read_wells(int n, const fams_grid* grids, const fams_wells* wells, HostWells& hw) {
  hw.nw.assign(n, 0);
  hw.nperf.assign(n, 0);
  if (!wells) return FAMS_OK;
  for (int i = 0; i < n; ++i) {
    const fams_wells& W = wells[i];
    if (W.n < 0) { set_error("wells.n must be >= 0"); return FAMS_EINVAL; }
    if (W.n == 0) continue;
    if (!W.perf_ptr || !W.control || !W.value) { set_error("wells arrays are null"); return FAMS_EINVAL; }
    std::vector<int> ptr(W.n + 1), ctl(W.n);
    std::vector<double> val(W.n);
    FAMS_TRY(copy_to_host(ptr.data(), W.perf_ptr, sizeof(int) * (W.n + 1)));
    FAMS_TRY(copy_to_host(ctl.data(), W.control, sizeof(int) * W.n));
    FAMS_TRY(copy_to_host(val.data(), W.value, sizeof(double) * W.n));
    if (ptr[0] != 0) { set_error("wells.perf_ptr[0] must be 0"); return FAMS_EINVAL; }
    for (int w = 0; w < W.n; ++w)
      if (ptr[w + 1] < ptr[w]) { set_error("wells.perf_ptr must not decrease"); return FAMS_EINVAL; }
    const int np = ptr[W.n];
    if (np > 0 && (!W.perf_cell || !W.perf_pi)) { set_error("wells arrays are null"); return FAMS_EINVAL; }
    std::vector<int> cells(np);
    std::vector<double> pis(np);
    FAMS_TRY(copy_to_host(cells.data(), W.perf_cell, sizeof(int) * np));
    FAMS_TRY(copy_to_host(pis.data(), W.perf_pi, sizeof(double) * np));
    const fams_grid& g = grids[i];
    const long long nm = (long long)g.nx * g.ny * (g.dim == 3 ? g.nz : 1);
    for (int w = 0; w < W.n; ++w) {
      if (ctl[w] != FAMS_WELL_RATE && ctl[w] != FAMS_WELL_PRESSURE) {
        set_error("well control must be FAMS_WELL_RATE or FAMS_WELL_PRESSURE");
        return FAMS_EINVAL;
      }
      if (!std::isfinite(val[w])) { set_error("well value must be finite"); return FAMS_EINVAL; }
      if (ctl[w] == FAMS_WELL_RATE && ptr[w + 1] == ptr[w]) {
        set_error("a rate-controlled well needs a perforation");
        return FAMS_EINVAL;
      }
      for (int k = ptr[w]; k < ptr[w + 1]; ++k) {
        if (cells[k] < 0 || cells[k] >= nm) { set_error("perforation outside the matrix"); return FAMS_EINVAL; }
        if (k > ptr[w] && cells[k] <= cells[k - 1]) {
          set_error("perforations of a well must be strictly ascending");
          return FAMS_EINVAL;
        }
        if (!(pis[k] > 0.0) || !std::isfinite(pis[k])) {
          set_error("productivity index must be positive and finite");
          return FAMS_EINVAL;
        }
      }
    }
    for (int pass = 0; pass < 2; ++pass) {   // rate wells, then pressure wells
      for (int w = 0; w < W.n; ++w) {
        if ((ctl[w] == FAMS_WELL_RATE) != (pass == 0)) continue;
        for (int k = ptr[w]; k < ptr[w + 1]; ++k) {
          hw.inst.push_back(i);
          hw.cell.push_back(cells[k]);
          hw.wloc.push_back(pass == 0 ? hw.nw[i] : -1);
          hw.pi.push_back(pis[k]);
          hw.bhp.push_back(pass == 0 ? 0.0 : val[w]);
          ++hw.nperf[i];
        }
        if (pass == 0) {
          hw.rate.push_back(val[w]);
          ++hw.nw[i];
        }
      }
    }
  }
  return FAMS_OK;
}

int upload_wells(Batch& b, const HostWells& hw) {
  b.tot_perf = (long long)hw.cell.size();
  b.tot_w = (long long)hw.rate.size();
  if (b.tot_perf == 0 && b.tot_w == 0) return FAMS_OK;
  const long long np = b.tot_perf, nw = b.tot_w;
  std::vector<int> mcell(np), mptr(b.tot_m + 1, 0), midx(np);
  for (long long k = 0; k < np; ++k) {
    mcell[k] = b.h[hw.inst[k]].m_off + hw.cell[k];
    ++mptr[mcell[k] + 1];
  }
  for (long long c = 0; c < b.tot_m; ++c) mptr[c + 1] += mptr[c];
  {
    std::vector<int> cur(mptr.begin(), mptr.end() - 1);
    for (long long k = 0; k < np; ++k) midx[cur[mcell[k]]++] = (int)k;
  }
  // [first, end) perforation of each rate well (contiguous: a rate well's
  // perforations follow each other in the perforation order)
  std::vector<int> wrange(2 * (nw + 1), 0);
  for (long long k = 0; k < np; ++k) {
    if (hw.wloc[k] < 0) continue;
    const long long gw = b.h[hw.inst[k]].w_off + hw.wloc[k];
    if (wrange[2 * gw + 1] == 0) wrange[2 * gw] = (int)k;
    wrange[2 * gw + 1] = (int)k + 1;
  }
  std::vector<int> pcell(hw.cell.begin(), hw.cell.end()), pw(hw.wloc.begin(), hw.wloc.end());
  FAMS_TRY(b.alloc((void**)&b.perf_row, sizeof(int) * (np + 1)));
  FAMS_TRY(b.alloc((void**)&b.perf_wrow, sizeof(int) * (np + 1)));
  FAMS_TRY(b.alloc((void**)&b.perf_beta, sizeof(double) * (np + 1)));
  FAMS_TRY(b.alloc((void**)&b.perf_bhp, sizeof(double) * (np + 1)));
  FAMS_TRY(b.alloc((void**)&b.mperf_ptr, sizeof(int) * (b.tot_m + 1)));
  FAMS_TRY(b.alloc((void**)&b.mperf_idx, sizeof(int) * (np + 1)));
  FAMS_TRY(b.alloc((void**)&b.wperf_range, sizeof(int) * 2 * (nw + 1)));
  FAMS_TRY(b.alloc((void**)&b.w_rate, sizeof(double) * (nw + 1)));
  // staged on the device in the rows' and beta's places; k_perf_rows
  // turns them into global rows and PI k
  FAMS_CUDA(cudaMemcpyAsync(b.perf_row, pcell.data(), sizeof(int) * np, cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.perf_wrow, pw.data(), sizeof(int) * np, cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.perf_beta, hw.pi.data(), sizeof(double) * np, cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.perf_bhp, hw.bhp.data(), sizeof(double) * np, cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.mperf_ptr, mptr.data(), sizeof(int) * (b.tot_m + 1), cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.mperf_idx, midx.data(), sizeof(int) * np, cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.wperf_range, wrange.data(), sizeof(int) * 2 * (nw + 1),
                            cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.w_rate, hw.rate.data(), sizeof(double) * nw, cudaMemcpyHostToDevice, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));   // host vectors go out of scope
  return FAMS_OK;
}

int setup_batch(int n, const fams_grid* grids, const double* const* perms, const fams_fracs* fracs,
                const fams_wells* wells, const fams_opts* opts, Batch& b) {
  HostWells hw;
  FAMS_TRY(read_wells(n, grids, wells, hw));
  b.B = n;
  FAMS_CUDA(cudaGetDevice(&b.device));
  FAMS_CUDA(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
  {
    // keep freed blocks in this process's pool for the next context (up to
    // half of the device's memory, at least POOL_KEEP bytes) instead of
    // returning them at every synchronisation (unmapping the memory of a
    // large batch, and mapping it again for the next context, cost tens of
    // milliseconds each)
    cudaMemPool_t pool;
    FAMS_CUDA(cudaDeviceGetDefaultMemPool(&pool, b.device));
    size_t dev_free = 0, dev_total = 0;
    FAMS_CUDA(cudaMemGetInfo(&dev_free, &dev_total));
    uint64_t keep = std::max<uint64_t>(POOL_KEEP, dev_total / 2);
    FAMS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    // reuse across streams only once the free has completed: the pool then
    // never makes one context's stream wait for another's
    int no = 0;
    FAMS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no));
  }
  b.h.assign(n, Inst{});
  long long m = 0, fr = 0;
  for (int i = 0; i < n; ++i) {
    const fams_grid& g = grids[i];
    const fams_opts& o = opts[i];
    Inst& I = b.h[i];
    I.dim = g.dim; I.nx = g.nx; I.ny = g.ny; I.nz = g.dim == 3 ? g.nz : 1;
    I.dx = g.dx; I.dy = g.dy; I.dz = g.dz;
    I.bc_mask = g.bc_mask & (g.dim == 3 ? 0x3f : 0x0f);
    for (int k = 0; k < 6; ++k) I.bc_val[k] = g.bc_value[k];
    int nf = fracs ? fracs[i].n : 0;
    I.aperture = nf ? fracs[i].aperture : 1.0;
    I.hf = nf ? fracs[i].h_f : 1.0;
    I.cx = o.coarsen[0]; I.cy = o.coarsen[1]; I.cz = g.dim == 3 ? o.coarsen[2] : 1;
    I.dmin = o.frac_dmin; I.fcz = std::max(1, o.frac_cz);
    I.basis = o.basis; I.restriction = o.restriction; I.precision = o.precision;
    I.max_iter = o.max_iter; I.alpha = o.alpha;
    I.krylov = o.krylov; I.restart = o.krylov == FAMS_KRYLOV_GMRES ? o.restart : 0;
    I.merge_cap = o.basis == FAMS_COUPLED ? o.merge_cap : 0;
    I.grid_solve = o.grid_solve;
    I.subblock = o.subblock;
    I.bf16_p = o.bf16_p;
    I.coarse_mode = o.coarse_mode;
    b.prepare_flux = b.prepare_flux || o.prepare_flux == 1;
    I.nm = g.nx * g.ny * I.nz;
    I.m_off = (int)m;
    I.nw = hw.nw[i];
    I.w_off = i ? b.h[i - 1].w_off + b.h[i - 1].nw : 0;
    I.nperf = hw.nperf[i];
    I.perf_off = i ? b.h[i - 1].perf_off + b.h[i - 1].nperf : 0;
    I.nfr = nf;
    I.fr_off = (int)fr;
    m += I.nm;
    fr += nf;
  }
  b.tot_m = m;
  b.tot_fr = fr;
  FAMS_TRY(b.alloc((void**)&b.off_m, sizeof(int) * 8 * (n + 1)));
  b.off_fr = b.off_m + (n + 1);
  b.off_fc = b.off_m + 2 * (n + 1);
  b.off_s = b.off_m + 3 * (n + 1);
  b.off_row = b.off_m + 4 * (n + 1);
  b.off_pair = b.off_m + 5 * (n + 1);
  b.off_nc = b.off_m + 6 * (n + 1);
  b.off_net = b.off_m + 7 * (n + 1);
  FAMS_TRY(b.alloc((void**)&b.d_inst, sizeof(Inst) * n));
  FAMS_TRY(b.alloc((void**)&b.d_err, sizeof(int) * 3));
  FAMS_CUDA(cudaMemsetAsync(b.d_err, 0, sizeof(int) * 3, b.stream));
  // inputs (host or device pointers: unified addressing picks the direction)
  FAMS_TRY(b.alloc((void**)&b.perm, sizeof(double) * (m + 1)));
  FAMS_TRY(b.alloc((void**)&b.fracs, sizeof(double) * 6 * (fr + 1)));
  FAMS_TRY(b.alloc((void**)&b.kf, sizeof(double) * (fr + 1)));
  std::vector<double> hfr(6 * (fr + 1), 0.0), hkf(fr + 1, 0.0);
  for (int i = 0; i < n; ++i) {
    const Inst& I = b.h[i];
    FAMS_CUDA(cudaMemcpyAsync(b.perm + I.m_off, perms[i], sizeof(double) * I.nm, cudaMemcpyDefault,
                              b.stream));
    if (I.nfr) {
      int w = I.dim == 3 ? 6 : 4;
      std::vector<double> xy((size_t)w * I.nfr);
      FAMS_TRY(copy_to_host(xy.data(), fracs[i].xy, sizeof(double) * w * I.nfr));
      FAMS_TRY(copy_to_host(hkf.data() + I.fr_off, fracs[i].kf, sizeof(double) * I.nfr));
      for (int f = 0; f < I.nfr; ++f)
        for (int k = 0; k < w; ++k) hfr[6 * (I.fr_off + f) + k] = xy[(size_t)w * f + k];
    }
  }
  FAMS_CUDA(cudaMemcpyAsync(b.fracs, hfr.data(), sizeof(double) * hfr.size(), cudaMemcpyHostToDevice,
                            b.stream));
  FAMS_CUDA(cudaMemcpyAsync(b.kf, hkf.data(), sizeof(double) * hkf.size(), cudaMemcpyHostToDevice,
                            b.stream));
  {
    int* dbad = nullptr;
    FAMS_TRY(b.scratch((void**)&dbad, sizeof(int)));
    FAMS_CUDA(cudaMemsetAsync(dbad, 0, sizeof(int), b.stream));
    if (m > 0)
      fams::note_launch(), k_check_positive<<<grid_for(m, 256), 256, 0, b.stream>>>(b.perm, m, dbad);
    int hbad = 0;
    FAMS_CUDA(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
    FAMS_CUDA(cudaStreamSynchronize(b.stream));
    if (hbad) {
      set_error("permeability must be positive and finite");
      return FAMS_EINVAL;
    }
    for (long long f = 0; f < fr; ++f)
      if (!(hkf[f] > 0.0) || !std::isfinite(hkf[f])) {
        set_error("fracture permeability must be positive and finite");
        return FAMS_EINVAL;
      }
  }
  FAMS_TRY(upload_wells(b, hw));
  FAMS_TRY(b.upload_inst());
  // wall time of each setup phase (every phase ends synchronised with the
  // device): geometry, system, coarse grids, basis, coarse operator, ILU(0)
  auto tick = [&](int k, double t0) {
    b.setup_ms[k] = 1e3 * (std::chrono::duration<double>(
                               std::chrono::steady_clock::now().time_since_epoch()).count() - t0);
  };
  auto now = [] {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
  };
  double t0 = now();
  FAMS_TRY(phase_geometry(b));
  tick(0, t0), t0 = now();
  FAMS_TRY(phase_system(b));
  tick(1, t0), t0 = now();
  FAMS_TRY(phase_coarse(b));
  tick(2, t0), t0 = now();
  FAMS_TRY(phase_basis(b));
  tick(3, t0), t0 = now();
  FAMS_TRY(phase_coarse_op(b, -1));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  tick(4, t0), t0 = now();
  FAMS_TRY(phase_ilu(b));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  tick(5, t0);
  FAMS_TRY(phase_alloc_work(b));
  FAMS_CUDA(cudaMemcpyAsync(b.q, b.qD, sizeof(double) * b.tot_row, cudaMemcpyDeviceToDevice, b.stream));
  FAMS_CUDA(cudaMemsetAsync(b.x, 0, sizeof(double) * b.tot_row, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  b.free_tmp();
  return FAMS_OK;
}

void destroy_batch(Batch& b) {
  if (b.stream) cudaStreamSynchronize(b.stream);
  b.free_tmp();
  for (void* p : b.owned) cudaFreeAsync(p, b.stream);
  b.owned.clear();
  if (b.stream) cudaStreamSynchronize(b.stream);
  if (b.stream) cudaStreamDestroy(b.stream);
  b.stream = nullptr;
  if (b.side) cudaStreamDestroy(b.side);
  if (b.side_done) cudaEventDestroy(b.side_done);
  b.side = nullptr;
  b.side_done = nullptr;
  for (int i = 0; i < 3; ++i)
    if (b.fk_st[i]) cudaStreamDestroy(b.fk_st[i]);
  for (int i = 0; i < 4; ++i)
    if (b.fk_ev[i]) cudaEventDestroy(b.fk_ev[i]);
  if (b.aux) cudaStreamDestroy(b.aux);
  if (b.aux_ev) cudaEventDestroy(b.aux_ev);
  if (b.aux_done) cudaEventDestroy(b.aux_done);
  b.aux = nullptr;
  b.aux_ev = b.aux_done = nullptr;
}

template <class T>
int fetch(const Batch& b, const T* src, long long n, std::vector<T>& out) {
  out.resize(n);
  if (n > 0) {
    FAMS_CUDA(cudaMemcpyAsync(out.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost, b.stream));
    FAMS_CUDA(cudaStreamSynchronize(b.stream));
  }
  return FAMS_OK;
}

}  // namespace

int make_q(Batch& b, const double* rhs_dev);
int solve_static(Batch& b, const double* rhs, double* x, double tol, fams_stats* st);

namespace {

long long faces_host(const Inst& I) {
  long long nz = I.dim == 3 ? I.nz : 1;
  return (long long)(I.nx + 1) * I.ny * nz + (long long)I.nx * (I.ny + 1) * nz +
         (I.dim == 3 ? (long long)I.nx * I.ny * (nz + 1) : 0);
}

// reconstruction of the listed instances; per-instance status (nullable)
int flux_some(Batch& b, const std::vector<int>& want, const double* const* x,
              double* const* face, double* const* nnc, int* status) {
  for (int ii : want)
    if (ii < 0 || ii >= b.B) {
      set_error("bad instance");
      return FAMS_EINVAL;
    }
  if (!b.fx) {
    long long nf = 0, nn = 0;
    for (auto& I : b.h) nf += faces_host(I), nn += (long long)I.nnc + I.nff + I.nperf;
    FAMS_TRY(b.alloc((void**)&b.fx, sizeof(double) * (b.tot_row + 1)));
    FAMS_TRY(b.alloc((void**)&b.fface, sizeof(double) * (nf + 1)));
    FAMS_TRY(b.alloc((void**)&b.fnnc, sizeof(double) * (nn + 1)));
  }
  const CoarseHost* ch = nullptr;
  FAMS_TRY(flux_prepare(b, &ch));
  std::vector<int> list;
  std::vector<int> slot;  // position of each wanted instance in the call's arrays
  int result = FAMS_OK;
  for (size_t k = 0; k < want.size(); ++k) {
    int ii = want[k];
    if (ch->bad[ii]) {
      if (status) status[k] = FAMS_EBREAKDOWN;
      if (result == FAMS_OK)
        set_error("instance " + std::to_string(ii) + ": the finite-volume coarse system is "
                  "numerically singular (zero pivot at LU step " + std::to_string(ch->bad[ii] - 1) +
                  "); no conservative reconstruction");
      result = FAMS_EBREAKDOWN;
      continue;
    }
    if (status) status[k] = FAMS_OK;
    list.push_back(ii);
    slot.push_back((int)k);
  }
  std::vector<long long> foff(list.size() + 1, 0), noff(list.size() + 1, 0);
  for (size_t k = 0; k < list.size(); ++k) {
    const Inst& I = b.h[list[k]];
    foff[k + 1] = foff[k] + faces_host(I);
    noff[k + 1] = noff[k] + I.nnc + I.nff + I.nperf;
    FAMS_CUDA(cudaMemcpyAsync(b.fx + I.row_off, x[slot[k]], sizeof(double) * I.n,
                              cudaMemcpyDefault, b.stream));
  }
  int s = run_flux(b, list, b.fx, b.fface, foff, b.fnnc, noff);
  if (s != FAMS_OK) return s;
  for (size_t k = 0; k < list.size(); ++k) {
    long long nf = foff[k + 1] - foff[k], nn = noff[k + 1] - noff[k];
    FAMS_CUDA(cudaMemcpyAsync(face[slot[k]], b.fface + foff[k], sizeof(double) * nf,
                              cudaMemcpyDefault, b.stream));
    if (nn > 0)
      FAMS_CUDA(cudaMemcpyAsync(nnc[slot[k]], b.fnnc + noff[k], sizeof(double) * nn,
                                cudaMemcpyDefault, b.stream));
  }
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  return result;
}

}  // namespace

}  // namespace fams

using namespace fams;

extern "C" {

int fams_setup_batch(int n, const fams_grid* grids, const double* const* perms,
                     const fams_fracs* fracs, const fams_opts* opts, fams_ctx** out) {
  return fams_setup_batch_wells(n, grids, perms, fracs, nullptr, opts, out);
}

int fams_setup_batch_wells(int n, const fams_grid* grids, const double* const* perms,
                           const fams_fracs* fracs, const fams_wells* wells,
                           const fams_opts* opts, fams_ctx** out) {
  if (!out || n < 1 || !grids || !perms || !opts) {
    set_error("null argument or n < 1");
    return FAMS_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    FAMS_TRY(validate(grids[i], fracs ? &fracs[i] : nullptr, opts[i]));
    if (!perms[i]) { set_error("perm is null"); return FAMS_EINVAL; }
  }
  fams_ctx* c = new fams_ctx();
  int s = setup_batch(n, grids, perms, fracs, wells, opts, c->b);
  if (s != FAMS_OK) {
    destroy_batch(c->b);
    delete c;
    return s;
  }
  *out = c;
  return FAMS_OK;
}

int fams_setup(const fams_grid* grid, const double* perm, const fams_fracs* fracs,
               const fams_opts* opts, fams_ctx** out) {
  if (!grid || !perm || !opts) {
    set_error("null argument");
    return FAMS_EINVAL;
  }
  const double* perms[1] = {perm};
  return fams_setup_batch(1, grid, perms, fracs, opts, out);
}

int fams_setup_wells(const fams_grid* grid, const double* perm, const fams_fracs* fracs,
                     const fams_wells* wells, const fams_opts* opts, fams_ctx** out) {
  if (!grid || !perm || !opts) {
    set_error("null argument");
    return FAMS_EINVAL;
  }
  const double* perms[1] = {perm};
  return fams_setup_batch_wells(1, grid, perms, fracs, wells, opts, out);
}

int fams_sizes_wells(const fams_ctx* ctx, int inst, int* n_well, int* n_perf) {
  if (!ctx || inst < 0 || inst >= ctx->b.B) { set_error("bad context or instance"); return FAMS_EINVAL; }
  if (n_well) *n_well = ctx->b.h[inst].nw;
  if (n_perf) *n_perf = ctx->b.h[inst].nperf;
  return FAMS_OK;
}

int fams_num_instances(const fams_ctx* ctx) { return ctx ? ctx->b.B : 0; }

int fams_sizes(const fams_ctx* ctx, int inst, int* n_matrix, int* n_frac, int* n_coarse,
               int* n_faces, int* n_nnc) {
  if (!ctx || inst < 0 || inst >= ctx->b.B) { set_error("bad context or instance"); return FAMS_EINVAL; }
  const Inst& I = ctx->b.h[inst];
  int nz = I.dim == 3 ? I.nz : 1;
  if (n_matrix) *n_matrix = I.nm;
  if (n_frac) *n_frac = I.nf;
  if (n_coarse) *n_coarse = I.nc;
  if (n_faces)
    *n_faces = (I.nx + 1) * I.ny * nz + I.nx * (I.ny + 1) * nz + (I.dim == 3 ? I.nx * I.ny * (nz + 1) : 0);
  if (n_nnc) *n_nnc = I.nnc + I.nff + I.nperf;
  return FAMS_OK;
}

}  // extern "C"

namespace {

// the iteration on the listed instances (rhs, x and st indexed like list);
// instances not listed keep their state and launch nothing
int solve_list(fams_ctx* ctx, const std::vector<int>& list, const double* const* rhs,
               double* const* x, double tol, fams_stats* st) {
  if (!ctx || !x) { set_error("null argument"); return FAMS_EINVAL; }
  if (!(tol >= 0.0)) { set_error("tol must be >= 0"); return FAMS_EINVAL; }
  Batch& b = ctx->b;
  const int nl = (int)list.size();
  const bool all = nl == b.B;
  std::vector<int> act(b.B, 0);
  for (int k = 0; k < nl; ++k) {
    const int i = list[k];
    if (i < 0 || i >= b.B || act[i]) { set_error("bad or repeated instance in the list"); return FAMS_EINVAL; }
    if (!x[k]) { set_error("x is null"); return FAMS_EINVAL; }
    act[i] = 1;
  }
  if (nl == 0) return FAMS_OK;
  int* d_act = nullptr;
  if (!all) {
    if (whole_gpu(b)) { set_error("a whole-GPU context has one instance"); return FAMS_EINVAL; }
    if (!b.d_active) FAMS_TRY(b.alloc((void**)&b.d_active, sizeof(int) * b.B));
    FAMS_CUDA(cudaMemcpyAsync(b.d_active, act.data(), sizeof(int) * b.B, cudaMemcpyHostToDevice,
                              b.stream));
    d_act = b.d_active;
  }
  // rhs staged in the dp work vector
  FAMS_CUDA(cudaMemsetAsync(b.dp, 0, sizeof(double) * b.tot_row, b.stream));
  for (int k = 0; k < nl; ++k) {
    const Inst& I = b.h[list[k]];
    if (rhs && rhs[k])
      FAMS_CUDA(cudaMemcpyAsync(b.dp + I.row_off, rhs[k], sizeof(double) * I.n, cudaMemcpyDefault,
                                b.stream));
    FAMS_CUDA(cudaMemcpyAsync(b.x + I.row_off, x[k], sizeof(double) * I.n, cudaMemcpyDefault,
                              b.stream));
  }
  FAMS_TRY(make_q(b, b.dp));
  float ms = 0.f;
  FAMS_TRY(run_solve(b, tol, &ms, d_act));
  std::vector<double> stat;
  FAMS_TRY(fetch(b, b.stat, (long long)STAT_W * b.B, stat));
  int status = FAMS_OK;
  for (int k = 0; k < nl; ++k) {
    const int i = list[k];
    const Inst& I = b.h[i];
    FAMS_CUDA(cudaMemcpyAsync(x[k], b.x + I.row_off, sizeof(double) * I.n, cudaMemcpyDefault,
                              b.stream));
    if (st) {
      st[k].iterations = (int)stat[STAT_W * i];
      st[k].rel_residual = stat[STAT_W * i + 1];
      st[k].converged = stat[STAT_W * i + 2] > 0.5;
      st[k].solve_ms = ms;
    }
    if (stat[STAT_W * i + STAT_BAD] > 0.5) {
      if (status != FAMS_EBREAKDOWN)
        set_error("instance " + std::to_string(i) + ": numerically singular coarse system "
                  "(zero pivot at LU step " + std::to_string(b.csh[0].bad[i] - 1) + ")");
      status = FAMS_EBREAKDOWN;
    } else if (!std::isfinite(stat[STAT_W * i + 1])) {
      set_error("the iteration produced a non-finite residual");
      status = FAMS_EBREAKDOWN;
    } else if (stat[STAT_W * i + 2] < 0.5 && status == FAMS_OK) {
      set_error("max_iter reached before the tolerance");
      status = FAMS_ENOCONV;
    }
  }
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  return status;
}

}  // namespace

extern "C" {

int fams_solve_batch(fams_ctx* ctx, const double* const* rhs, double* const* x, double tol,
                     fams_stats* st) {
  if (!ctx) { set_error("null argument"); return FAMS_EINVAL; }
  std::vector<int> all(ctx->b.B);
  for (int i = 0; i < ctx->b.B; ++i) all[i] = i;
  return solve_list(ctx, all, rhs, x, tol, st);
}

int fams_solve_subset(fams_ctx* ctx, int n_list, const int* list, const double* const* rhs,
                      double* const* x, double tol, fams_stats* st) {
  if (!ctx || n_list < 0 || (n_list > 0 && !list)) { set_error("null argument"); return FAMS_EINVAL; }
  return solve_list(ctx, std::vector<int>(list, list + n_list), rhs, x, tol, st);
}

int fams_solve(fams_ctx* ctx, const double* rhs, double* x, double tol, fams_stats* st) {
  if (!ctx || ctx->b.B != 1) { set_error("fams_solve needs a single-instance context"); return FAMS_EINVAL; }
  const double* r[1] = {rhs};
  double* xx[1] = {x};
  return fams_solve_batch(ctx, r, xx, tol, st);
}

int fams_solve_static(fams_ctx* ctx, const double* rhs, double* x, double tol, fams_stats* st) {
  if (!ctx || ctx->b.B != 1) {
    set_error("fams_solve_static needs a single-instance context");
    return FAMS_EINVAL;
  }
  if (ctx->b.h[0].krylov != FAMS_KRYLOV_NONE || ctx->b.h[0].precision != FAMS_FP64) {
    set_error("fams_solve_static runs the FP64 Table 1 loop only (krylov = FAMS_KRYLOV_NONE, "
              "precision = FAMS_FP64)");
    return FAMS_EINVAL;
  }
  if (!x) { set_error("x is null"); return FAMS_EINVAL; }
  if (!(tol >= 0.0)) { set_error("tol must be >= 0"); return FAMS_EINVAL; }
  return solve_static(ctx->b, rhs, x, tol, st);
}

int fams_update_batch(fams_ctx* ctx, const double* const* mobility_scale) {
  if (!ctx) { set_error("null argument"); return FAMS_EINVAL; }
  return phase_update(ctx->b, mobility_scale);
}

int fams_update_basis(fams_ctx* ctx, const double* const* mobility_scale, double eps,
                      int* rebuilt) {
  if (!ctx) { set_error("null argument"); return FAMS_EINVAL; }
  if (eps != eps) { set_error("eps is NaN"); return FAMS_EINVAL; }
  return phase_update_basis(ctx->b, mobility_scale, eps, rebuilt);
}

int fams_update(fams_ctx* ctx, const double* mobility_scale) {
  if (!ctx || ctx->b.B != 1) { set_error("fams_update needs a single-instance context"); return FAMS_EINVAL; }
  const double* s[1] = {mobility_scale};
  return phase_update(ctx->b, s);
}

int fams_flux(fams_ctx* ctx, int inst, const double* x, double* face_flux, double* nnc_flux) {
  if (!ctx || !x || !face_flux || !nnc_flux || inst < 0 || inst >= ctx->b.B) {
    set_error("null argument or bad instance");
    return FAMS_EINVAL;
  }
  const double* xs[1] = {x};
  double* fs[1] = {face_flux};
  double* ns[1] = {nnc_flux};
  return flux_some(ctx->b, std::vector<int>{inst}, xs, fs, ns, nullptr);
}

int fams_flux_batch(fams_ctx* ctx, const double* const* x, double* const* face_flux,
                    double* const* nnc_flux, int* status) {
  if (!ctx || !x || !face_flux || !nnc_flux) {
    set_error("null argument");
    return FAMS_EINVAL;
  }
  std::vector<int> all(ctx->b.B);
  for (int i = 0; i < ctx->b.B; ++i) {
    if (!x[i] || !face_flux[i] || !nnc_flux[i]) {
      set_error("null buffer");
      return FAMS_EINVAL;
    }
    all[i] = i;
  }
  return flux_some(ctx->b, all, x, face_flux, nnc_flux, status);
}

int fams_query(const fams_ctx* ctx, int inst, int what, void* out, long long cap) {
  if (!ctx || inst < 0 || inst >= ctx->b.B) { set_error("bad context or instance"); return FAMS_EINVAL; }
  const Batch& b = ctx->b;
  const Inst& I = b.h[inst];
  std::vector<int> vi;
  std::vector<double> vd;
  bool isint = true;
  auto ints = [&](const int* src, long long n, long long sub) -> int {
    FAMS_TRY(fetch(b, src, n, vi));
    for (auto& v : vi) v -= (int)sub;
    return FAMS_OK;
  };
  auto dbls = [&](const double* src, long long n) -> int {
    isint = false;
    return fetch(b, src, n, vd);
  };
  int pbeg = 0, pend = 0;
  switch (what) {
    case FAMS_Q_NNC_FRAC: FAMS_TRY(ints(b.nnc_row_f + I.nnc_off, I.nnc, I.row_off + I.nm)); break;
    case FAMS_Q_NNC_MATRIX: FAMS_TRY(ints(b.nnc_row_m + I.nnc_off, I.nnc, I.row_off)); break;
    case FAMS_Q_NNC_AREA: FAMS_TRY(dbls(b.nnc_area + I.nnc_off, I.nnc)); break;
    case FAMS_Q_NNC_DIST: FAMS_TRY(dbls(b.nnc_dist + I.nnc_off, I.nnc)); break;
    case FAMS_Q_FF_A: FAMS_TRY(ints(b.ff_a + I.ff_off, I.nff, I.row_off + I.nm)); break;
    case FAMS_Q_FF_B: FAMS_TRY(ints(b.ff_b + I.ff_off, I.nff, I.row_off + I.nm)); break;
    case FAMS_Q_FF_T: FAMS_TRY(dbls(b.ff_T + I.ff_off, I.nff)); break;
    case FAMS_Q_A_ROWPTR: FAMS_TRY(ints(b.rowptr + I.row_off, I.n + 1, I.nnz_off)); break;
    case FAMS_Q_A_COL: FAMS_TRY(ints(b.col + I.nnz_off, I.nnz, I.row_off)); break;
    case FAMS_Q_A_VAL: FAMS_TRY(dbls(b.val + I.nnz_off, I.nnz)); break;
    case FAMS_Q_Q: FAMS_TRY(dbls(b.q + I.row_off, I.n)); break;
    case FAMS_Q_RANK: FAMS_TRY(ints(b.rank + I.row_off, I.n, 0)); break;
    case FAMS_Q_PRIMAL: FAMS_TRY(ints(b.primal + I.row_off, I.n, 0)); break;
    case FAMS_Q_NODE_CELL: FAMS_TRY(ints(b.node_cell + I.nc_off, I.nc, I.row_off)); break;
    case FAMS_Q_P_ROWPTR:
    case FAMS_Q_P_COL:
    case FAMS_Q_P_VAL: {
      std::vector<int> pp;
      FAMS_TRY(fetch(b, b.p_ptr + I.row_off, I.n + 1, pp));
      pbeg = pp[0];
      pend = pp[I.n];
      if (what == FAMS_Q_P_ROWPTR) {
        vi = pp;
        for (auto& v : vi) v -= pbeg;
      } else if (what == FAMS_Q_P_COL) {
        FAMS_TRY(ints(b.p_col + pbeg, pend - pbeg, 0));
      } else {
        FAMS_TRY(dbls(b.p_val + pbeg, pend - pbeg));
      }
      break;
    }
    case FAMS_Q_AC: FAMS_TRY(dbls(b.cs[0].Ac + b.csh[0].ac_off[inst], (long long)I.nc * I.nc)); break;
    case FAMS_Q_ILU_VAL: FAMS_TRY(dbls(b.ilu + I.nnz_off, I.nnz)); break;
    case FAMS_Q_LEVELS: vi.assign(1, I.nlev); break;
    case FAMS_Q_COARSE_PERM: FAMS_TRY(ints(b.cs[0].perm + I.nc_off, I.nc, 0)); break;
    case FAMS_Q_COARSE_IPIV: FAMS_TRY(ints(b.cs[0].ipiv + I.nc_off, I.nc, 0)); break;
    case FAMS_Q_BAND_KLKU: vi = {b.csh[0].kl[inst], b.csh[0].ku[inst]}; break;
    case FAMS_Q_BAND:
      FAMS_TRY(dbls(b.cs[0].band + b.csh[0].band_off[inst],
                    (long long)(2 * b.csh[0].kl[inst] + b.csh[0].ku[inst] + 1) * I.nc));
      break;
    case FAMS_Q_STAGE_CYCLES: FAMS_TRY(dbls(b.stat + STAT_W * inst + 4, 6)); break;
    case FAMS_Q_SETUP_MS: isint = false; vd.assign(b.setup_ms, b.setup_ms + 6); break;
    case FAMS_Q_CLASS_COUNTS: vi.assign(b.class_cnt, b.class_cnt + 8); break;
    case FAMS_Q_LAST_DP1: FAMS_TRY(dbls(b.dp + I.row_off, I.n)); break;
    case FAMS_Q_LAST_DP2: FAMS_TRY(dbls(b.y + I.row_off, I.n)); break;
    case FAMS_Q_LAST_RC: FAMS_TRY(dbls(b.rc + I.nc_off, I.nc)); break;
    case FAMS_Q_LAST_EC: FAMS_TRY(dbls(b.ec + I.nc_off, I.nc)); break;
    case FAMS_Q_HISTORY: {
      std::vector<double> st;
      FAMS_TRY(fetch(b, b.stat + STAT_W * inst, STAT_W, st));
      FAMS_TRY(dbls(b.hist + (long long)inst * (b.hist_len), (long long)st[0] + 1));
      break;
    }
    default: set_error("unknown query"); return FAMS_EINVAL;
  }
  long long n = isint ? (long long)vi.size() : (long long)vd.size();
  if (!out) return (int)n;
  if (cap < n) { set_error("output buffer too small"); return FAMS_EINVAL; }
  size_t bytes = isint ? sizeof(int) * n : sizeof(double) * n;
  const void* src = isint ? (const void*)vi.data() : (const void*)vd.data();
  if (n > 0) FAMS_CUDA(cudaMemcpy(out, src, bytes, cudaMemcpyDefault));
  return (int)n;
}

void fams_destroy(fams_ctx* ctx) {
  if (!ctx) return;
  destroy_batch(ctx->b);
  delete ctx;
}

const char* fams_strerror(int s) {
  switch (s) {
    case FAMS_OK: return "ok";
    case FAMS_EINVAL: return "invalid argument or unsupported input";
    case FAMS_ENOMEM: return "device memory allocation failed";
    case FAMS_ENOCONV: return "iteration did not reach the tolerance";
    case FAMS_EBREAKDOWN: return "zero or non-finite pivot";
    case FAMS_ETIMEOUT: return "bounded device wait timed out";
    case FAMS_ECUDA: return "CUDA runtime error";
    case FAMS_ECAPACITY: return "problem exceeds a compiled-in capacity";
    default: return "unknown status";
  }
}

const char* fams_last_error(void) { return g_err.c_str(); }

long long fams_launch_count(void) { return g_launches.load(); }

long long fams_alloc_count(void) { return g_allocs.load(); }

}  // extern "C"
