// The device state of a batch of independent F-AMS instances.  Every array
// is the concatenation of the instances' arrays (a block-diagonal system);
// Inst::*_off give each instance's slice.
#pragma once
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace fams {

// Coarse system of every instance of a batch (device pointers; per-instance
// arrays have B entries, per-coarse-unknown arrays tot_nc).
struct CoarseSys {
  double* Ac = nullptr;         // dense R A P, row-major, at ac_off[i]
  long long* ac_off = nullptr;
  double* band = nullptr;       // band LU factors (column-major, ldab = 2kl+ku+1)
  long long* band_off = nullptr;
  int* kl = nullptr;            // lower / upper bandwidth after reordering
  int* ku = nullptr;
  int* ipiv = nullptr;          // pivot rows (band positions)
  int* perm = nullptr;          // band position -> coarse index
  int* bad = nullptr;           // per instance: 0, or 1 + the LU step with a zero pivot
  // factors without row interchanges (LDL^T): inverses of the diagonal
  // blocks of COARSE_NB band positions, L_bb^-1 then U_bb^-1 per block,
  // column-major, for the blocked band solve
  int* nopiv = nullptr;         // per instance: 1 if factored without interchanges
  double* binv = nullptr;
  long long* binv_off = nullptr;
};

constexpr int COARSE_NB = 32;   // band positions per block of the blocked band solve

struct CoarseHost {
  std::vector<long long> ac_off, band_off;
  long long band_tot = 0;
  std::vector<int> kl, ku;
  std::vector<int> bad;         // host copy of CoarseSys::bad
  std::vector<long long> binv_off;
};

struct Batch {
  int B = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;        // second stream: the R^FV system built beside a solve
  cudaEvent_t side_done = nullptr;
  cudaStream_t aux = nullptr;         // concurrent band LU passes of disjoint instance sets
  cudaEvent_t aux_ev = nullptr, aux_done = nullptr;
  cudaStream_t fk_st[3] = {nullptr, nullptr, nullptr};   // size classes of local solves
  cudaEvent_t fk_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool prepare_flux = false;          // some instance asked for it (fams_opts.prepare_flux)
  int device = 0;
  std::vector<Inst> h;          // host copy of the descriptors
  Inst* d_inst = nullptr;       // device copy
  int* d_active = nullptr;      // instances a subset solve runs (allocated on first use)
  int* d_err = nullptr;         // device status word
  std::vector<void*> owned;     // freed by fams_destroy
  std::vector<void*> tmp;       // freed at the end of setup

  // per-item-kind instance offsets on the device (B+1 each)
  int* off_m = nullptr;    // matrix cells
  int* off_fr = nullptr;   // input fractures
  int* off_fc = nullptr;   // fracture cells
  int* off_s = nullptr;    // strike cells
  int* off_row = nullptr;  // unknowns
  int* off_pair = nullptr; // fracture pairs
  int* off_nc = nullptr;   // coarse unknowns
  int* off_net = nullptr;  // fracture networks

  // totals
  long long tot_m = 0, tot_fr = 0, tot_fc = 0, tot_s = 0, tot_row = 0, tot_pair = 0,
            tot_nnc = 0, tot_ff = 0, tot_nc = 0, tot_net = 0, tot_nnz = 0, tot_pnnz = 0;

  // ---- wells (none: all null, tot_perf = 0) ----
  long long tot_w = 0, tot_perf = 0;   // rate-controlled wells, perforations
  int* perf_row = nullptr;     // per perforation: global row of the perforated matrix cell
  int* perf_wrow = nullptr;    // ... global row of its rate well, -1 for a pressure well
  double* perf_beta = nullptr; // ... PI k of the cell
  double* perf_bhp = nullptr;  // ... bottom-hole pressure (pressure wells)
  int* mperf_ptr = nullptr;    // per global matrix cell: its perforations (tot_m + 1)
  int* mperf_idx = nullptr;
  int* wperf_range = nullptr;  // per rate well: [first, end) of its perforations
  double* w_rate = nullptr;    // per rate well: total injection rate
  // ---- inputs ----
  double* perm = nullptr;      // tot_m
  double* fracs = nullptr;     // 6 per input fracture
  double* kf = nullptr;        // per input fracture
  // ---- geometry ----
  double* seg = nullptr;       // 4 per input fracture (clipped)
  int* f_ns = nullptr;         // strike cells per fracture
  int* f_k0 = nullptr;         // first layer (3D)
  int* f_nk = nullptr;         // layers (3D), 1 in 2D
  int* f_cfirst = nullptr;     // global fracture-cell index of the first cell
  int* f_sfirst = nullptr;     // global strike index of the first strike cell
  int* s_ovcnt = nullptr;      // overlaps per strike cell
  int* s_ovcol = nullptr;      // MAX_OVERLAP per strike cell: 2D column index
  double* s_ovlen = nullptr;   // overlap length
  double* s_ovdist = nullptr;  // <d>
  int* nnc_first = nullptr;    // per fracture cell: first connection (tot_fc+1)
  int* ff_first = nullptr;     // per fracture cell: first link where it is the lower cell
  int* nnc_row_f = nullptr;    // global row of the fracture cell
  int* nnc_row_m = nullptr;    // global row of the matrix cell
  double* nnc_T = nullptr;     // CI * k_m
  double* nnc_area = nullptr;
  double* nnc_dist = nullptr;
  int* ff_a = nullptr;         // global rows, a < b
  int* ff_b = nullptr;
  double* ff_T = nullptr;
  int* inter_hit = nullptr;    // per pair: 1 if the segments cross
  int* inter_sa = nullptr;     // strike cell index within fracture a
  int* inter_sb = nullptr;
  double* inter_T = nullptr;
  // ---- fine system ----
  int* rowptr = nullptr;       // tot_row + 1
  int* col = nullptr;          // global column indices
  double* val = nullptr;
  int* diag = nullptr;         // position of the diagonal in each row
  double* TD = nullptr;        // Dirichlet half transmissibility per row
  double* qD = nullptr;        // Dirichlet part of q
  // time-step update: mobility scale per row and the setup-time values it
  // scales (allocated by the first update)
  double* mob = nullptr;
  double* mob_basis = nullptr;   // mobility scales the current P was built with (null: setup's)
  double* val0 = nullptr;
  double* TD0 = nullptr;
  double* qD0 = nullptr;
  double* nnc_T0 = nullptr;
  double* ff_T0 = nullptr;
  // ---- coarse grids ----
  int* rank = nullptr;         // per row
  int* primal = nullptr;       // per row: instance-local coarse index
  int* node_cell = nullptr;    // per coarse unknown: global row
  int* s_net = nullptr;        // per strike cell: global network index
  int* s_prim = nullptr;       // per strike cell: network-local block
  int* s_vert = nullptr;       // per strike cell: 1 if coarse node
  int* net_nv = nullptr;       // vertices per network
  int* net_k0 = nullptr;       // layer range of each network (3D)
  int* net_nk = nullptr;
  int* net_base = nullptr;     // instance-local coarse index of the network's first node
  // ---- prolongation ----
  int* p_ptr = nullptr;        // CSR of P, instance-local columns
  int* p_col = nullptr;
  double* p_val = nullptr;
  int* pt_ptr = nullptr;       // CSR of P^T (rows = global coarse index)
  int* pt_col = nullptr;       // global fine rows
  double* pt_val = nullptr;
  // the flux reconstruction's P: the basis functions before truncation (its
  // finite-volume stage, Sec. 3.2); the same arrays as P when no instance
  // truncates (pf_alias)
  int* pf_ptr = nullptr;
  int* pf_col = nullptr;
  double* pf_val = nullptr;
  bool pf_alias = true;
  int* blk_ptr = nullptr;      // cells of each primal block (global coarse index)
  int* blk_cell = nullptr;
  std::vector<int> h_blk_ptr;  // host copy of blk_ptr (taken on the first reconstruction)
  int* blk_bw = nullptr;       // per primal block: bandwidths of its local problem
  std::vector<int> h_blk_bw;
  // ---- coarse system: [0] the iteration's restriction, [1] R^FV for the
  // flux reconstruction when the iteration uses R^FE ----
  CoarseSys cs[2];
  CoarseHost csh[2];
  // ---- ILU(0) ----
  double* ilu = nullptr;       // factors in the pattern of A
  int* lev_ptr = nullptr;      // per instance: nlev+1 offsets (Inst-local slice)
  int* lev_rows = nullptr;     // global rows grouped by level
  int* lev_off = nullptr;      // per instance offset into lev_ptr
  // the factors again in level order (position t of lev_rows), structure of
  // arrays, PK entries of each triangle inline, for the sweeps
  int* pk_pos = nullptr;       // row -> position t
  int* pk_nl = nullptr;        // L entries of the row
  int* pk_lp = nullptr;        // first L entry in the CSR (for entries beyond PK)
  int* pk_lc = nullptr;        // PK x tot_row neighbours, as level positions
  double* pk_lv = nullptr;     // PK x tot_row values
  int* pk_nu = nullptr;        // U entries right of the diagonal
  int* pk_uc = nullptr;
  double* pk_uv = nullptr;
  double* pk_ud = nullptr;     // reciprocal of the U diagonal
  double* ylev = nullptr;      // sweep right-hand side in level order
  double* xlev = nullptr;      // base + multiscale correction in level order (U sweep)
  // the sub-block smoothing stage (instances with fams_opts.subblock): ILU(0)
  // of A without its cross-medium entries, in A's pattern and level order
  double* ilu_b = nullptr;
  double* pk_lv_b = nullptr;
  double* pk_uv_b = nullptr;
  double* pk_ud_b = nullptr;
  // ---- iteration work vectors ----
  double* q = nullptr;
  double* x = nullptr;
  double* r = nullptr;
  double* dp = nullptr;
  double* y = nullptr;
  double* rc = nullptr;
  double* ec = nullptr;
  double* stat = nullptr;      // per instance: 4 doubles (iters, relres, converged, qnorm)
  double* hist = nullptr;      // per instance: relative residual after each sweep
  double* krylov = nullptr;    // GMRES bases of the instances that use GMRES
  // whole-GPU solve of a single large instance (solve_grid.cu): A_c^-1 of
  // the iteration's coarse system (nc x nc, row-major), its validity, the
  // grid barrier and the partial sums of the grid reductions
  double* ainv = nullptr;
  bool ainv_ready = false;
  void* gbar = nullptr;
  double* gpart = nullptr;
  int gpart_n = 0;
  // mixed precision: FP32 copies of P, P^T and the ILU(0) factors (plain and
  // level-ordered), the saved iterate, the FP32 sweep vectors and the FP64
  // restart vectors Z of flexible GMRES
  float* p_val32 = nullptr;
  float* pt_val32 = nullptr;
  unsigned short* p_val16 = nullptr;    // BF16 storage of P and P^T (fams_opts.bf16_p)
  unsigned short* pt_val16 = nullptr;
  float* ilu32 = nullptr;
  float* pk_lv32 = nullptr;
  float* pk_uv32 = nullptr;
  float* pk_ud32 = nullptr;
  double* xs = nullptr;
  float* yf = nullptr;
  float* ylevf = nullptr;
  double* krylov_z = nullptr;
  long long hist_len = 0;      // max_iter + 1 of the batch
  // flux (FV coarse factor built on first use)
  bool fv_ready = false;       // R^FV coarse system current
  bool fv_built = false;       // ... and allocated (a time-step update only refactors it)
  double setup_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // per setup phase, wall time
  // local problems solved per size class (one warp, 128-thread CTA, 256-thread
  // CTA in shared memory, 512-thread CTA on a global workspace): dual blocks
  // of the basis stages [0..3], primal blocks of the flux reconstruction [4..7]
  int class_cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // flux reconstruction buffers (allocated on first use): iterates and outputs
  double* fx = nullptr;
  double* fface = nullptr;
  double* fnnc = nullptr;

  // Device memory is stream-ordered (cudaMallocAsync on the context's
  // stream, from the device's memory pool): unlike cudaMalloc/cudaFree it
  // never synchronises the device, so contexts on other streams (the
  // request server's micro-batches) keep running.
  int alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMallocAsync(p, bytes, stream);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
      return FAMS_ENOMEM;
    }
    note_alloc();
    owned.push_back(*p);
    return FAMS_OK;
  }
  int scratch(void** p, size_t bytes) {
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMallocAsync(p, bytes, stream);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
      return FAMS_ENOMEM;
    }
    note_alloc();
    tmp.push_back(*p);
    return FAMS_OK;
  }
  void free_tmp() {
    for (void* p : tmp) cudaFreeAsync(p, stream);
    tmp.clear();
  }
  // free one owned array (stream-ordered) before it is built anew
  template <class T>
  void release(T*& p) {
    if (!p) return;
    void* v = static_cast<void*>(p);
    cudaFreeAsync(v, stream);
    owned.erase(std::remove(owned.begin(), owned.end(), v), owned.end());
    p = nullptr;
  }
  int upload_inst();
  int check_err(const char* phase);
};

// util.cu
int exclusive_scan(Batch& b, const int* in, int* out, long long n, long long* total);
// out[i] = src[idx[i]] for i < n, on the host (idx in device memory)
int take_ints(Batch& b, const int* src, const int* idx, int n, std::vector<int>& out);
// whether any of v[0..n) is negative
int any_negative(Batch& b, const int* v, long long n, bool* res);
// k (<= 3) extra streams that start after the work queued on b.stream so far,
// and the join that makes b.stream wait for them
int fork_streams(Batch& b, int k, cudaStream_t* out);
int join_streams(Batch& b, int k);
int sort_segments(Batch& b, const int* ptr, int nseg, int* key, double* val, bool strict);
int transpose(Batch& b, const int* rowptr, const int* col, const double* val, int nrows,
              int ncols, long long nnz, int** tptr, int** tcol, double** tval, bool keep);

// phases (each file)
int phase_geometry(Batch& b);     // geometry.cu
int phase_system(Batch& b);       // system.cu: CSR of A, q_D
int phase_coarse(Batch& b);       // coarse.cu: matrix blocks, networks, BFS, ranks
// basis.cu: P.  marked (device, per row; null: every block) selects the
// adaptive update: only dual blocks holding a marked row, or reading a row
// solved again in an earlier stage, are solved (rows flagged in rec); the
// others keep their rows of the untruncated P of the last build (pf_*)
int phase_basis(Batch& b, const int* marked = nullptr, int* rec = nullptr, int* n_solved = nullptr);
int phase_coarse_op(Batch& b, int restriction);  // coarseop.cu: R A P, band LU
// R A P with the prolongation (p_ptr, p_col, p_val): P, or the reconstruction's
int build_coarse_system(Batch& b, CoarseSys& cs, int mode, CoarseHost& ch, bool reuse,
                        const int* p_ptr, const int* p_col, const double* p_val);
int phase_update(Batch& b, const double* const* scale);
int phase_update_basis(Batch& b, const double* const* scale, double eps, int* rebuilt);
int ilu_refactor(Batch& b);                               // ilu.cu
int refresh_mixed(Batch& b);                              // solve.cu
int phase_ilu(Batch& b);          // ilu.cu
int phase_alloc_work(Batch& b);   // solve.cu
// active: device array, 1 per instance to solve (null: all)
int run_solve(Batch& b, double tol, float* ms, const int* active = nullptr);   // solve.cu
// solve_grid.cu: a single-instance context whose iteration runs on every SM
constexpr long long GRID_SOLVE_ROWS = 1LL << 18;
bool whole_gpu(const Batch& b);       // single instance, large or asked for: every SM
bool one_cta_fits(const Batch& b, int nc, int kl, int ku, int m);   // solve.cu
bool solve_on_grid(const Batch& b);   // ... and its iteration is FP64 GMRES
int run_solve_grid(Batch& b, double tol, float* ms);
int ilu_factor_grid(Batch& b, double* F);   // ILU(0) factorisation (values in F) on every SM
int band_lu_grid(Batch& b, CoarseSys& cs, CoarseHost& ch);   // coarse band LU on every SM
// flux.cu
int flux_prepare(Batch& b, const CoarseHost** ch);
int flux_beside(Batch& b, cudaEvent_t ready);   // flux.cu: flux_prepare on the side stream
int run_flux(Batch& b, const std::vector<int>& list, const double* x, double* face,
             const std::vector<long long>& foff, double* nnc, const std::vector<long long>& noff);

}  // namespace fams
