/*
 * fams.h - C ABI of libfams, a GB300 (sm_103a) implementation of the F-AMS
 * two-stage pressure solver for heterogeneous porous media with embedded
 * discrete fractures (Tene, Al Kobaisi, Hajibeygi, arXiv 1705.05784).
 *
 * Conventions shared by every call
 *  - Every function returns an int status: FAMS_OK (0) or a negative FAMS_E*
 *    code; fams_strerror() gives its text and fams_last_error() a one-line
 *    detail of the most recent failure on the calling thread.  No C++
 *    exception crosses this boundary.
 *  - Array arguments may be host or device pointers (detected with
 *    cudaPointerGetAttributes).  Input arrays stay owned by the caller and are
 *    copied during the call; output arrays are written during the call.
 *  - Unknown ordering (Eq. 8, block order [m; f]): matrix cells first in
 *    natural order (x fastest, then y, then z), then fracture cells: fractures
 *    in input order, within a fracture along-strike index fastest, then layer.
 *  - A context owns all device memory of its instances (fine system, coarse
 *    grids, P, R, coarse factors, ILU(0) factors, work vectors); it is freed
 *    by fams_destroy().  Memory comes from the device's default memory pool
 *    (stream-ordered allocation); setup raises the pool's release threshold
 *    to half of the device's memory (at least 32 GiB), so freed memory stays
 *    in this process for the next context instead of being unmapped and
 *    mapped again (other allocators of the process see it as in use).  All work is issued on the context's own CUDA stream
 *    and every call returns only after that work has finished.
 *  - A batch context holds several independent instances (a block-diagonal
 *    system): kernels process all instances together and one CTA per instance
 *    runs the sequential parts, so results of an instance do not depend on
 *    what else is in the batch (beyond rounding: the coarse operator is
 *    summed with atomic additions).
 */
#ifndef FAMS_H
#define FAMS_H

#ifdef __cplusplus
extern "C" {
#endif

/* coupling strategy of the basis functions (Sec. 3.1, Eqs. 19-22) */
enum { FAMS_DECOUPLED = 0, FAMS_FRAC = 1, FAMS_ROCK = 2, FAMS_COUPLED = 3 };
/* restriction operator (Sec. 3.2): finite volume (R^FV) or finite element (R^FE = P^T) */
/* restriction (Sec. 3.2): finite volume (primal-block indicators), finite
   element (P^T), or MSMIX: P^T rows for the matrix coarse nodes and
   indicator rows for the fracture coarse nodes */
enum { FAMS_R_FV = 0, FAMS_R_FE = 1, FAMS_R_MIX = 2 };
/* arithmetic of the iteration: FP64 throughout, or mixed: the two-stage
   step's restriction, prolongation and ILU(0) sweeps in FP32 (FP32 copies of
   P, P^T and the factors), with the residuals, r - A dp1, the coarse solve,
   the GMRES basis and the iterate in FP64 (iterative refinement; flexible
   GMRES with FP64 restart vectors) */
enum { FAMS_FP64 = 0, FAMS_MIXED = 1 };
/* outer iteration: the Table 1 loop, or GMRES with the two-stage step as
   right preconditioner (Sec. 4.5, 4.6) */
enum { FAMS_KRYLOV_NONE = 0, FAMS_KRYLOV_GMRES = 1 };
#define FAMS_MAX_RESTART 64

enum {
  FAMS_OK = 0,
  FAMS_EINVAL = -1,      /* bad argument or an input the method cannot handle */
  FAMS_ENOMEM = -2,      /* device allocation failed */
  FAMS_ENOCONV = -3,     /* max_iter reached; x holds the last iterate */
  FAMS_EBREAKDOWN = -4,  /* zero or non-finite pivot in a factorisation */
  FAMS_ETIMEOUT = -5,    /* a bounded device wait gave up */
  FAMS_ECUDA = -6,       /* a CUDA runtime call failed */
  FAMS_ECAPACITY = -7    /* a local problem exceeds a compiled-in size limit */
};

/* Dirichlet face bits; faces not in the mask are no-flow */
enum { FAMS_BC_WEST = 1, FAMS_BC_EAST = 2, FAMS_BC_SOUTH = 4, FAMS_BC_NORTH = 8,
       FAMS_BC_BOTTOM = 16, FAMS_BC_TOP = 32 };

typedef struct fams_ctx fams_ctx;   /* opaque, owned by the library */

/* Structured matrix grid (Sec. 2).  dim = 2 or 3; in 2D nz must be 1 and dz is
   the slab thickness.  bc_value[f] is the pressure on Dirichlet face f
   (order W, E, S, N, B, T).  At least one Dirichlet face is required. */
typedef struct {
  int dim, nx, ny, nz;
  double dx, dy, dz;
  int bc_mask;
  double bc_value[6];
} fams_grid;

/* Fractures (Sec. 2, Eqs. 4-7).  2D: n segments, xy[4i..4i+3] = x0,y0,x1,y1.
   3D: n vertical plates, xy[6i..6i+5] = x0,y0,x1,y1,z0,z1 (layers whose centre
   lies in [z0,z1)).  Coordinates are physical; segments are clipped to the
   domain.  kf[i] is the fracture permeability (mu = 1), aperture the width a_f,
   h_f the target fracture cell length. */
typedef struct {
  int n;
  const double* xy;
  const double* kf;
  double aperture;
  double h_f;
} fams_fracs;

/* Peaceman wells (Sec. 2: q^mw = PI lambda^m (p^w - p^m) per perforated matrix
   cell, volume-integrated; lambda^m = k).  Well w perforates the matrix cells
   perf_cell[perf_ptr[w] .. perf_ptr[w+1]) (natural index, strictly ascending
   within a well) with geometric productivity indices perf_pi (> 0).  A
   FAMS_WELL_RATE well injects value[w] in total (negative: produces); its
   pressure is one more unknown with the equation sum_i PI_i k_i (p^w - p_i) =
   value[w], and it is one coarse node with P^ww = I and its own basis
   function (Sec. 3.1).  A FAMS_WELL_PRESSURE well holds p^w = value[w]: its
   perforations act like Dirichlet half-cells PI_i k_i (p_i - p^w).  All
   arrays host or device memory, copied during setup. */
enum { FAMS_WELL_RATE = 0, FAMS_WELL_PRESSURE = 1 };
typedef struct {
  int n;
  const int* perf_ptr;
  const int* perf_cell;
  const double* perf_pi;
  const int* control;
  const double* value;
} fams_wells;

/* Method options.  coarsen[] = matrix coarsening ratio per axis; frac_dmin =
   d_min of the distance-based fracture coarsening (Table 2; <= 0 means
   infinity, one coarse node per network); frac_cz = vertical coarsening of 3D
   fracture plates; alpha = truncation threshold of P (Sec. 4.3, 0 = none;
   the iteration's P only: the flux reconstruction uses the basis functions
   before truncation);
   max_iter bounds the Table 1 loop (or the GMRES iterations); precision =
   FAMS_FP64 or FAMS_MIXED.  krylov = FAMS_KRYLOV_GMRES runs the two-stage
   step as the right preconditioner of GMRES(restart), the paper's benchmark
   mode (Sec. 4.5, 4.6): every iteration is one preconditioner application,
   and a cycle ends when the least-squares residual estimate reaches tol, after
   `restart` iterations, or at max_iter; the true residual then decides.
   Zero-initialise the struct: fields added later default to 0. */
typedef struct {
  int coarsen[3];
  int frac_dmin;
  int frac_cz;
  int basis;
  int restriction;
  double alpha;
  int max_iter;
  int precision;
  int krylov;    /* FAMS_KRYLOV_NONE: the Table 1 loop; FAMS_KRYLOV_GMRES: GMRES(restart) */
  int restart;   /* GMRES cycle length, 1..FAMS_MAX_RESTART (ignored otherwise) */
  int prepare_flux;  /* 1: the caller will reconstruct fluxes (fams_flux*).  The
                        R^FV coarse system of the reconstruction (Sec. 3.2) is then
                        built on a second stream while the first solve runs,
                        filling the SMs that early-converging instances leave
                        idle; 0: built on the first fams_flux* call.  Results are
                        the same either way. */
  int merge_cap;     /* Coupled-AMS: largest dual block that same-rank links across the
                        media may merge (Sec. 3.1: one can limit the merged blocks);
                        0 = no limit.  The blocks of each medium are merged through the
                        cross-medium links in the order of A's rows and columns, a link
                        joining two blocks only while the merged block stays within the
                        cap; a link left between two blocks is dropped and removed from
                        the diagonal. */
  int grid_solve;    /* the iteration of a single-instance context on every SM of the GPU
                        (one cooperative kernel; GMRES in FP64): 0 = when the instance
                        has at least 2^18 unknowns, 1 = always, -1 = never (one CTA per
                        instance, as for batches).  The same arithmetic either way, up to
                        the order of the sums. */
  int subblock;      /* 1: after the ILU(0) stage, a sub-block smoothing stage (Sec. 3.2:
                        iterations on the sub-block systems of each medium): r2 = r1 -
                        A dp2, dp3 = ILU(0) of A without its cross-medium entries (the
                        blocks A^mm, A^ff and the wells') applied to r2, p += dp3; once
                        per Table 1 sweep or GMRES preconditioner application.  FP64
                        only (FAMS_EINVAL with FAMS_MIXED). */
  int bf16_p;        /* 1 (with FAMS_MIXED only): P and P^T values of the FP32 restriction
                        and prolongation stored in BF16 (8-bit mantissa, FP32 arithmetic);
                        R A P keeps the FP64 P.  A trial of the storage precision: the
                        FP64 residual still decides convergence. */
  int coarse_mode;   /* the whole-GPU iteration's coarse solve: 0 automatic (A_c^-1 while
                        it takes at most 8 GiB, else the band factors), 1 A_c^-1 formed
                        once (a product per iteration on every SM), 2 the band factors
                        solved by one CTA per iteration.  The same solution up to
                        rounding. */
} fams_opts;

/* Per-solve statistics (nullable argument). */
typedef struct {
  int iterations;        /* completed Table 1 sweeps (GMRES: preconditioner applications) */
  double rel_residual;   /* ||q - A x||_2 / ||q||_2 of the returned x */
  int converged;
  double solve_ms;       /* device time of the iteration */
} fams_stats;

/* fams_setup - build one instance: EDFM geometry and fine system (Sec. 2),
   coarse grids (Sec. 3, Table 2), basis functions and P (Sec. 3.1, App. A),
   truncation (Sec. 4.3), R and the coarse factor of R A P (Sec. 3.2), and the
   ILU(0) smoother (Sec. 3.2).
   perm: n_matrix permeabilities, x fastest.  On success *out owns the
   context.  Errors: FAMS_EINVAL (bad sizes, no Dirichlet face, plates of one
   network with different layer ranges), FAMS_ENOMEM, FAMS_EBREAKDOWN,
   FAMS_ECAPACITY, FAMS_ECUDA. */
int fams_setup(const fams_grid* grid, const double* perm, const fams_fracs* fracs,
               const fams_opts* opts, fams_ctx** out);

/* fams_setup_batch - n independent instances in one context (instance i uses
   grids[i], perms[i], fracs[i], opts[i]).  Same errors as fams_setup. */
int fams_setup_batch(int n, const fams_grid* grids, const double* const* perms,
                     const fams_fracs* fracs, const fams_opts* opts, fams_ctx** out);

/* fams_setup_wells / fams_setup_batch_wells - the same with Peaceman wells
   (wells nullable, or wells[i] per instance; fams_wells above).  Unknown
   order [matrix; fractures; rate-controlled wells in input order]: every
   vector of the instance (rhs, x) holds n_matrix + n_frac + n_well values
   (fams_sizes_wells).  Errors as fams_setup; FAMS_EINVAL for a perforation
   outside the matrix, perforations of a well not strictly ascending, a
   non-positive or non-finite PI, an unknown control or a non-finite value. */
int fams_setup_wells(const fams_grid* grid, const double* perm, const fams_fracs* fracs,
                     const fams_wells* wells, const fams_opts* opts, fams_ctx** out);
int fams_setup_batch_wells(int n, const fams_grid* grids, const double* const* perms,
                           const fams_fracs* fracs, const fams_wells* wells,
                           const fams_opts* opts, fams_ctx** out);

/* fams_sizes_wells - rate-controlled wells (unknowns after the fracture
   cells) and perforations of instance `inst`.  The fluxes of fams_flux follow
   the fracture connections with one value per perforation (rate-controlled
   wells first, then pressure-controlled, each in input order; positive from
   the cell into the well), included in n_nnc of fams_sizes.  Null pointers
   are skipped. */
int fams_sizes_wells(const fams_ctx* ctx, int inst, int* n_well, int* n_perf);

/* fams_sizes - counts of instance `inst`: fine unknowns of the matrix and the
   fractures, coarse unknowns, matrix faces (x, y then z faces including the
   boundary faces), and fracture connections (matrix-fracture then
   fracture-fracture, then well perforations).  Null pointers are skipped. */
int fams_sizes(const fams_ctx* ctx, int inst, int* n_matrix, int* n_frac, int* n_coarse,
               int* n_faces, int* n_nnc);

/* fams_solve - Table 1 (steps 3, 5-8) on instance 0 of ctx from the initial
   guess in x until ||q - A x||_2 <= tol ||q||_2, q = rhs + Dirichlet terms.
   rhs: n_matrix + n_frac sources (+ n_well values added to the rate wells'
   rates; nullable = 0); x: in initial guess, out pressure (n_matrix + n_frac
   + n_well values: the rate wells' pressures last).  FAMS_ENOCONV leaves the last iterate in x; FAMS_EBREAKDOWN
   reports a numerically singular coarse system (the test of fams_flux_batch). */
int fams_solve(fams_ctx* ctx, const double* rhs, double* x, double tol, fams_stats* st);

/* fams_solve_batch - the same for every instance of a batch context; rhs[i]
   (nullable) and x[i] per instance, st nullable or an array of n_instances.
   Returns FAMS_ENOCONV if any instance did not converge. */
int fams_solve_batch(fams_ctx* ctx, const double* const* rhs, double* const* x, double tol,
                     fams_stats* st);
/* fams_solve_subset - fams_solve_batch on the n_list distinct instances in
   list only (the others keep their state and launch nothing); rhs, x and st
   are indexed like list.  A whole-GPU context (one instance) takes list {0}.
   FAMS_EINVAL for an index out of range or repeated. */
int fams_solve_subset(fams_ctx* ctx, int n_list, const int* list, const double* const* rhs,
                      double* const* x, double tol, fams_stats* st);

/* fams_update - time-step update of instance 0: every connection's
   transmissibility (matrix faces, matrix-fracture and fracture-fracture) is
   the setup-time value times the harmonic mean 2 s_i s_j / (s_i + s_j) of its
   two cells' mobility scales, a Dirichlet half-cell's the setup-time value
   times its cell's scale.  The coarse grids and P (Sec. 3.1) are kept; R A P
   and its factors, the ILU(0) smoother and the fluxes' transmissibilities
   follow.  mobility_scale: n_matrix + n_frac positive finite values (not
   checked), relative to the setup (nullable: all 1, i.e. back to the setup
   values); host or device.  A perforation scales like a connection whose
   well side keeps scale 1 (rate well) or like a Dirichlet half-cell
   (pressure well). */
int fams_update(fams_ctx* ctx, const double* mobility_scale);
/* the same for every instance of a batch context (scale[i] nullable) */
int fams_update_batch(fams_ctx* ctx, const double* const* mobility_scale);

/* fams_update_basis - fams_update_batch, then the adaptive basis update of
   Sec. 3.1 (basis functions recomputed only where the fine-scale properties
   change beyond a threshold), per dual block: a cell is marked when its
   mobility scale differs from the scale its basis row was last computed with
   (the setup's, 1, until then) by more than a factor 1 + eps (eps < 0 marks
   every cell, +infinity none); the dual blocks holding a marked cell, and,
   stage by stage, the blocks that read a row solved again in an earlier
   stage, are solved again from the updated operator on the same coarse
   grids, the others keep their rows; truncation, P^T, R A P and its factors
   follow (ILU(0) as after the update).  *rebuilt (nullable) receives the
   number of dual blocks solved (0: P unchanged).  Errors as fams_update;
   FAMS_EINVAL for a NaN eps. */
int fams_update_basis(fams_ctx* ctx, const double* const* mobility_scale, double eps,
                      int* rebuilt);

/* Limits of fams_solve_static (its fixed work array, about 15 MB per GPU). */
#define FAMS_STATIC_MAX_ROWS 262144   /* n_matrix + n_frac of the instance */
#define FAMS_STATIC_MAX_COARSE 16384  /* n_coarse of the instance */
#define FAMS_STATIC_MAX_ITER 16383    /* the instance's max_iter */

/* fams_solve_static - the solve of fams_solve (same arguments, same result)
   for callers that cannot allocate device memory when they solve: a code
   that hands the free device memory to its own pool allocator and leaves
   none to libraries, or a time-step loop that must not enter cudaMalloc or
   cudaFree (both can synchronise the device, and can fail under memory
   pressure mid-run).  The paper has no counterpart; it is a deployment
   variant of the same iteration.
   It allocates nothing, on any call: the iteration's work vectors (the
   right-hand side with its Dirichlet terms, iterate, residual, multiscale
   and ILU corrections, the coarse vectors, status words and residual
   history) live in one device array compiled into the library, of fixed size
   (the FAMS_STATIC_MAX_* limits; every GPU that loads the library holds it
   until the process exits).  Every call looks up that array's address on the
   context's device (cudaGetSymbolAddress, a host query), so the address
   stays right if the device's context is recreated; the first call on a
   device also loads the library's kernels there: make the first call on each
   device before any stream capture starts.
   ctx must be a single-instance context; x (in initial guess, out pressure)
   and rhs (nullable) may be host or device memory.  Instances above a limit
   are rejected with FAMS_ECAPACITY before anything runs.  Every call, from any
   context, shares the one array per device and it keeps the last call's
   contents; each call clears the status words and writes every other value
   it reads.  Calls that overlap on the GPU (other threads, other streams)
   race on the array: serialise them.  stats.solve_ms is host wall time of the
   launch and its completion. */
int fams_solve_static(fams_ctx* ctx, const double* rhs, double* x, double tol, fams_stats* st);

/* fams_flux - conservative fine-scale flux field from an iterate x of
   instance `inst`: one finite-volume multiscale stage, then a local TPFA
   problem per primal block with the block-boundary fluxes as Neumann data
   (Sec. 3.2; after any iteration, Sec. 1); the finite-volume stage uses the
   basis functions before truncation.  face_flux: n_faces values, x faces
   ((nx+1) ny nz, x fastest), then y faces, then z faces, positive along +axis
   (no-flow boundary faces are 0).  nnc_flux: n_nnc values, matrix-fracture
   connections (positive matrix -> fracture) in fams_query(FAMS_Q_NNC_*) order,
   then fracture-fracture connections (positive from the lower to the higher
   fracture cell index). */
int fams_flux(fams_ctx* ctx, int inst, const double* x, double* face_flux, double* nnc_flux);

/* fams_flux_batch - the same reconstruction for every instance of a batch
   context in one pass (x[i], face_flux[i], nnc_flux[i] per instance, host or
   device).  status (nullable, n_instances entries) receives each instance's
   result; an instance whose finite-volume coarse system R^FV A P is
   numerically singular gets FAMS_EBREAKDOWN and its buffers are left
   untouched while the others are reconstructed.  Numerically singular: a
   pivot of its band LU is at most 1e-13 times the largest entry of its row as
   assembled (e.g. a node cell 1e-300 times as permeable as its neighbours:
   its basis function is 1e-300 outside the node cell, and its R^FV column is
   that small).  The reconstruction's R^FV A P is built with the basis
   functions before truncation (a truncated basis function can lie inside
   its own primal block, which makes its column of R^FV A P zero).  Returns
   FAMS_EBREAKDOWN if any instance failed that way. */
int fams_flux_batch(fams_ctx* ctx, const double* const* x, double* const* face_flux,
                    double* const* nnc_flux, int* status);

/* fams_query - copy an internal array of instance `inst` into out (host or
   device, capacity `cap` elements of the stated type).  Returns the element
   count (>= 0) or a negative error; with out == NULL only the count.  For the
   parity tests and for diagnostics. */
enum {
  FAMS_Q_NNC_FRAC = 1,     /* int32  matrix-fracture connections: fracture cell (local) */
  FAMS_Q_NNC_MATRIX = 2,   /* int32  ... matrix cell */
  FAMS_Q_NNC_AREA = 3,     /* double ... A_ij */
  FAMS_Q_NNC_DIST = 4,     /* double ... <d>_ij */
  FAMS_Q_FF_A = 5,         /* int32  fracture-fracture connections: lower cell */
  FAMS_Q_FF_B = 6,         /* int32  ... higher cell */
  FAMS_Q_FF_T = 7,         /* double ... transmissibility */
  FAMS_Q_A_ROWPTR = 8,     /* int32  CSR of A (n+1) */
  FAMS_Q_A_COL = 9,        /* int32 */
  FAMS_Q_A_VAL = 10,       /* double */
  FAMS_Q_Q = 11,           /* double total rhs q (sources + Dirichlet terms) */
  FAMS_Q_RANK = 12,        /* int32  wirebasket rank per cell (V=3,E=2,F=1,I=0) */
  FAMS_Q_PRIMAL = 13,      /* int32  primal block = coarse index per cell */
  FAMS_Q_NODE_CELL = 14,   /* int32  node cell of each coarse unknown */
  FAMS_Q_P_ROWPTR = 15,    /* int32  CSR of P (after truncation) */
  FAMS_Q_P_COL = 16,       /* int32 */
  FAMS_Q_P_VAL = 17,       /* double */
  FAMS_Q_AC = 18,          /* double dense coarse operator R A P, row-major */
  FAMS_Q_ILU_VAL = 19,     /* double ILU(0) factors in the pattern of A */
  FAMS_Q_LEVELS = 20,      /* int32  number of ILU(0) levels (1 value) */
  FAMS_Q_COARSE_PERM = 21, /* int32  band position -> coarse unknown (reverse Cuthill-McKee) */
  FAMS_Q_COARSE_IPIV = 22, /* int32  pivot row (band position) of each LU step */
  FAMS_Q_BAND_KLKU = 23,   /* int32  lower and upper bandwidth (2 values) */
  FAMS_Q_BAND = 24,        /* double band LU factors, column-major, 2kl+ku+1 rows */
  FAMS_Q_HISTORY = 25,     /* double relative residual after each sweep of the last solve */
  FAMS_Q_LAST_DP1 = 26,    /* double multiscale correction of the last sweep (Table 1 step 5) */
  FAMS_Q_LAST_DP2 = 27,    /* double smoother correction of the last sweep (Table 1 step 7) */
  FAMS_Q_LAST_RC = 28,     /* double coarse right-hand side R r of the last sweep */
  FAMS_Q_LAST_EC = 29,     /* double coarse solution (R A P)^-1 R r of the last sweep */
  FAMS_Q_STAGE_CYCLES = 30, /* double SM cycles of the last solve per phase: residual,
                               restriction, band solve, prolongation + r1, L sweep, U sweep */
  FAMS_Q_SETUP_MS = 31,    /* double wall ms of the setup phases of the whole context:
                              geometry, fine system, coarse grids, basis, coarse operator,
                              ILU(0) */
  FAMS_Q_CLASS_COUNTS = 32 /* int32  local problems of the whole context solved per size
                              class (one warp; a 128-thread CTA; a 256-thread CTA in shared
                              memory; a 512-thread CTA on a global-memory workspace): the
                              basis functions' dual blocks (4 values, all setups and
                              rebuilds), then the flux reconstruction's primal blocks (4
                              values, all calls) */
};
int fams_query(const fams_ctx* ctx, int inst, int what, void* out, long long cap);

int fams_num_instances(const fams_ctx* ctx);
void fams_destroy(fams_ctx* ctx);
const char* fams_strerror(int status);
const char* fams_last_error(void);

/* Request server: continuous batching of independent solves (setup, solve
   to tol and, optionally, the flux reconstruction).  The paper has no
   counterpart; it is the deployment layer around the solver.  Problems are
   copied at submission.  `pipelines` worker threads, each with its own
   context and CUDA stream, repeatedly take up to `max_batch` waiting
   requests in arrival order -- of the oldest one's kind (whether its coarse
   band factorisation is estimated to be large), as many as fit in
   `hbm_budget` bytes of
   device memory (an estimate from the problem sizes) next to the
   micro-batches already in flight, and always at least one on an idle
   device -- and process them as one batch; requests that arrive meanwhile
   go to the next free worker.  A result does not depend on what the request
   was batched with (up to the rounding of the coarse operator's atomic
   sums).  rhs, if given, holds n_matrix matrix-cell sources (fracture sources
   are zero).  Finished micro-batches stay resident for time-step updates
   (fams_server_submit_update) and count against hbm_budget until all their
   requests are released or the memory is needed.  Calls are thread-safe. */
typedef struct fams_server fams_server;
typedef struct {
  int max_batch;         /* instances per micro-batch, >= 1 */
  int pipelines;         /* micro-batches in flight, 1..16 */
  long long hbm_budget;  /* bytes the in-flight micro-batches and resident setups may use */
  double tol;            /* relative residual of every solve */
  int with_flux;         /* also reconstruct the conservative fluxes */
} fams_server_opts;

int fams_server_create(const fams_server_opts* opts, fams_server** out);
/* ticket: identifies the request in the calls below */
int fams_server_submit(fams_server* s, const fams_grid* grid, const double* perm,
                       const fams_fracs* fracs, const fams_opts* opts, const double* rhs,
                       long long* ticket);
/* fams_server_submit_update - a time-step update of the earlier new
   realisation `base` (finished or not): its problem with every cell's
   mobility scaled by mobility_scale (n_scale = n_matrix + n_frac values,
   relative to the base's setup as in fams_update; copied), solved with the
   basis functions of the base's setup (Sec. 3.1 end; the server keeps each
   finished micro-batch's context resident for this) from the base's
   pressure as initial guess.  rhs (n_rhs matrix-cell sources; nullable: the
   base's).  Updates of one resident context are batched; an update of a
   setup evicted for memory sets the base problem up again first.  The
   result is collected like any request's; its status is FAMS_EINVAL when
   the base failed, was released before the update ran, or n_scale does not
   match its unknowns. */
int fams_server_submit_update(fams_server* s, long long base, const double* mobility_scale,
                              long long n_scale, const double* rhs, long long n_rhs,
                              long long* ticket);
/* waits up to timeout_ms (<= 0: no wait); *done = 1 once the result is ready */
int fams_server_wait(fams_server* s, long long ticket, double timeout_ms, int* done);
/* copies a finished request's pressure (n_matrix + n_frac values), fluxes (as
   fams_flux; with_flux only; host or device memory) and statistics (st->solve_ms: from the start of
   the request's micro-batch to its completion); latency_ms = completion minus
   submission time.  Returns the request's status.  Null outputs are skipped;
   a capacity below the result's size is FAMS_EINVAL. */
int fams_server_result(fams_server* s, long long ticket, double* x, long long x_cap,
                       double* face_flux, long long face_cap, double* nnc_flux, long long nnc_cap,
                       fams_stats* st, double* latency_ms);
/* sizes of a finished request's results: unknowns, face fluxes, NNC fluxes
   (0 without fluxes; one placeholder value when the instance has no NNC) */
int fams_server_sizes(fams_server* s, long long ticket, long long* n, long long* n_faces,
                      long long* n_nnc);
/* frees a finished request */
int fams_server_release(fams_server* s, long long ticket);
/* finishes every submitted request, then stops the workers and frees all */
void fams_server_destroy(fams_server* s);

/* Number of CUDA kernels the library has launched since it was loaded (all
   contexts, all threads); the difference across a call counts its launches. */
long long fams_launch_count(void);

/* Number of device allocations the library has made since it was loaded (all
   contexts, all threads); the difference across a call counts its
   allocations (0 across fams_solve_static). */
long long fams_alloc_count(void);

#ifdef __cplusplus
}
#endif
#endif /* FAMS_H */
