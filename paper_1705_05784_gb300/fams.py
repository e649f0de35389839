"""Thin ctypes binding of libfams (include/fams.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  Importing this
module loads the in-tree libfams.so and raises if it is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libfams.so")

DECOUPLED, FRAC, ROCK, COUPLED = 0, 1, 2, 3
R_FV, R_FE, R_MIX = 0, 1, 2
FP64, MIXED = 0, 1
KRYLOV_NONE, KRYLOV_GMRES = 0, 1
OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, ETIMEOUT, ECUDA, ECAPACITY = 0, -1, -2, -3, -4, -5, -6, -7

Q = dict(NNC_FRAC=1, NNC_MATRIX=2, NNC_AREA=3, NNC_DIST=4, FF_A=5, FF_B=6, FF_T=7,
         A_ROWPTR=8, A_COL=9, A_VAL=10, Q=11, RANK=12, PRIMAL=13, NODE_CELL=14,
         P_ROWPTR=15, P_COL=16, P_VAL=17, AC=18, ILU_VAL=19, LEVELS=20,
         COARSE_PERM=21, COARSE_IPIV=22, BAND_KLKU=23, BAND=24, HISTORY=25,
         LAST_DP1=26, LAST_DP2=27, LAST_RC=28, LAST_EC=29, STAGE_CYCLES=30, SETUP_MS=31,
         CLASS_COUNTS=32)
_INT_QUERIES = {1, 2, 5, 6, 8, 9, 12, 13, 14, 15, 16, 20, 21, 22, 23, 32}


class fams_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("bc_mask", C.c_int), ("bc_value", C.c_double * 6)]


class fams_fracs(C.Structure):
    _fields_ = [("n", C.c_int), ("xy", C.POINTER(C.c_double)), ("kf", C.POINTER(C.c_double)),
                ("aperture", C.c_double), ("h_f", C.c_double)]


class fams_opts(C.Structure):
    _fields_ = [("coarsen", C.c_int * 3), ("frac_dmin", C.c_int), ("frac_cz", C.c_int),
                ("basis", C.c_int), ("restriction", C.c_int), ("alpha", C.c_double),
                ("max_iter", C.c_int), ("precision", C.c_int), ("krylov", C.c_int),
                ("restart", C.c_int),
                ("prepare_flux", C.c_int), ("merge_cap", C.c_int),
                ("grid_solve", C.c_int), ("subblock", C.c_int), ("bf16_p", C.c_int),
                ("coarse_mode", C.c_int)]


class fams_wells(C.Structure):
    _fields_ = [("n", C.c_int), ("perf_ptr", C.POINTER(C.c_int)),
                ("perf_cell", C.POINTER(C.c_int)), ("perf_pi", C.POINTER(C.c_double)),
                ("control", C.POINTER(C.c_int)), ("value", C.POINTER(C.c_double))]


class fams_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("converged", C.c_int),
                ("solve_ms", C.c_double)]


class fams_server_opts(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("pipelines", C.c_int), ("hbm_budget", C.c_longlong),
                ("tol", C.c_double), ("with_flux", C.c_int)]


class FamsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libfams status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; build it with "
                          "paper_1705_05784_gb300.build.build() (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    lib.fams_setup_batch.argtypes = [C.c_int, P(fams_grid), P(P(C.c_double)), P(fams_fracs),
                                     P(fams_opts), P(C.c_void_p)]
    lib.fams_setup.argtypes = [P(fams_grid), P(C.c_double), P(fams_fracs), P(fams_opts),
                               P(C.c_void_p)]
    lib.fams_setup_batch_wells.argtypes = [C.c_int, P(fams_grid), P(P(C.c_double)), P(fams_fracs),
                                           P(fams_wells), P(fams_opts), P(C.c_void_p)]
    lib.fams_sizes_wells.argtypes = [C.c_void_p, C.c_int, P(C.c_int), P(C.c_int)]
    lib.fams_sizes.argtypes = [C.c_void_p, C.c_int] + [P(C.c_int)] * 5
    lib.fams_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, P(fams_stats)]
    lib.fams_solve_batch.argtypes = [C.c_void_p, P(C.c_void_p), P(C.c_void_p), C.c_double,
                                     P(fams_stats)]
    lib.fams_solve_subset.argtypes = [C.c_void_p, C.c_int, P(C.c_int), P(C.c_void_p),
                                      P(C.c_void_p), C.c_double, P(fams_stats)]
    lib.fams_solve_static.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                      P(fams_stats)]
    lib.fams_flux.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.fams_update.argtypes = [C.c_void_p, C.c_void_p]
    lib.fams_update_batch.argtypes = [C.c_void_p, P(C.c_void_p)]
    lib.fams_update_basis.argtypes = [C.c_void_p, P(C.c_void_p), C.c_double, P(C.c_int)]
    lib.fams_flux_batch.argtypes = [C.c_void_p, P(C.c_void_p), P(C.c_void_p), P(C.c_void_p),
                                    P(C.c_int)]
    lib.fams_query.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_longlong]
    lib.fams_num_instances.argtypes = [C.c_void_p]
    lib.fams_destroy.argtypes = [C.c_void_p]
    lib.fams_destroy.restype = None
    lib.fams_strerror.argtypes = [C.c_int]
    lib.fams_strerror.restype = C.c_char_p
    lib.fams_last_error.argtypes = []
    lib.fams_last_error.restype = C.c_char_p
    lib.fams_launch_count.argtypes = []
    lib.fams_launch_count.restype = C.c_longlong
    lib.fams_alloc_count.argtypes = []
    lib.fams_alloc_count.restype = C.c_longlong
    lib.fams_server_create.argtypes = [P(fams_server_opts), P(C.c_void_p)]
    lib.fams_server_submit.argtypes = [C.c_void_p, P(fams_grid), P(C.c_double), P(fams_fracs),
                                       P(fams_opts), P(C.c_double), P(C.c_longlong)]
    lib.fams_server_submit_update.argtypes = [C.c_void_p, C.c_longlong, P(C.c_double),
                                              C.c_longlong, P(C.c_double), C.c_longlong,
                                              P(C.c_longlong)]
    lib.fams_server_wait.argtypes = [C.c_void_p, C.c_longlong, C.c_double, P(C.c_int)]
    lib.fams_server_result.argtypes = [C.c_void_p, C.c_longlong, P(C.c_double), C.c_longlong,
                                       P(C.c_double), C.c_longlong, P(C.c_double), C.c_longlong,
                                       P(fams_stats), P(C.c_double)]
    lib.fams_server_release.argtypes = [C.c_void_p, C.c_longlong]
    lib.fams_server_sizes.argtypes = [C.c_void_p, C.c_longlong] + [P(C.c_longlong)] * 3
    lib.fams_server_destroy.argtypes = [C.c_void_p]
    lib.fams_server_destroy.restype = None
    return lib


lib = _load()


def _check(status, allow=()):
    if status < 0 and status not in allow:
        raise FamsError(status, (lib.fams_strerror(status).decode() + ": "
                                 + lib.fams_last_error().decode()))
    return status


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _args(prob):
    """ctypes structs (and the arrays they point into) for one inputs.Problem."""
    g = fams_grid(prob.dim, prob.nx, prob.ny, prob.nz if prob.dim == 3 else 1,
                  prob.dx, prob.dy, prob.dz, prob.bc_mask, (C.c_double * 6)(*prob.bc_value))
    perm = np.ascontiguousarray(prob.perm, dtype=np.float64)
    fr = np.zeros((0, 6 if prob.dim == 3 else 4)) if prob.fracs is None else prob.fracs
    xy = np.ascontiguousarray(fr, dtype=np.float64).ravel()
    kf = np.ascontiguousarray(np.zeros(0) if prob.kf is None else prob.kf, dtype=np.float64)
    f = fams_fracs(len(fr), _dptr(xy) if len(fr) else None, _dptr(kf) if len(fr) else None,
                   prob.aperture, prob.h_f)
    cz = prob.coarsen[2] if prob.dim == 3 else 1
    o = fams_opts((C.c_int * 3)(prob.coarsen[0], prob.coarsen[1], cz), prob.frac_dmin,
                  max(1, prob.frac_cz), prob.basis, prob.restriction, prob.alpha,
                  prob.max_iter, getattr(prob, "precision", FP64), getattr(prob, "krylov", 0),
                  getattr(prob, "restart", 30), getattr(prob, "prepare_flux", 0),
                  getattr(prob, "merge_cap", 0), getattr(prob, "grid_solve", 0),
                  getattr(prob, "subblock", 0), getattr(prob, "bf16_p", 0),
                  getattr(prob, "coarse_mode", 0))
    return g, perm, f, o, (xy, kf)


def _wells(prob):
    """fams_wells (and the arrays it points into) for the wells of a problem."""
    ws = getattr(prob, "wells", None) or []
    if not ws:
        return fams_wells(0, None, None, None, None, None), ()
    ptr = np.zeros(len(ws) + 1, np.int32)
    for i, w in enumerate(ws):
        ptr[i + 1] = ptr[i] + len(w.cells)
    cells = np.ascontiguousarray(np.concatenate([np.asarray(w.cells) for w in ws]), np.int32)
    pis = np.ascontiguousarray(np.concatenate([np.asarray(w.pi, np.float64) for w in ws]))
    ctl = np.array([int(w.control) for w in ws], np.int32)
    val = np.array([float(w.value) for w in ws], np.float64)
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    out = fams_wells(len(ws), ip(ptr), ip(cells), _dptr(pis), ip(ctl), _dptr(val))
    return out, (ptr, cells, pis, ctl, val)


def launch_count():
    """Kernels launched by the library since it was loaded."""
    return int(lib.fams_launch_count())


def alloc_count():
    """Device allocations made by the library since it was loaded."""
    return int(lib.fams_alloc_count())


class Context:
    """One libfams context (a batch of one or more instances).

    device_perm: optional list of device pointers (one per instance) holding
    the permeability arrays already resident in GPU memory; the library then
    copies device to device."""

    def __init__(self, problems, device_perm=None):
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        n = len(problems)
        parts = [_args(p) for p in problems]
        grids = (fams_grid * n)(*[p[0] for p in parts])
        if device_perm is not None:
            perms = (C.POINTER(C.c_double) * n)(
                *[C.cast(C.c_void_p(int(d)), C.POINTER(C.c_double)) for d in device_perm])
        else:
            perms = (C.POINTER(C.c_double) * n)(*[_dptr(p[1]) for p in parts])
        fracs = (fams_fracs * n)(*[p[2] for p in parts])
        opts = (fams_opts * n)(*[p[3] for p in parts])
        wl = [_wells(p) for p in problems]
        self._keep = (parts, wl)
        self.h = C.c_void_p()
        if any(w[0].n for w in wl):
            wells = (fams_wells * n)(*[w[0] for w in wl])
            _check(lib.fams_setup_batch_wells(n, grids, perms, fracs, wells, opts, C.byref(self.h)))
        else:
            _check(lib.fams_setup_batch(n, grids, perms, fracs, opts, C.byref(self.h)))
        self.n = n
        self.problems = problems

    def close(self):
        if self.h:
            lib.fams_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sizes(self, inst=0):
        """Counts of an instance; "n" = every unknown (matrix, fracture and
        rate-well pressures), the length of its rhs and x."""
        v = [C.c_int() for _ in range(7)]
        _check(lib.fams_sizes(self.h, inst, *[C.byref(x) for x in v[:5]]))
        _check(lib.fams_sizes_wells(self.h, inst, C.byref(v[5]), C.byref(v[6])))
        d = dict(zip(("n_matrix", "n_frac", "n_coarse", "n_faces", "n_nnc", "n_well", "n_perf"),
                     [x.value for x in v]))
        d["n"] = d["n_matrix"] + d["n_frac"] + d["n_well"]
        return d

    def query(self, what, inst=0):
        code = Q[what] if isinstance(what, str) else what
        n = _check(lib.fams_query(self.h, inst, code, None, 0))
        dt = np.int32 if code in _INT_QUERIES else np.float64
        out = np.zeros(n, dt)
        _check(lib.fams_query(self.h, inst, code, out.ctypes.data_as(C.c_void_p), n))
        return out

    def solve(self, rhs=None, x0=None, tol=1e-8, allow_noconv=True):
        """Solve every instance; rhs/x0: list per instance (or one array for a
        single instance).  Returns (list of pressures, list of stats dicts)."""
        n = self.n
        sz = [self.sizes(i) for i in range(n)]
        N = [s["n"] for s in sz]
        if rhs is not None and not isinstance(rhs, (list, tuple)):
            rhs = [rhs]
        if x0 is not None and not isinstance(x0, (list, tuple)):
            x0 = [x0]
        xs = [np.ascontiguousarray(x0[i] if x0 is not None else np.zeros(N[i]), np.float64).copy()
              for i in range(n)]
        rs = [None if rhs is None or rhs[i] is None else np.ascontiguousarray(rhs[i], np.float64)
              for i in range(n)]
        xp = (C.c_void_p * n)(*[x.ctypes.data for x in xs])
        rp = (C.c_void_p * n)(*[0 if r is None else r.ctypes.data for r in rs])
        st = (fams_stats * n)()
        s = lib.fams_solve_batch(self.h, rp, xp, tol, st)
        _check(s, allow=(ENOCONV,) if allow_noconv else ())
        stats = [dict(iterations=st[i].iterations, rel_residual=st[i].rel_residual,
                      converged=bool(st[i].converged), solve_ms=st[i].solve_ms, status=s)
                 for i in range(n)]
        return xs, stats

    def solve_subset(self, insts, rhs=None, x0=None, tol=1e-8):
        """fams_solve_subset: solve only the listed instances (the others keep
        their state).  rhs/x0: lists indexed like insts.  Returns (pressures,
        stats dicts) indexed like insts."""
        m = len(insts)
        N = [self.sizes(i)["n"] for i in insts]
        xs = [np.ascontiguousarray(x0[k] if x0 is not None else np.zeros(N[k]), np.float64).copy()
              for k in range(m)]
        rs = [None if rhs is None or rhs[k] is None else np.ascontiguousarray(rhs[k], np.float64)
              for k in range(m)]
        li = (C.c_int * max(m, 1))(*insts)
        xp = (C.c_void_p * max(m, 1))(*[x.ctypes.data for x in xs])
        rp = (C.c_void_p * max(m, 1))(*[0 if r is None else r.ctypes.data for r in rs])
        st = (fams_stats * max(m, 1))()
        s = lib.fams_solve_subset(self.h, m, li, rp, xp, tol, st)
        _check(s, allow=(ENOCONV,))
        return xs, [dict(iterations=st[k].iterations, rel_residual=st[k].rel_residual,
                         converged=bool(st[k].converged), solve_ms=st[k].solve_ms, status=s)
                    for k in range(m)]

    def update(self, scales):
        """fams_update_batch: scales is a list per instance (None: all 1) or
        one array for a single instance."""
        if not isinstance(scales, (list, tuple)):
            scales = [scales]
        arrs = [None if sc is None else np.ascontiguousarray(sc, np.float64) for sc in scales]
        ptrs = (C.c_void_p * self.n)(*[0 if a is None else a.ctypes.data for a in arrs])
        _check(lib.fams_update_batch(self.h, ptrs))

    def update_basis(self, scales, eps):
        """fams_update_basis: the update of `update`, then the adaptive basis
        update: dual blocks holding a cell whose scale moved by more than a
        factor 1 + eps since its basis row was computed (eps < 0: every
        block), and their downstream blocks, solved again.  Returns the number
        of dual blocks solved (0: P unchanged)."""
        if not isinstance(scales, (list, tuple)):
            scales = [scales]
        arrs = [None if sc is None else np.ascontiguousarray(sc, np.float64) for sc in scales]
        ptrs = (C.c_void_p * self.n)(*[0 if a is None else a.ctypes.data for a in arrs])
        r = C.c_int(0)
        _check(lib.fams_update_basis(self.h, ptrs, float(eps), C.byref(r)))
        return int(r.value)

    def solve_device(self, rhs_ptrs, x_ptrs, tol):
        """The same call with caller-owned buffers given as raw pointers (host
        or device), for timing the C-ABI path without copies in Python."""
        n = self.n
        xp = (C.c_void_p * n)(*x_ptrs)
        rp = (C.c_void_p * n)(*[p or 0 for p in rhs_ptrs])
        st = (fams_stats * n)()
        s = lib.fams_solve_batch(self.h, rp, xp, tol, st)
        _check(s, allow=(ENOCONV, EBREAKDOWN))
        return [dict(iterations=st[i].iterations, rel_residual=st[i].rel_residual,
                     converged=bool(st[i].converged), solve_ms=st[i].solve_ms)
                for i in range(n)]

    def solve_static(self, rhs=None, x0=None, tol=1e-8):
        """fams_solve_static on this single-instance context: the solve of
        fams_solve with the library's fixed work array instead of any
        allocation.  Returns (pressure, stats dict)."""
        N = self.sizes(0)["n"]
        x = np.ascontiguousarray(x0 if x0 is not None else np.zeros(N), np.float64).copy()
        r = None if rhs is None else np.ascontiguousarray(rhs, np.float64)
        st = fams_stats()
        s = lib.fams_solve_static(self.h, None if r is None else r.ctypes.data_as(C.c_void_p),
                                  x.ctypes.data_as(C.c_void_p), tol, C.byref(st))
        _check(s, allow=(ENOCONV, EBREAKDOWN))
        return x, dict(iterations=st.iterations, rel_residual=st.rel_residual,
                       converged=bool(st.converged), solve_ms=st.solve_ms, status=s)

    def flux_batch_ptr(self, x_ptrs, face_ptrs, nnc_ptrs):
        """fams_flux_batch on caller-owned buffers (raw pointers, host or
        device); returns the per-instance status list."""
        n = self.n
        st = (C.c_int * n)()
        xp = (C.c_void_p * n)(*[int(p) for p in x_ptrs])
        fp = (C.c_void_p * n)(*[int(p) for p in face_ptrs])
        npp = (C.c_void_p * n)(*[int(p) for p in nnc_ptrs])
        _check(lib.fams_flux_batch(self.h, xp, fp, npp, st), allow=(EBREAKDOWN,))
        return list(st)

    def flux_ptr(self, inst, x_ptr, face_ptr, nnc_ptr):
        """fams_flux on caller-owned buffers given as raw pointers (host or device)."""
        _check(lib.fams_flux(self.h, inst, C.c_void_p(int(x_ptr)), C.c_void_p(int(face_ptr)),
                             C.c_void_p(int(nnc_ptr))))

    def flux(self, x, inst=0):
        s = self.sizes(inst)
        face = np.zeros(s["n_faces"])
        nnc = np.zeros(max(s["n_nnc"], 1))
        x = np.ascontiguousarray(x, np.float64)
        _check(lib.fams_flux(self.h, inst, x.ctypes.data_as(C.c_void_p),
                             face.ctypes.data_as(C.c_void_p), nnc.ctypes.data_as(C.c_void_p)))
        return face, nnc[: s["n_nnc"]]


class Server:
    """fams_server_*: continuous batching of independent solves."""

    def __init__(self, max_batch=64, pipelines=2, hbm_budget=64 << 30, tol=1e-8, with_flux=True):
        o = fams_server_opts(max_batch, pipelines, hbm_budget, tol, 1 if with_flux else 0)
        self.h = C.c_void_p()
        _check(lib.fams_server_create(C.byref(o), C.byref(self.h)))
        self.with_flux = with_flux
        self._sizes = {}

    def submit(self, prob, rhs=None):
        g, perm, f, o, keep = _args(prob)
        t = C.c_longlong()
        r = None if rhs is None else np.ascontiguousarray(rhs, np.float64)
        _check(lib.fams_server_submit(self.h, C.byref(g), _dptr(perm), C.byref(f), C.byref(o),
                                      None if r is None else _dptr(r), C.byref(t)))
        return t.value

    def submit_update(self, base, scale, rhs=None):
        """Time-step update of the new realisation `base`: mobility scale per
        cell (n_matrix + n_frac values), basis functions of the base's setup."""
        sc = np.ascontiguousarray(scale, np.float64)
        r = None if rhs is None else np.ascontiguousarray(rhs, np.float64)
        t = C.c_longlong()
        _check(lib.fams_server_submit_update(self.h, base, _dptr(sc), len(sc),
                                             None if r is None else _dptr(r),
                                             0 if r is None else len(r), C.byref(t)))
        return t.value

    def wait(self, ticket, timeout_ms=60000.0):
        d = C.c_int()
        _check(lib.fams_server_wait(self.h, ticket, timeout_ms, C.byref(d)))
        return bool(d.value)

    def result(self, ticket, n, n_faces=0, n_nnc=0):
        """Pressure (n values), face and NNC fluxes (if the server makes them),
        stats dict with latency_ms, and the request's status."""
        x = np.zeros(n)
        face = np.zeros(max(n_faces, 1))
        nnc = np.zeros(max(n_nnc, 1))
        st = fams_stats()
        lat = C.c_double()
        s = lib.fams_server_result(self.h, ticket, _dptr(x), n, _dptr(face), len(face), _dptr(nnc),
                                   len(nnc), C.byref(st), C.byref(lat))
        # a failed request reports its status (and fams_last_error its reason)
        return x, face[:n_faces], nnc[:n_nnc], dict(iterations=st.iterations,
                                                    rel_residual=st.rel_residual,
                                                    converged=bool(st.converged),
                                                    latency_ms=lat.value, status=s,
                                                    service_ms=st.solve_ms,
                                                    error=lib.fams_last_error().decode()
                                                    if s != OK else "")

    def sizes(self, ticket):
        v = [C.c_longlong() for _ in range(3)]
        _check(lib.fams_server_sizes(self.h, ticket, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def fetch(self, ticket):
        """result() with buffers sized by the finished request itself."""
        n, nf, nn = self.sizes(ticket)
        return self.result(ticket, n, nf, nn)

    def status(self, ticket):
        return lib.fams_server_result(self.h, ticket, None, 0, None, 0, None, 0, None, None)

    def release(self, ticket):
        _check(lib.fams_server_release(self.h, ticket))

    def close(self):
        if self.h:
            lib.fams_server_destroy(self.h)
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
