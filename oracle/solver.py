"""Oracle: restriction, coarse system, ILU(0) smoother and the two-stage
iteration (Sec. 3.2, Table 1), and conservative flux reconstruction.

TEST INFRASTRUCTURE ONLY (see oracle/geometry.py).

* R^FV: R[I, i] = 1 when fine cell i lies in primal block I (Sec. 3.2);
  R^FE = P^T (MSFE); MSMIX: P^T rows for matrix coarse nodes, R^FV rows for
  fracture coarse nodes (the paper's example of the hybrid, Sec. 3.2).
* coarse operator A_c = R A P, solved by LU with partial pivoting (the paper
  uses a direct LU solver, Sec. 4).
* ILU(0) of the complete fine A in natural order (matrix cells then fracture
  cells), no pivoting: the textbook IKJ variant restricted to the pattern of A.
* Table 1, steps 3 and 5-8, with A and q fixed (incompressible, no step 2):
    r = q - A p;  dp1 = P (R A P)^-1 R r;  r1 = r - A dp1;
    dp2 = (LU)^-1 r1;  p = p + dp1 + dp2
  iterated until ||q - A p||_2 <= tol ||q||_2 (q including Dirichlet terms).
* optional sub-block smoothing stage (Sec. 3.2: iterations on the sub-block
  systems of each medium, A^mm and A^ff): after step 7,
    r2 = r1 - A dp2;  dp3 = (L_B U_B)^-1 r2;  p = p + dp3
  with L_B U_B the ILU(0) of A without its cross-medium entries (the media's
  diagonal blocks, wells a block of their own), one application per sweep
  (reading: the paper leaves the stage's iterations open).
* numerically singular coarse system (a reading; the paper is silent):
  Gaussian elimination with partial pivoting meets a pivot at most SING_EPS
  times the largest entry of its row as assembled (`singular_step`).
* flux reconstruction: one FV multiscale stage from x gives p', fluxes across
  primal-block boundaries are T (p'_i - p'_j), and every primal block then
  solves its own TPFA problem with those fluxes as Neumann data (pinned at its
  coarse node when it has no Dirichlet face); fluxes inside a block come from
  that local solution.  R^FV (q - A p') = 0 makes each local problem
  consistent.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

R_FV, R_FE, R_MIX = 0, 1, 2


def restriction(P, primal, n_coarse, kind, n_matrix=None):
    """R^FV (primal-block indicators), R^FE = P^T, or MSMIX (Sec. 3.2): the
    rows of matrix coarse nodes from P^T, the rows of fracture coarse nodes
    (indices from the first fracture block on) from the indicators."""
    n = P.shape[0]
    fv = sp.csr_matrix((np.ones(n), (primal, np.arange(n))), shape=(n_coarse, n))
    if kind == R_FV:
        return fv
    fe = sp.csr_matrix(P.T)
    if kind == R_FE:
        return fe
    nm = n if n_matrix is None else n_matrix
    ncm = int(primal[:nm].max()) + 1 if nm > 0 else 0
    frac_row = (np.arange(n_coarse) >= ncm).astype(np.float64)
    return sp.csr_matrix(sp.diags(1.0 - frac_row) @ fe + sp.diags(frac_row) @ fv)


def coarse_operator(R, A, P):
    Ac = (R @ A @ P).toarray()
    return Ac


def ilu0(A):
    """ILU(0): returns a CSR matrix with the strict lower part of L (unit
    diagonal implied) and the upper part of U in the pattern of A."""
    A = sp.csr_matrix(A, copy=True)
    A.sort_indices()
    n = A.shape[0]
    ip, ix, v = A.indptr, A.indices, A.data.astype(np.float64).copy()
    diag = np.zeros(n, np.int64)
    for i in range(n):
        row = ix[ip[i]:ip[i + 1]]
        k = np.searchsorted(row, i)
        assert k < len(row) and row[k] == i, "missing diagonal"
        diag[i] = ip[i] + k
    for i in range(n):
        a, b = ip[i], ip[i + 1]
        pos = {ix[p]: p for p in range(a, b)}
        for p in range(a, diag[i]):
            k = ix[p]
            v[p] = v[p] / v[diag[k]]
            lik = v[p]
            for q in range(diag[k] + 1, ip[k + 1]):
                j = ix[q]
                pj = pos.get(j)
                if pj is not None:
                    v[pj] -= lik * v[q]
        if v[diag[i]] == 0.0:
            raise ZeroDivisionError("zero pivot in ILU(0)")
    F = sp.csr_matrix((v, ix.copy(), ip.copy()), shape=A.shape)
    return F


def block_matrix(A, medium):
    """A with every entry that couples two media removed, its pattern kept:
    the diagonal blocks A^mm, A^ff (and the wells') in place."""
    C = sp.csr_matrix(A, copy=True)
    rows = np.repeat(np.arange(C.shape[0]), np.diff(C.indptr))
    C.data[np.asarray(medium)[rows] != np.asarray(medium)[C.indices]] = 0.0
    return C


def ilu0_apply(F, r):
    """Solve L U x = r with the factors from ilu0()."""
    L = sp.tril(F, k=-1, format="csr") + sp.identity(F.shape[0], format="csr")
    U = sp.triu(F, k=0, format="csr")
    y = spla.spsolve_triangular(L, r, lower=True, unit_diagonal=True)
    return spla.spsolve_triangular(U, y, lower=False)


class Setup:
    pass


# a pivot at most this fraction of the largest entry of its row (as assembled)
# is numerically zero
SING_EPS = 1e-13


def singular_step(M):
    """First step at which Gaussian elimination with partial pivoting on M
    meets a numerically zero pivot, |u_kk| <= SING_EPS max_j |m_ij| for the
    original row i that became pivot row k; -1 if none.  Invariant under row
    scaling.  An exactly zero column is the extreme case: a coarse node whose
    truncated basis function is its own cell, inside its own primal block, has
    an R^FV column R^FV A e_node that sums A's column over the block, i.e. to
    zero."""
    U = np.array(M, dtype=np.float64, copy=True)
    n = U.shape[0]
    scale = np.abs(U).max(axis=1) if n else np.zeros(0)
    for k in range(n):
        p = k + int(np.argmax(np.abs(U[k:, k])))
        if p != k:
            U[[k, p]] = U[[p, k]]
            scale[[k, p]] = scale[[p, k]]
        if not abs(U[k, k]) > SING_EPS * scale[k]:
            return k
        lk = U[k + 1:, k] / U[k, k]
        U[k + 1:, k:] -= np.outer(lk, U[k, k:])
    return -1


def setup(sysm, P, primal, n_coarse, kind, medium=None):
    """medium (per unknown), when given, adds the sub-block smoothing stage."""
    s = Setup()
    s.A = sysm.A
    s.q = sysm.q
    s.P = P
    s.R = restriction(P, primal, n_coarse, kind, sysm.n_matrix)
    s.Ac = coarse_operator(s.R, sysm.A, P)
    s.lu = sla.lu_factor(s.Ac)
    s.F = ilu0(sysm.A)
    s.Fb = None if medium is None else ilu0(block_matrix(sysm.A, medium))
    return s


def two_stage_solve(s, x0=None, tol=1e-8, max_iter=200, smoother=True, history=False):
    """Table 1 loop.  Returns (p, iterations, final relative residual, converged
    flag, residual history)."""
    A, q = s.A, s.q
    p = np.zeros(A.shape[0]) if x0 is None else np.asarray(x0, np.float64).copy()
    qn = np.linalg.norm(q)
    qn = qn if qn > 0 else 1.0
    r = q - A @ p
    hist = [np.linalg.norm(r) / qn]
    it = 0
    while hist[-1] > tol and it < max_iter:
        dp1 = s.P @ sla.lu_solve(s.lu, s.R @ r)          # step 5
        p = p + dp1
        if smoother:
            r1 = r - A @ dp1                              # step 6
            dp2 = ilu0_apply(s.F, r1)                     # step 7
            p = p + dp2                                   # step 8
            if getattr(s, "Fb", None) is not None:        # sub-block smoothing
                p = p + ilu0_apply(s.Fb, r1 - A @ dp2)
        it += 1
        r = q - A @ p                                     # step 3 of the next sweep
        hist.append(np.linalg.norm(r) / qn)
    return p, it, hist[-1], hist[-1] <= tol, (hist if history else None)


def precondition(s, r, smoother=True):
    """The two-stage step of Table 1 as an operator on a residual r (steps 5-7
    with p = 0): z = dp1 + dp2, dp1 = P A_c^-1 R r, dp2 = (LU)^-1 (r - A dp1).
    Linear in r, so it can precondition a Krylov method (Sec. 4.5, 4.6)."""
    dp1 = s.P @ sla.lu_solve(s.lu, s.R @ r)
    if not smoother:
        return dp1
    z = dp1 + ilu0_apply(s.F, r - s.A @ dp1)
    if getattr(s, "Fb", None) is not None:
        z = z + ilu0_apply(s.Fb, r - s.A @ z)
    return z


def gmres_solve(s, x0=None, tol=1e-8, max_iter=200, restart=30, history=False):
    """GMRES(m) with the two-stage step as right preconditioner: F-AMS as a
    preconditioner for GMRES, the paper's benchmark mode (Sec. 4.5, 4.6, the
    method of Saad's "Iterative Methods for Sparse Linear Systems", right
    preconditioning, Arnoldi by modified Gram-Schmidt, least-squares problem
    by Givens rotations).

    Every Arnoldi step is one iteration (one preconditioner application).
    history[k] is the relative residual after k iterations: the true one at
    the start of each cycle, the least-squares one |g_{j+1}| / ||q|| inside a
    cycle.  A cycle ends when that estimate reaches tol, after `restart`
    steps, or at max_iter; then x = x0 + M^-1 V y and the true residual
    decides whether to stop.  Returns (p, iterations, final true relative
    residual, converged flag, history)."""
    A, q = s.A, s.q
    n = A.shape[0]
    m = int(restart)
    x = np.zeros(n) if x0 is None else np.asarray(x0, np.float64).copy()
    qn = np.linalg.norm(q)
    qn = qn if qn > 0 else 1.0
    r = q - A @ x
    beta = np.linalg.norm(r)
    hist = [beta / qn]
    it = 0
    while hist[-1] > tol and it < max_iter and beta > 0.0:
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        k = 0
        while k < m and it < max_iter:
            w = A @ precondition(s, V[k])
            for i in range(k + 1):                     # modified Gram-Schmidt
                H[i, k] = V[i] @ w
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                         # previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            d = np.hypot(H[k, k], H[k + 1, k])         # new rotation
            cs[k], sn[k] = H[k, k] / d, H[k + 1, k] / d
            H[k, k] = d
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k += 1
            it += 1
            hist.append(abs(g[k]) / qn)
            if hist[-1] <= tol:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):                 # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + precondition(s, V[:k].T @ y)
        r = q - A @ x
        beta = np.linalg.norm(r)
        hist[-1] = beta / qn                           # the true residual ends a cycle
    return x, it, hist[-1], hist[-1] <= tol, (hist if history else None)


def multiscale_stage(s, x):
    """p' = x + P (R A P)^-1 R (q - A x)  (one multiscale stage)."""
    r = s.q - s.A @ x
    return x + s.P @ sla.lu_solve(s.lu, s.R @ r)


def connections(sysm, prob):
    """Every connection (i, j, T) with i < j, in a fixed order: matrix x, y, z
    faces, then matrix-fracture, then fracture-fracture, then the
    perforations of the rate-controlled wells (cell - well, wells in order)."""
    from .assemble import matrix_faces
    nm = sysm.n_matrix
    g = sysm.geom
    out = []
    for lo, hi, T, axis in matrix_faces(prob):
        out.append((lo, hi, T))
    out.append((g.nnc_m, nm + g.nnc_f, sysm.Tmf))
    out.append((nm + g.ff_a, nm + g.ff_b, g.ff_T))
    for cells, wk, beta in getattr(sysm, "well_conn", []):   # rate-controlled wells
        out.append((cells, nm + sysm.n_frac + wk, beta))
    ci = np.concatenate([o[0] for o in out]).astype(np.int64)
    cj = np.concatenate([o[1] for o in out]).astype(np.int64)
    cT = np.concatenate([o[2] for o in out]).astype(np.float64)
    sc = getattr(sysm, "scale", None)
    if sc is not None:
        # a time-step update scaled every connection by the harmonic mean of
        # its cells' mobility scales (Tmf is stored scaled already)
        nmf = len(sysm.Tmf)
        nmat = len(cT) - nmf - len(g.ff_T)
        hm = 2.0 * sc[ci] * sc[cj] / (sc[ci] + sc[cj])
        cT[:nmat] *= hm[:nmat]
        cT[nmat + nmf:] *= hm[nmat + nmf:]
    return ci, cj, cT


def reconstruct_flux(sysm, prob, s_fv, x, primal, node_cell):
    """Conservative flux field from an iterate x.  Returns (conn_flux for every
    connection of connections(), dirichlet_flux for each Dirichlet face), flux
    positive from the first to the second cell / out of the domain."""
    pp = multiscale_stage(s_fv, x)
    ci, cj, cT = connections(sysm, prob)
    dc, dT, dp, _ = sysm.dirichlet
    n = sysm.n
    q_src = sysm.q - sysm.q_dirichlet
    flux = cT * (pp[ci] - pp[cj])
    dflux = np.zeros(len(dc))
    nblk = int(primal.max()) + 1
    members = [[] for _ in range(nblk)]
    for i in range(n):
        members[primal[i]].append(i)
    internal = primal[ci] == primal[cj]
    # boundary (cross-block) fluxes are final: accumulate them as Neumann data
    bnd_out = np.zeros(n)
    np.add.at(bnd_out, ci[~internal], flux[~internal])
    np.subtract.at(bnd_out, cj[~internal], flux[~internal])
    TD = np.zeros(n)
    np.add.at(TD, dc, dT)
    qD = np.zeros(n)
    np.add.at(qD, dc, dT * dp)
    int_idx = np.nonzero(internal)[0]
    blk_of_conn = primal[ci[int_idx]]
    conns_of_blk = [[] for _ in range(nblk)]
    for k, b in zip(int_idx, blk_of_conn):
        conns_of_blk[b].append(k)
    ptil = pp.copy()
    for b in range(nblk):
        cells = members[b]
        m = len(cells)
        loc = {c: t for t, c in enumerate(cells)}
        K = np.zeros((m, m))
        rhs = np.zeros(m)
        for k in conns_of_blk[b]:
            a, c = loc[ci[k]], loc[cj[k]]
            K[a, a] += cT[k]
            K[c, c] += cT[k]
            K[a, c] -= cT[k]
            K[c, a] -= cT[k]
        for t, c in enumerate(cells):
            K[t, t] += TD[c]
            rhs[t] = q_src[c] + qD[c] - bnd_out[c]
        if not np.any(TD[cells] > 0):
            v = loc[node_cell[b]]
            K[v, :] = 0.0
            K[v, v] = 1.0
            rhs[v] = pp[node_cell[b]]
        sol = np.linalg.solve(K, rhs)
        for t, c in enumerate(cells):
            ptil[c] = sol[t]
    flux[internal] = cT[internal] * (ptil[ci[internal]] - ptil[cj[internal]])
    dflux = dT * (ptil[dc] - dp)
    return flux, dflux, pp, ptil


def cell_balance(sysm, prob, flux, dflux):
    """Net outflow minus source per cell (zero for a conservative field)."""
    ci, cj, _ = connections(sysm, prob)
    dc = sysm.dirichlet[0]
    out = np.zeros(sysm.n)
    np.add.at(out, ci, flux)
    np.subtract.at(out, cj, flux)
    np.add.at(out, dc, dflux)
    return out - (sysm.q - sysm.q_dirichlet)
