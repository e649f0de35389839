"""Oracle: the fine-scale EDFM pressure system A p = q (Sec. 2, Eqs. 1-8).

TEST INFRASTRUCTURE ONLY (see oracle/geometry.py).

Incompressible single phase, mu = rho = 1, so lambda = k.  The system is
integrated over each control volume, so every connection contributes one
transmissibility T to both of its cells and A is symmetric:

  row i:  sum_j T_ij (p_i - p_j) + T_D,i (p_i - p_D) = q_i

* matrix-matrix: two-point flux, harmonic average of the half-cell
  transmissibilities, T = A_face / (h/(2 k_i) + h/(2 k_j));
* Dirichlet faces: half-cell transmissibility T_D = 2 k_i A_face / h;
* matrix-fracture: T = CI_ij lambda^{f-m} with CI_ij = A_ij / <d>_ij (Eq. 7)
  and lambda^{f-m} read as the matrix cell's k (the paper leaves it open);
  eta^m V = eta^f A = CI lambda (Eqs. 4-6) makes the pair symmetric;
* fracture-fracture: along strike k_f a_f depth / h_s, vertically
  k_f a_f h_s / dz, intersections as built in geometry.py.

* wells (Sec. 2, q^mw = PI lambda^m (p^w - p^m) / V, volume-integrated): a
  perforation of matrix cell i connects it to its well with
  beta_i = PI_i k_i.  A rate-controlled well is one more unknown p^w (the
  paper gives each well a single fine-scale DOF, Sec. 3) with the equation
  sum_i beta_i (p^w - p_i) = Q_w; a pressure-controlled well (p^w fixed)
  acts on its perforated cells like a Dirichlet half-cell: beta_i (p_i -
  p_bhp), kept out of A0 like the Dirichlet faces.

Unknown order: matrix cells (x fastest, then y, then z), then fracture cells,
then the rate-controlled wells in input order (Eq. 8 block order [m; f; w]).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import build_geometry


class System:
    pass


def matrix_faces(prob):
    """All interior matrix faces as (cell_lo, cell_hi, T, axis), ordered by axis
    then by the low cell."""
    nx, ny = prob.nx, prob.ny
    nz = prob.nz if prob.dim == 3 else 1
    k = np.asarray(prob.perm, np.float64).reshape(nz, ny, nx)
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    out = []
    # x faces
    area, h = dy * dz, dx
    kl, kr = k[:, :, :-1], k[:, :, 1:]
    T = area / (h / (2 * kl) + h / (2 * kr))
    out.append((idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel(), T.ravel(), 0))
    area, h = dx * dz, dy
    kl, kr = k[:, :-1, :], k[:, 1:, :]
    T = area / (h / (2 * kl) + h / (2 * kr))
    out.append((idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel(), T.ravel(), 1))
    if prob.dim == 3:
        area, h = dx * dy, dz
        kl, kr = k[:-1, :, :], k[1:, :, :]
        T = area / (h / (2 * kl) + h / (2 * kr))
        out.append((idx[:-1, :, :].ravel(), idx[1:, :, :].ravel(), T.ravel(), 2))
    return out


def dirichlet_terms(prob):
    """Half-cell transmissibility and value on each Dirichlet boundary face.
    Returns (cell, T_D, p_D, face_id) arrays; face ids 0..5 = W,E,S,N,B,T."""
    nx, ny = prob.nx, prob.ny
    nz = prob.nz if prob.dim == 3 else 1
    k = np.asarray(prob.perm, np.float64).reshape(nz, ny, nx)
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    cells, tds, pds, fids = [], [], [], []
    faces = [
        (0, idx[:, :, 0], k[:, :, 0], dy * dz, dx),
        (1, idx[:, :, -1], k[:, :, -1], dy * dz, dx),
        (2, idx[:, 0, :], k[:, 0, :], dx * dz, dy),
        (3, idx[:, -1, :], k[:, -1, :], dx * dz, dy),
    ]
    if prob.dim == 3:
        faces += [(4, idx[0, :, :], k[0, :, :], dx * dy, dz),
                  (5, idx[-1, :, :], k[-1, :, :], dx * dy, dz)]
    for fid, cid, kk, area, h in faces:
        if not (prob.bc_mask >> fid) & 1:
            continue
        cells.append(cid.ravel())
        tds.append((2.0 * kk * area / h).ravel())
        pds.append(np.full(cid.size, float(prob.bc_value[fid])))
        fids.append(np.full(cid.size, fid))
    if not cells:
        return (np.zeros(0, np.int64), np.zeros(0), np.zeros(0), np.zeros(0, np.int64))
    return (np.concatenate(cells), np.concatenate(tds), np.concatenate(pds),
            np.concatenate(fids))


WELL_RATE, WELL_PRESSURE = 0, 1


def well_terms(prob):
    """(rate-well connections (cell, well k, beta), pressure-well terms (cell,
    beta, p_bhp, well index)) in input order; beta = PI k of the cell."""
    perm = np.asarray(prob.perm, np.float64)
    rate, pres = [], []
    nw = 0
    for w, wl in enumerate(getattr(prob, "wells", None) or []):
        cells = np.asarray(wl.cells, np.int64)
        beta = np.asarray(wl.pi, np.float64) * perm[cells]
        if wl.control == WELL_RATE:
            rate.append((cells, np.full(len(cells), nw), beta))
            nw += 1
        else:
            pres.append((cells, beta, np.full(len(cells), float(wl.value)), np.full(len(cells), w)))
    return rate, pres, nw


def assemble(prob, geom=None):
    """Build A (with Dirichlet terms), A0 (without them) and the total rhs."""
    g = build_geometry(prob) if geom is None else geom
    nm, nf = g.n_matrix, g.n_frac
    rate, pres, nw = well_terms(prob)
    n = nm + nf + nw
    perm = np.asarray(prob.perm, np.float64)
    rows, cols, vals = [], [], []
    conns = []  # (i, j, T) for every connection, i < j

    for lo, hi, T, axis in matrix_faces(prob):
        conns.append((lo, hi, T))
    # matrix-fracture: T = CI * k_m  (Eqs. 4-7)
    Tmf = g.nnc_area / g.nnc_dist * perm[g.nnc_m]
    conns.append((g.nnc_m, nm + g.nnc_f, Tmf))
    conns.append((nm + g.ff_a, nm + g.ff_b, g.ff_T))
    # rate-controlled wells: perforated cell - well DOF
    for cells, wk, beta in rate:
        conns.append((cells, nm + nf + wk, beta))

    for i, j, T in conns:
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [-T, -T, T, T]
    A0 = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n, n))
    A0.sum_duplicates()
    A0.sort_indices()
    dc, dT, dp, dfid = dirichlet_terms(prob)
    # pressure-controlled wells join the Dirichlet terms (face id 6 + well)
    for cells, beta, pb, w in pres:
        dc = np.concatenate([dc, cells])
        dT = np.concatenate([dT, beta])
        dp = np.concatenate([dp, pb])
        dfid = np.concatenate([dfid, 6 + w])
    D = np.zeros(n)
    np.add.at(D, dc, dT)
    qD = np.zeros(n)
    np.add.at(qD, dc, dT * dp)
    A = (A0 + sp.diags(D)).tocsr()
    A.sort_indices()
    # A0's pattern must include the diagonal even where it is 0 (it never is here)
    s = System()
    s.geom = g
    s.n = n
    s.n_matrix = nm
    s.n_frac = nf
    s.n_well = nw
    s.well_conn = rate
    s.A = A
    s.A0 = A0
    s.T_D = D
    s.q_dirichlet = qD
    src = np.zeros(n)
    if prob.rhs is not None:
        r = np.asarray(prob.rhs, np.float64)
        src[:len(r)] = r
    k = 0
    for wl in getattr(prob, "wells", None) or []:
        if wl.control == WELL_RATE:
            src[nm + nf + k] += wl.value   # total injection rate Q_w
            k += 1
    s.q = src + qD
    s.dirichlet = (dc, dT, dp, dfid)
    s.Tmf = Tmf
    return s


def update_mobility(sysm, scale):
    """Time-step update of the fine system (the reading of a mobility change
    between time steps, where the basis functions are kept): every
    connection's transmissibility is multiplied by the harmonic mean
    2 s_i s_j / (s_i + s_j) of its two cells' mobility scales, a Dirichlet
    half-cell transmissibility by its cell's scale.  The pattern does not
    change; A0, A, the Dirichlet terms and q follow.  Returns a new System
    carrying `scale` (the flux reconstruction applies it to the connections)."""
    import copy
    sc = np.asarray(scale, np.float64)
    out = copy.copy(sysm)
    C = sp.coo_matrix(sysm.A0)
    off = C.row != C.col
    r, c, v = C.row[off], C.col[off], C.data[off]
    hm = 2.0 * sc[r] * sc[c] / (sc[r] + sc[c])
    v = v * hm
    n = sysm.n
    diag = np.zeros(n)
    np.subtract.at(diag, r, v)
    A0 = sp.csr_matrix((np.concatenate([v, diag]), (np.concatenate([r, np.arange(n)]),
                                                   np.concatenate([c, np.arange(n)]))),
                       shape=(n, n))
    A0.sort_indices()
    out.A0 = A0
    out.T_D = sysm.T_D * sc
    src = sysm.q - sysm.q_dirichlet
    out.q_dirichlet = sysm.q_dirichlet * sc
    out.q = src + out.q_dirichlet
    out.A = (A0 + sp.diags(out.T_D)).tocsr()
    out.A.sort_indices()
    dc, dT, dp, dfid = sysm.dirichlet
    out.dirichlet = (dc, dT * sc[dc], dp, dfid)
    out.Tmf = sysm.Tmf * (2.0 * sc[sysm.geom.nnc_m] * sc[sysm.n_matrix + sysm.geom.nnc_f]
                          / (sc[sysm.geom.nnc_m] + sc[sysm.n_matrix + sysm.geom.nnc_f]))
    out.scale = sc
    return out
