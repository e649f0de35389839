"""Oracle: F-AMS basis functions and the prolongation P (Sec. 3.1, Eqs. 9-22;
Appendix A, Eqs. A.1-A.12), and truncation (Sec. 4.3).

TEST INFRASTRUCTURE ONLY (see oracle/geometry.py).

Two routes, checked against each other in the tests:

1. ``prolongation_staged`` - the wirebasket procedure of Sec. 3.1 applied row
   block by row block: vertex rows are the Kronecker delta (Eq. 16); then every
   stage (edges, faces, interiors; per coupling strategy also per medium)
   solves, for each connected dual block B of the stage,
       A'_BB P_B = sum_{known c} T_rc P_c
   where A' keeps the links that the coupling strategy keeps and removes every
   dropped link from the diagonal (the overline / underline notation of
   Appendix A).  Kept links point to cells of equal or higher rank, so their
   rows are already known.
2. ``prolongation_appendix`` - the block formulas printed in Appendix A for
   each strategy (Eqs. A.5, A.7-A.8, A.9-A.10, A.12), evaluated on the
   permuted blocks I/F/E/V of each medium with sparse direct solves.

Keep rule (row r, neighbour c, ranks V=3 > E=2 > F=1 > I=0):
  Decoupled : same medium and rank(c) >= rank(r)
  Frac-AMS  : matrix rows also keep every fracture link (Phi^ff is known and
              acts as Dirichlet data, Eq. 20); fracture rows drop matrix links
  Rock-AMS  : mirror image (Eq. 21)
  Coupled   : rank(c) >= rank(r) regardless of medium; same-rank links across
              the media merge dual blocks (Fig. 7, Eq. 22)
The basis is built from A0, the fine matrix without Dirichlet terms, so every
row of P sums to one (partition of unity, end of Sec. 3.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

from .coarsen import RANK_E, RANK_F, RANK_I, RANK_V

DECOUPLED, FRAC, ROCK, COUPLED = 0, 1, 2, 3
M, F, W = 0, 1, 2   # media: matrix, fractures, wells


def keep_link(variant, med_r, rank_r, med_c, rank_c, cross=0):
    """cross: 1 if the link joins cells of two different fractures of one
    coarsening network (a crossing), 2 if of two different networks.  Two
    fracture faces never share a link: faces of different fractures meet only
    along edges, so a face-face link across a crossing is dropped.  Networks
    are coarsened apart (3D plates of other layer ranges that cross), so
    their wirebaskets are unrelated and no link between two of them is
    kept: each network's basis functions are built on that network alone."""
    if med_c == W:
        return True    # a well's value is known (P^ww = I): the beta term of Eq. 18
    if med_r == W:
        return False   # well rows are coarse nodes
    if cross == 2 and med_r == F and med_c == F:
        return False
    if cross and med_r == F and med_c == F and rank_r == RANK_F and rank_c == RANK_F:
        return False
    if variant == DECOUPLED:
        return med_r == med_c and rank_c >= rank_r
    if variant == FRAC:
        if med_r == M:
            return med_c == F or rank_c >= rank_r
        return med_c == F and rank_c >= rank_r
    if variant == ROCK:
        if med_r == F:
            return med_c == M or rank_c >= rank_r
        return med_c == M and rank_c >= rank_r
    return rank_c >= rank_r


def stage_list(variant):
    """Stages as lists of (medium, rank) classes, in solve order."""
    mE, mF, mI = (M, RANK_E), (M, RANK_F), (M, RANK_I)
    fE, fF = (F, RANK_E), (F, RANK_F)
    if variant == DECOUPLED:
        return [[mE], [fE], [mF], [fF], [mI]]
    if variant == FRAC:
        return [[fE], [fF], [mE], [mF], [mI]]
    if variant == ROCK:
        return [[mE], [mF], [mI], [fE], [fF]]
    return [[mE, fE], [mF, fF], [mI]]


def _plate_of(n, plate):
    return np.full(n, -1, np.int64) if plate is None else np.asarray(plate, np.int64)


def _cross(plate, net, r, c):
    """0: not two fractures' cells; 1: two fractures of one network; 2: two
    networks (net None: one network)."""
    if plate[r] < 0 or plate[c] < 0 or plate[r] == plate[c]:
        return 0
    if net is not None and net[r] != net[c]:
        return 2
    return 1


def merge_capped(n_cells, same_links, cross_links, cap):
    """Dual blocks of a Coupled stage under a merge cap (Sec. 3.1: one can
    limit the size of the blocks that same-rank links across the media
    merge).  Reading: the blocks of each medium alone (connected components
    of `same_links`) are merged through the cross-medium links taken in the
    given order (the CSR order of A: lower row first, then column), a link
    joining two blocks only when the merged block holds at most `cap` cells.
    Returns a block label per cell (the lowest cell of its block)."""
    parent = list(range(n_cells))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in same_links:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    size = [0] * n_cells
    for x in range(n_cells):
        size[find(x)] += 1
    for a, b in cross_links:
        ra, rb = find(a), find(b)
        if ra != rb and size[ra] + size[rb] <= cap:
            lo, hi = min(ra, rb), max(ra, rb)
            parent[hi] = lo
            size[lo] += size[hi]
    return [find(x) for x in range(n_cells)]


def _stage_labels(A0, S, in_stage, medium, keep, variant, merge_cap):
    """Block label (position in S of the block's lowest cell) of every cell of
    a stage S: connected components of the kept links inside the stage; for
    Coupled with merge_cap > 0, cross-medium links merge blocks only within
    the cap (merge_capped)."""
    ip, ix = A0.indptr, A0.indices
    loc = -np.ones(A0.shape[0], np.int64)
    loc[S] = np.arange(S.size)
    same, cross = [], []
    for r in S:
        for p in range(ip[r], ip[r + 1]):
            c = ix[p]
            if c > r and in_stage[c] and keep(r, c):
                (cross if (variant == COUPLED and merge_cap > 0 and medium[r] != medium[c])
                 else same).append((int(loc[r]), int(loc[c])))
    cap = merge_cap if merge_cap > 0 else S.size
    return np.asarray(merge_capped(S.size, same, cross, cap), np.int64)


def stage_blocks(A0, rank, medium, node_cell, variant, plate=None, net=None, merge_cap=0,
                 with_stage=False):
    """The dual blocks of every stage (lists of rows), in solve order
    (with_stage: (stage index, rows) pairs)."""
    A0 = sp.csr_matrix(A0)
    n = A0.shape[0]
    plate = _plate_of(n, plate)
    known = np.zeros(n, bool)
    known[np.asarray(node_cell)] = True
    ip, ix = A0.indptr, A0.indices
    out = []
    for si, stage in enumerate(stage_list(variant)):
        in_stage = np.zeros(n, bool)
        for (med, rk) in stage:
            in_stage |= (medium == med) & (rank == rk)
        in_stage &= ~known
        S = np.nonzero(in_stage)[0]
        if S.size == 0:
            continue

        def keep(r, c):
            return keep_link(variant, medium[r], rank[r], medium[c], rank[c],
                             _cross(plate, net, r, c))
        lab = _stage_labels(A0, S, in_stage, medium, keep, variant, merge_cap)
        members = {}
        for li, r in enumerate(S):
            members.setdefault(int(lab[li]), []).append(int(r))
        for k in sorted(members):
            out.append((si, members[k]) if with_stage else members[k])
        known |= in_stage
    return out


def cut_links(A0, rank, medium, node_cell, variant, plate=None, net=None, merge_cap=0):
    """Links that the keep rule keeps but the merge cap cuts: same-stage
    cross-medium links between two different blocks (Coupled only)."""
    A0 = sp.csr_matrix(A0)
    blocks = stage_blocks(A0, rank, medium, node_cell, variant, plate, net, merge_cap, True)
    blk = -np.ones(A0.shape[0], np.int64)
    stg = -np.ones(A0.shape[0], np.int64)
    for b, (si, cells) in enumerate(blocks):
        blk[cells] = b
        stg[cells] = si
    out = []
    ip, ix = A0.indptr, A0.indices
    for r in range(A0.shape[0]):
        if blk[r] < 0:
            continue
        for p in range(ip[r], ip[r + 1]):
            c = ix[p]
            if c != r and stg[c] == stg[r] and blk[c] != blk[r] and keep_link(
                    variant, medium[r], rank[r], medium[c], rank[c], _cross(plate, net, r, c)):
                out.append((r, c))
    return out


def prolongation_staged(A0, rank, medium, node_cell, variant, plate=None, net=None,
                        merge_cap=0, old=None, marked=None):
    """P (CSR, n x n_coarse) by the staged wirebasket rule.  plate[r]: input
    fracture of fracture row r (-1 for matrix rows; None: no crossings);
    net[r]: coarsening network of fracture row r (None: a single network);
    merge_cap: largest Coupled block merged across the media (0: no cap); a
    kept link between two blocks of one stage (cut by the cap) is dropped
    and removed from the diagonal.

    Adaptive update (old: the untruncated P of the last build, marked: the
    cells whose mobility moved beyond the threshold): a dual block is solved
    again, with this A0, only if it holds a marked cell or reads a row of a
    block solved again in an earlier stage; the other blocks keep their rows
    of `old`.  Returns (P, recomputed rows, blocks solved) then."""
    A0 = sp.csr_matrix(A0)
    n = A0.shape[0]
    plate = _plate_of(n, plate)

    def keep(r, c):
        return keep_link(variant, medium[r], rank[r], medium[c], rank[c], _cross(plate, net, r, c))

    nc = len(node_cell)
    rows = [dict() for _ in range(n)]
    known = np.zeros(n, bool)
    for j, v in enumerate(node_cell):
        rows[v] = {j: 1.0}
        known[v] = True
    ip, ix, dv = A0.indptr, A0.indices, A0.data
    adaptive = old is not None
    recomputed = np.zeros(n, bool)
    solved = 0
    if adaptive:
        old = sp.csr_matrix(old)
    for stage in stage_list(variant):
        in_stage = np.zeros(n, bool)
        for (med, rk) in stage:
            in_stage |= (medium == med) & (rank == rk)
        in_stage &= ~known
        S = np.nonzero(in_stage)[0]
        if S.size == 0:
            continue
        # links kept inside the stage define the dual blocks
        lab = _stage_labels(A0, S, in_stage, medium, keep, variant, merge_cap)
        members = {}
        for li, r in enumerate(S):
            members.setdefault(int(lab[li]), []).append(r)
        for key in sorted(members):
            cells = members[key]
            cells = sorted(cells)
            if adaptive:
                dirty = bool(np.asarray(marked)[cells].any())
                if not dirty:
                    for r in cells:
                        for p in range(ip[r], ip[r + 1]):
                            c = ix[p]
                            if c != r and recomputed[c] and keep(r, c) and not in_stage[c]:
                                dirty = True
                                break
                        if dirty:
                            break
                if not dirty:
                    for r in cells:
                        a, e = old.indptr[r], old.indptr[r + 1]
                        rows[r] = dict(zip(old.indices[a:e].tolist(), old.data[a:e].tolist()))
                    continue
                recomputed[cells] = True
                solved += 1
            b = len(cells)
            bl = {r: i for i, r in enumerate(cells)}
            Ab = np.zeros((b, b))
            rhs = {}
            for i, r in enumerate(cells):
                diag = 0.0
                for p in range(ip[r], ip[r + 1]):
                    c = ix[p]
                    a = dv[p]
                    if c == r:
                        diag += a
                        continue
                    T = -a
                    if keep(r, c) and (c in bl or not in_stage[c]):
                        if c in bl:
                            Ab[i, bl[c]] = a
                        else:
                            assert known[c], "kept link to a row that is not built yet"
                            for col, val in rows[c].items():
                                rhs.setdefault(col, np.zeros(b))[i] += T * val
                    else:
                        diag -= T
                Ab[i, i] = diag
            if not rhs:
                raise ValueError("dual block without a link to known values")
            cols = sorted(rhs)
            B = np.stack([rhs[c] for c in cols], axis=1)
            X = np.linalg.solve(Ab, B)
            for i, r in enumerate(cells):
                rows[r] = {col: X[i, k] for k, col in enumerate(cols) if X[i, k] != 0.0}
        known |= in_stage
    assert known.all(), "cells left without a basis row"
    ri, ci, vv = [], [], []
    for r in range(n):
        for col in sorted(rows[r]):
            ri.append(r)
            ci.append(col)
            vv.append(rows[r][col])
    P = sp.csr_matrix((vv, (ri, ci)), shape=(n, nc))
    P.sort_indices()
    if adaptive:
        return P, recomputed, solved
    return P


def _mod_diag(A0, X, drop):
    """A0[X,X] with every link from a row of X to a cell of `drop` removed from
    its diagonal (the overline/underline of Appendix A)."""
    sub = A0[X][:, X].tolil()
    Ad = A0[X][:, drop] if len(drop) else None
    if Ad is not None:
        s = np.asarray(Ad.sum(axis=1)).ravel()   # sum of -T over dropped links
        for i in range(len(X)):
            sub[i, i] = sub[i, i] + s[i]
    return sp.csc_matrix(sub)


def _solve(Ablk, R):
    if Ablk.shape[0] == 0:
        return sp.csr_matrix(R.shape)
    lu = spla.splu(sp.csc_matrix(Ablk))
    Rd = R.toarray() if sp.issparse(R) else np.asarray(R)
    return sp.csr_matrix(lu.solve(Rd))


def prolongation_appendix(A0, rank, medium, node_cell, variant, plate=None, net=None,
                          merge_cap=0):
    """P from the printed block formulas of Appendix A (regular wirebasket:
    the blocks that the TPFA stencil makes zero are taken as zero).  Face-face
    links across fracture crossings, every link between two coarsening
    networks, and the links a Coupled merge cap cuts, are dropped from A0
    first (removed from the diagonal), as in keep_link and
    prolongation_staged."""
    A0 = sp.csr_matrix(A0)
    n = A0.shape[0]
    plate = _plate_of(n, plate)
    cut = cut_links(A0, rank, medium, node_cell, variant, plate, net, merge_cap) \
        if merge_cap > 0 else []
    A0 = A0.tolil()
    for r, c in cut:
        A0[r, r] = A0[r, r] + A0[r, c]
        A0[r, c] = 0.0
    for r in np.nonzero(medium == F)[0]:
        for c in list(A0.rows[r]):
            if c == r or medium[c] != F:
                continue
            x = _cross(plate, net, r, c)
            if x == 2 or (x == 1 and rank[r] == RANK_F and rank[c] == RANK_F):
                A0[r, r] = A0[r, r] + A0[r, c]
                A0[r, c] = 0.0
    A0 = sp.csr_matrix(A0)
    A0.eliminate_zeros()
    nc = len(node_cell)
    cls = {}
    for med in (M, F):
        for rk in (RANK_I, RANK_F, RANK_E, RANK_V):
            cls[(med, rk)] = np.nonzero((medium == med) & (rank == rk))[0]
    allm = np.nonzero(medium == M)[0]
    allf = np.nonzero(medium == F)[0]
    col_of = {v: j for j, v in enumerate(node_cell)}
    Vm, Vf = cls[(M, RANK_V)], cls[(F, RANK_V)]
    colsVm = np.array([col_of[v] for v in Vm], np.int64)
    colsVf = np.array([col_of[v] for v in Vf], np.int64)
    Im, Fm, Em = cls[(M, RANK_I)], cls[(M, RANK_F)], cls[(M, RANK_E)]
    Ff, Ef = cls[(F, RANK_F)], cls[(F, RANK_E)]

    def lower(X_rank, med):
        return np.nonzero((medium == med) & (rank < X_rank))[0]

    def B(X, Y):
        return A0[X][:, Y]

    P = sp.lil_matrix((n, nc))
    for v, j in col_of.items():
        P[v, j] = 1.0

    def put(rows, cols, val):
        val = sp.csr_matrix(val)
        val.eliminate_zeros()
        for i, r in enumerate(rows):
            for p in range(val.indptr[i], val.indptr[i + 1]):
                P[r, cols[val.indices[p]]] = val.data[p]

    def medium_chain(med, other_drop, extra_cols=None):
        """Decoupled-style chain E -> F -> I inside one medium, columns = own V.
        other_drop: also remove the other medium's links from the diagonal."""
        E_, F_, I_ = (Em, Fm, Im) if med == M else (Ef, Ff, np.zeros(0, np.int64))
        V_ = Vm if med == M else Vf
        oth = allf if med == M else allm
        dropE = np.concatenate([lower(RANK_E, med), oth if other_drop else []]).astype(np.int64)
        dropF = np.concatenate([lower(RANK_F, med), oth if other_drop else []]).astype(np.int64)
        dropI = (oth if other_drop else np.zeros(0)).astype(np.int64)
        PE = -_solve(_mod_diag(A0, E_, dropE), B(E_, V_)) if len(E_) else sp.csr_matrix((0, len(V_)))
        PF = -_solve(_mod_diag(A0, F_, dropF), B(F_, E_) @ PE) if len(F_) else sp.csr_matrix((0, len(V_)))
        PI = -_solve(_mod_diag(A0, I_, dropI), B(I_, F_) @ PF) if len(I_) else sp.csr_matrix((0, len(V_)))
        return PE, PF, PI

    if variant in (DECOUPLED, FRAC, ROCK):
        # own-medium columns
        dropm = variant in (DECOUPLED, ROCK)     # matrix rows drop fracture links
        dropf = variant in (DECOUPLED, FRAC)     # fracture rows drop matrix links
        PEm, PFm, PIm = medium_chain(M, dropm)
        PEf, PFf, _ = medium_chain(F, dropf)
        put(Em, colsVm, PEm)
        put(Fm, colsVm, PFm)
        put(Im, colsVm, PIm)
        put(Ef, colsVf, PEf)
        put(Ff, colsVf, PFf)
        if variant == FRAC:
            # Eqs. A.7-A.8: matrix rows, fracture columns, with P^{fV^f} as data
            PfVf = sp.lil_matrix((len(allf), len(Vf)))
            fpos = {c: i for i, c in enumerate(allf)}
            for r in allf:
                for k, v in enumerate(Vf):
                    PfVf[fpos[r], k] = P[r, colsVf[k]]
            PfVf = sp.csr_matrix(PfVf)
            PEmf = -_solve(_mod_diag(A0, Em, lower(RANK_E, M)), B(Em, allf) @ PfVf)
            PFmf = -_solve(_mod_diag(A0, Fm, lower(RANK_F, M)),
                           B(Fm, Em) @ PEmf + B(Fm, allf) @ PfVf)
            put(Em, colsVf, PEmf)
            put(Fm, colsVf, PFmf)
            if len(Im):
                PImf = -_solve(_mod_diag(A0, Im, np.zeros(0, np.int64)),
                               B(Im, Fm) @ PFmf + B(Im, allf) @ PfVf)
                put(Im, colsVf, PImf)
            # matrix rows, matrix columns: overline only (fracture links stay on the diagonal)
            PEm2 = -_solve(_mod_diag(A0, Em, lower(RANK_E, M)), B(Em, Vm))
            PFm2 = -_solve(_mod_diag(A0, Fm, lower(RANK_F, M)), B(Fm, Em) @ PEm2)
            put(Em, colsVm, PEm2)
            put(Fm, colsVm, PFm2)
            if len(Im):
                PIm2 = -_solve(_mod_diag(A0, Im, np.zeros(0, np.int64)), B(Im, Fm) @ PFm2)
                put(Im, colsVm, PIm2)
        if variant == ROCK:
            # Eqs. A.9-A.10: fracture rows, matrix columns, with P^{mV^m} as data
            PmVm = sp.lil_matrix((len(allm), len(Vm)))
            mpos = {c: i for i, c in enumerate(allm)}
            Pl = sp.csr_matrix(P)
            for r in allm:
                for p in range(Pl.indptr[r], Pl.indptr[r + 1]):
                    c = Pl.indices[p]
                    k = np.nonzero(colsVm == c)[0]
                    if k.size:
                        PmVm[mpos[r], k[0]] = Pl.data[p]
            PmVm = sp.csr_matrix(PmVm)
            PEfm = -_solve(_mod_diag(A0, Ef, lower(RANK_E, F)), B(Ef, allm) @ PmVm)
            put(Ef, colsVm, PEfm)
            if len(Ff):
                PFfm = -_solve(_mod_diag(A0, Ff, lower(RANK_F, F)),
                               B(Ff, Ef) @ PEfm + B(Ff, allm) @ PmVm)
                put(Ff, colsVm, PFfm)
            PEf2 = -_solve(_mod_diag(A0, Ef, lower(RANK_E, F)), B(Ef, Vf))
            put(Ef, colsVf, PEf2)
            if len(Ff):
                PFf2 = -_solve(_mod_diag(A0, Ff, lower(RANK_F, F)), B(Ff, Ef) @ PEf2)
                put(Ff, colsVf, PFf2)
    else:
        # Coupled (Eq. A.12): merged classes, all coarse nodes together
        E_ = np.sort(np.concatenate([Em, Ef]))
        F_ = np.sort(np.concatenate([Fm, Ff]))
        I_ = Im
        V_ = np.array(list(col_of.keys()), np.int64)
        colsV = np.array([col_of[v] for v in V_], np.int64)
        lowE = np.nonzero(rank < RANK_E)[0]
        lowF = np.nonzero(rank < RANK_F)[0]
        PEV = -_solve(_mod_diag(A0, E_, lowE), B(E_, V_)) if len(E_) else None
        put(E_, colsV, PEV) if len(E_) else None
        if len(F_):
            rhsF = B(F_, V_) + (B(F_, E_) @ PEV if len(E_) else 0)
            PFV = -_solve(_mod_diag(A0, F_, lowF), rhsF)
            put(F_, colsV, PFV)
        if len(I_):
            rhsI = B(I_, V_) + B(I_, F_) @ PFV + (B(I_, E_) @ PEV if len(E_) else 0)
            PIV = -_solve(_mod_diag(A0, I_, np.zeros(0, np.int64)), rhsI)
            put(I_, colsV, PIV)
    P = sp.csr_matrix(P)
    P.eliminate_zeros()
    P.sort_indices()
    return P


def truncate(P, alpha):
    """Sec. 4.3: drop entries with |P_ij| < alpha and divide each row by its new
    sum.  A row that would lose every entry keeps its largest one (lowest
    column on ties).  alpha = 0 leaves P unchanged."""
    P = sp.csr_matrix(P, copy=True)
    if alpha <= 0.0:
        return P
    ri, ci, vv = [], [], []
    for r in range(P.shape[0]):
        a, b = P.indptr[r], P.indptr[r + 1]
        cols = P.indices[a:b]
        vals = P.data[a:b]
        keep = np.abs(vals) >= alpha
        if not keep.any() and b > a:
            keep = np.zeros(b - a, bool)
            keep[int(np.argmax(np.abs(vals)))] = True
        s = vals[keep].sum()
        for c, v in zip(cols[keep], vals[keep]):
            ri.append(r)
            ci.append(c)
            vv.append(v / s)
    Q = sp.csr_matrix((vv, (ri, ci)), shape=P.shape)
    Q.sort_indices()
    return Q
