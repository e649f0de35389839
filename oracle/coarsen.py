"""Oracle: primal/dual coarse grids and the wirebasket classes (Sec. 3, Fig. 2;
Sec. 4.1 Table 2 "distance-based fracture coarsening"; Sec. 4.3 extrusion;
Appendix A permutation of I/F/E/V cells).

TEST INFRASTRUCTURE ONLY (see oracle/geometry.py).

Readings where the paper is silent:
* matrix primal blocks are boxes of C cells per axis (the last one may be
  shorter); the coarse node of a block is the cell start + floor(size/2) along
  each axis, except that with more than one block per axis the first and last
  node lines sit on the boundary cells 0 and n-1 (so that no dual block is a
  half-block with a flat basis function against a Dirichlet face);
* a matrix cell's rank is the number of axes on which it lies on its block's
  node line: 3D ranks V=3, E=2, F=1, I=0; in 2D the same count plus one, so the
  matrix has V, E and F (faces are the lowest class in 2D);
* fracture networks are the connected components of the fracture graph (along
  strike and through intersections; in 3D of its x-y projection, where two
  crossing plates join one network only when they span the same layers: the
  vertical coarse grid of a network is one uniform extrusion, Sec. 4.3, and
  plates of other layer ranges that cross are coarsened as separate networks
  while their fracture-fracture connections stay in A).  Table 2 is
  run per network with: start cell = lowest-index cell of degree 1 (lowest
  index if none), neighbours visited in ascending index, FIFO queues, and a
  candidate removed from Q_vertex whenever its level is lowered;
* 2D fracture cells are V (coarse nodes) or E; 3D fracture cells are V on a
  vertex column and a node layer, E on exactly one of the two, F otherwise;
  the vertical coarse grid of a network starts at its lowest layer with
  frac_cz layers per block (uniform extrusion, Sec. 4.3);
* coarse numbering: matrix blocks lexicographically, then the fracture blocks
  network by network (networks in order of their lowest cell), strike block
  fastest, then vertical block.
"""
from __future__ import annotations

from collections import deque

import numpy as np

RANK_I, RANK_F, RANK_E, RANK_V = 0, 1, 2, 3


def axis_blocks(n, C, boundary_nodes=True):
    """Per cell: block index, and per block: node coordinate.  With more than one
    block the first and last nodes sit on the boundary cells 0 and n-1; every
    other node is at start + floor(size/2)."""
    nb = (n + C - 1) // C
    blk = np.arange(n) // C
    node = np.array([b * C + min(C, n - b * C) // 2 for b in range(nb)], np.int64)
    if boundary_nodes and nb > 1:
        node[0] = 0
        node[-1] = n - 1
    return blk, node, nb


def matrix_coarse(prob):
    nx, ny = prob.nx, prob.ny
    nz = prob.nz if prob.dim == 3 else 1
    cx, cy = prob.coarsen[0], prob.coarsen[1]
    cz = prob.coarsen[2] if prob.dim == 3 else 1
    bx, nodex, nbx = axis_blocks(nx, cx)
    by, nodey, nby = axis_blocks(ny, cy)
    bz, nodez, nbz = axis_blocks(nz, cz)
    X, Y, Z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    X, Y, Z = (a.transpose(2, 1, 0).ravel() for a in (X, Y, Z))
    onx = (X == nodex[bx[X]]).astype(np.int64)
    ony = (Y == nodey[by[Y]]).astype(np.int64)
    cnt = onx + ony
    if prob.dim == 3:
        onz = (Z == nodez[bz[Z]]).astype(np.int64)
        cnt = cnt + onz
        rank = cnt
    else:
        rank = cnt + 1
    primal = bx[X] + nbx * (by[Y] + nby * bz[Z])
    n_coarse = nbx * nby * nbz
    # node cell of each block
    node_cell = np.zeros(n_coarse, np.int64)
    for kz in range(nbz):
        for ky in range(nby):
            for kx in range(nbx):
                node_cell[kx + nbx * (ky + nby * kz)] = (
                    nodex[kx] + nx * (nodey[ky] + ny * (nodez[kz] if prob.dim == 3 else 0)))
    return rank.astype(np.int64), primal.astype(np.int64), node_cell, n_coarse


def fracture_networks(adj):
    """Connected components of the strike graph, labelled in order of their
    lowest cell; returns (label per cell, list of sorted member lists)."""
    n = len(adj)
    lab = np.full(n, -1, np.int64)
    nets = []
    for s in range(n):
        if lab[s] >= 0:
            continue
        comp = [s]
        lab[s] = len(nets)
        q = deque([s])
        while q:
            c = q.popleft()
            for m in adj[c]:
                if lab[m] < 0:
                    lab[m] = len(nets)
                    comp.append(m)
                    q.append(m)
        nets.append(sorted(comp))
    return lab, nets


def bfs_coarsen(cells, adj, dmin):
    """Table 2 on one network.  cells: sorted member list; adj: neighbour lists
    (global strike indices).  dmin <= 0 means infinity.  Returns
    (vertices in creation order, primal dict cell -> block number (0-based),
    level dict)."""
    INF = 1 << 60
    dmax = INF if dmin <= 0 else dmin
    level = {c: INF for c in cells}
    primal = {c: -1 for c in cells}
    deg1 = [c for c in cells if len(adj[c]) == 1]
    start = deg1[0] if deg1 else cells[0]
    qv = deque([start])
    in_qv = {start}
    vertices = []
    while qv:
        v = qv.popleft()
        in_qv.discard(v)
        nprim = len(vertices)
        vertices.append(v)
        primal[v] = nprim
        level[v] = 0
        q1 = deque([v])
        q2 = deque()
        dist = 1
        while dist <= dmax and q1:
            while q1:
                c = q1.popleft()
                for m in adj[c]:
                    if level[m] > dist:
                        if m in in_qv:
                            qv.remove(m)
                            in_qv.discard(m)
                        level[m] = dist
                        primal[m] = nprim
                        q2.append(m)
            q1, q2 = q2, q1
            dist += 1
        # cells reached at exactly dmin become vertex candidates
        if dist > dmax:
            for c in q1:
                qv.append(c)
                in_qv.add(c)
    assert all(p >= 0 for p in primal.values()), "BFS left a cell unassigned"
    return vertices, primal, level


class Coarse:
    pass


def build_coarse(prob, geom):
    """Ranks, primal block ids and coarse numbering for matrix and fracture cells."""
    g = geom
    rank_m, primal_m, node_m, ncm = matrix_coarse(prob)
    nm = g.n_matrix
    nf = g.n_frac
    rank = np.zeros(nm + nf, np.int64)
    primal = np.zeros(nm + nf, np.int64)
    rank[:nm] = rank_m
    primal[:nm] = primal_m
    node_cell = list(node_m)
    lab, nets = fracture_networks(g.strike_adj)
    # strike index -> (fracture, s)
    n_strike = g.n_strike
    s_frac = np.zeros(n_strike, np.int64)
    s_loc = np.zeros(n_strike, np.int64)
    for f in range(len(g.frac_ns)):
        for s in range(g.frac_ns[f]):
            s_frac[g.strike_first[f] + s] = f
            s_loc[g.strike_first[f] + s] = s
    base = ncm
    c = Coarse()
    c.networks = nets
    c.vertices = []
    c.net_layers = []
    dmin = prob.frac_dmin
    for ni, cells in enumerate(nets):
        verts, prim, level = bfs_coarsen(cells, g.strike_adj, dmin)
        c.vertices.append(verts)
        vset = set(verts)
        npr = len(verts)
        if prob.dim == 2:
            for sidx in cells:
                fc = nm + g.frac_first[s_frac[sidx]] + s_loc[sidx]
                rank[fc] = RANK_V if sidx in vset else RANK_E
                primal[fc] = base + prim[sidx]
            for v in verts:
                node_cell.append(nm + g.frac_first[s_frac[v]] + s_loc[v])
            base += npr
            c.net_layers.append((0, 1))
        else:
            fr = sorted({int(s_frac[s]) for s in cells})
            k0s = {(int(g.frac_k0[f]), int(g.frac_nk[f])) for f in fr}
            assert len(k0s) == 1, "a network joins plates of different layer ranges"
            k0, nk = k0s.pop()
            c.net_layers.append((k0, nk))
            cz = max(1, prob.frac_cz)
            vblk, vnode, nvb = axis_blocks(nk, cz)
            for sidx in cells:
                f = s_frac[sidx]
                s = s_loc[sidx]
                ns = g.frac_ns[f]
                for kk in range(nk):
                    fc = nm + g.frac_first[f] + s + ns * kk
                    onv = sidx in vset
                    onl = kk == vnode[vblk[kk]]
                    rank[fc] = RANK_V if (onv and onl) else (RANK_E if (onv or onl) else RANK_F)
                    primal[fc] = base + prim[sidx] + npr * vblk[kk]
            for vb in range(nvb):
                for v in verts:
                    f = s_frac[v]
                    node_cell.append(nm + g.frac_first[f] + s_loc[v] + g.frac_ns[f] * vnode[vb])
            base += npr * nvb
    # each rate-controlled well: one fine DOF, its own coarse node and primal
    # block (Sec. 3: mapped to the coarse scale by the identity), rank V
    nw = sum(1 for wl in (getattr(prob, "wells", None) or []) if wl.control == 0)
    if nw:
        rank = np.concatenate([rank, np.full(nw, RANK_V, np.int64)])
        primal = np.concatenate([primal, base + np.arange(nw)])
        node_cell.extend(nm + nf + np.arange(nw))
        base += nw
    # coarsening network of every fracture row (-1 for matrix and well rows)
    row_net = np.full(nm + nf + nw, -1, np.int64)
    for f in range(len(g.frac_ns)):
        ns = g.frac_ns[f]
        nk = g.frac_nk[f] if prob.dim == 3 else 1
        for kk in range(nk):
            for s in range(ns):
                row_net[nm + g.frac_first[f] + s + ns * kk] = lab[g.strike_first[f] + s]
    c.row_net = row_net
    c.rank = rank
    c.primal = primal
    c.node_cell = np.array(node_cell, np.int64)
    c.n_coarse = base
    c.n_coarse_matrix = ncm
    c.n_well = nw
    c.medium = np.concatenate([np.zeros(nm, np.int64), np.ones(nf, np.int64),
                               np.full(nw, 2, np.int64)])
    return c
