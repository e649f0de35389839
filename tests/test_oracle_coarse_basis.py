"""Pins of the oracle's coarse grids (Sec. 3, Table 2) and basis functions
(Sec. 3.1, Appendix A)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble, basis, coarsen, geometry
from paper_1705_05784_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "bfs_networks.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, val = line.partition(" ")
        if key == "case":
            cur = {"name": val}
        elif key == "end":
            cases.append(cur)
        elif key == "edges":
            cur["edges"] = [tuple(int(t) for t in e.split("-")) for e in val.split()]
        elif key in ("vertices", "primal"):
            cur[key] = [int(t) for t in val.split()]
        else:
            cur[key] = int(val)
    return cases


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_bfs_golden(case):
    n = case["n"]
    adj = [set() for _ in range(n)]
    for a, b in case["edges"]:
        adj[a].add(b)
        adj[b].add(a)
    adj = [sorted(s) for s in adj]
    verts, prim, level = coarsen.bfs_coarsen(list(range(n)), adj, case["dmin"])
    assert verts == case["vertices"]
    assert [prim[c] for c in range(n)] == case["primal"]


def _bfs_dist(adj, src):
    from collections import deque
    d = {src: 0}
    q = deque([src])
    while q:
        c = q.popleft()
        for m in adj[c]:
            if m not in d:
                d[m] = d[c] + 1
                q.append(m)
    return d


def test_bfs_spacing_and_coverage_random_networks():
    for seed in range(6):
        p = inputs.config_2d(48, 1.0, 4.0, 12, (10, 40), 1e2, 8, 6, seed=seed)
        g = geometry.build_geometry(p)
        lab, nets = coarsen.fracture_networks(g.strike_adj)
        for cells in nets:
            verts, prim, level = coarsen.bfs_coarsen(cells, g.strike_adj, 6)
            # every cell assigned, each vertex owns its block
            assert sorted(prim) == cells
            for k, v in enumerate(verts):
                assert prim[v] == k and level[v] == 0
            # Table 2 guarantees at least d_min cells between coarse nodes
            for v in verts:
                d = _bfs_dist(g.strike_adj, v)
                for w in verts:
                    if w != v:
                        assert d[w] >= 6
            # each primal block is connected
            for k in range(len(verts)):
                blk = {c for c in cells if prim[c] == k}
                d = _bfs_dist({c: [m for m in g.strike_adj[c] if m in blk] for c in blk},
                              verts[k])
                assert set(d) == blk


def test_axis_blocks_nodes():
    blk, node, nb = coarsen.axis_blocks(32, 4)
    assert nb == 8 and list(node) == [0, 6, 10, 14, 18, 22, 26, 31]
    blk, node, nb = coarsen.axis_blocks(10, 4)
    assert list(node) == [0, 6, 9]
    blk, node, nb = coarsen.axis_blocks(5, 8)
    assert list(node) == [2]


def _setup(p):
    g = geometry.build_geometry(p)
    s = assemble.assemble(p, g)
    c = coarsen.build_coarse(p, g)
    return g, s, c


def test_matrix_rank_counts_2d():
    p = inputs.config_2d(32, 1.0, 4.0, 0, (1, 2), 1.0, 4, 4, seed=1)
    g, s, c = _setup(p)
    rk = c.rank[: g.n_matrix]
    nodes = 8
    assert (rk == 3).sum() == nodes * nodes
    assert (rk == 2).sum() == 2 * nodes * (32 - nodes)
    assert (rk == 1).sum() == (32 - nodes) ** 2


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("dim", [2, 3, "3layers"])
def test_staged_equals_appendix_formulas(variant, dim):
    """dim "3layers": plates of random heights, some crossing with other
    layer ranges (separate networks that stay connected in A)."""
    if dim == 2:
        p = inputs.config_2d(24, 1.0, 4.0, 4, (6, 16), 1e3, 4, 4, seed=7, basis=variant)
    elif dim == 3:
        p = inputs.config_3d(12, 12, 8, 1.0, (4, 4, 2), 3, (4, 9), 1e3, (4, 4, 4), 4, 4,
                             seed=3, basis=variant)
        p.fracs[:, 4] = 0.0
        p.fracs[:, 5] = 8.0
    else:
        p = _layered_plates(variant)
    g, s, c = _setup(p)
    plate = np.concatenate([np.full(g.n_matrix, -1), g.cell_frac])
    P1 = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, variant, plate,
                                   c.row_net)
    P2 = basis.prolongation_appendix(s.A0, c.rank, c.medium, c.node_cell, variant, plate,
                                     c.row_net)
    assert abs(P1 - P2).max() < 1e-12
    assert np.abs(np.asarray(P1.sum(axis=1)).ravel() - 1).max() < 1e-12


def _layered_plates(variant):
    """16x16x10 box, five plates of random layer ranges; plates 0 and 1 cross
    with different ranges, plates 2 and 3 cross with the same range."""
    p = inputs.config_3d(16, 16, 10, 1.0, (4, 4, 2), 0, (4, 9), 1e3, (4, 4, 4), 4, 3, seed=6,
                         basis=variant)
    p.fracs = np.array([[1.5, 4.3, 14.5, 4.3, 0.0, 7.0], [6.3, 1.5, 6.3, 14.5, 3.0, 10.0],
                        [2.2, 9.7, 13.6, 12.9, 2.0, 8.0], [11.7, 7.1, 10.1, 15.2, 2.0, 8.0],
                        [3.1, 14.4, 7.9, 14.1, 5.0, 9.0]])
    p.kf = np.array([1e3, 1e4, 1e3, 1e2, 1e3])
    return p


def test_crossing_plates_of_other_layer_ranges_are_separate_networks():
    p = _layered_plates(0)
    g, s, c = _setup(p)
    crossings = {(fa, fb) for fa, fb, _, _ in g.intersections}
    assert (0, 1) in crossings and (2, 3) in crossings
    lab, nets = coarsen.fracture_networks(g.strike_adj)
    sf = g.strike_first
    net_of = [int(lab[sf[f]]) for f in range(len(p.fracs))]
    assert net_of[0] != net_of[1] and net_of[2] == net_of[3]
    # the crossing still couples the two plates in A (through the f-f links)
    ff = set(zip(g.cell_frac[g.ff_a], g.cell_frac[g.ff_b]))
    assert (0, 1) in ff
    # ... but no dual block of a fracture stage spans two networks (Coupled
    # blocks may still join two networks through matrix cells)
    plate = np.concatenate([np.full(g.n_matrix, -1), g.cell_frac])
    for variant in range(3):
        for cells in basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, variant, plate,
                                        c.row_net):
            assert len({int(c.row_net[r]) for r in cells if c.row_net[r] >= 0}) <= 1
    merged = basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, 0, plate, None)
    assert any(len({int(c.row_net[r]) for r in cells if c.row_net[r] >= 0}) > 1
               for cells in merged)


def _crossing_plates(variant):
    """Two full-height plates crossing at right angles in a 16x16x8 box."""
    p = inputs.config_3d(16, 16, 8, 1.0, (4, 4, 2), 0, (4, 9), 1e3, (4, 4, 4), 4, 4, seed=5,
                         basis=variant)
    p.fracs = np.array([[1.5, 8.3, 14.5, 8.3, 0.0, 8.0], [8.3, 1.5, 8.3, 14.5, 0.0, 8.0]])
    p.kf = np.array([1e3, 1e3])
    return p


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_fracture_faces_do_not_merge_across_a_crossing(variant):
    """Faces of two crossing plates meet only along the crossing: no dual
    block of the face stage holds face cells of both plates, the staged and
    Appendix A routes agree with the crossing links dropped, and the rows of
    P still sum to one."""
    p = _crossing_plates(variant)
    g, s, c = _setup(p)
    assert (g.ff_kind == 2).any()
    plate = np.concatenate([np.full(g.n_matrix, -1), g.cell_frac])
    P1 = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, variant, plate)
    P2 = basis.prolongation_appendix(s.A0, c.rank, c.medium, c.node_cell, variant, plate)
    assert abs(P1 - P2).max() < 1e-12
    assert np.abs(np.asarray(P1.sum(axis=1)).ravel() - 1).max() < 1e-12
    blocks = basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, variant, plate)
    faces = (c.medium == 1) & (c.rank == basis.RANK_F)
    for cells in blocks:
        owners = {int(plate[r]) for r in cells if faces[r]}
        assert len(owners) <= 1
    # without the rule the two plates' faces would share a block
    merged = basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, variant, None)
    assert any(len({int(plate[r]) for r in cells if faces[r]}) > 1 for cells in merged)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_basis_invariants(variant):
    p = inputs.config_2d(32, 1.5, 6.0, 6, (8, 20), 1e4, 4, 5, seed=9, basis=variant)
    g, s, c = _setup(p)
    P = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, variant)
    nm = g.n_matrix
    ncm = c.n_coarse_matrix
    # partition of unity (end of Sec. 3.1)
    assert np.abs(np.asarray(P.sum(axis=1)).ravel() - 1).max() < 1e-12
    # vertex rows are the Kronecker delta (Eq. 16)
    for j, v in enumerate(c.node_cell):
        row = P.getrow(v)
        assert row.nnz == 1 and row.indices[0] == j and row.data[0] == 1.0
    # local SPD M-matrix problems: 0 <= P <= 1
    assert P.data.min() > -1e-13 and P.data.max() < 1 + 1e-13
    Pd = P.toarray()
    Pmf, Pfm = Pd[:nm, ncm:], Pd[nm:, :ncm]
    if variant == 0:
        assert not Pmf.any() and not Pfm.any()
    if variant == 1:
        assert not Pfm.any() and Pmf.any()
    if variant == 2:
        assert not Pmf.any() and Pfm.any()
    if variant == 3:
        assert Pmf.any() and Pfm.any()
    # truncation keeps partition of unity and drops small entries (Sec. 4.3)
    Q = basis.truncate(P, 1e-2)
    assert np.abs(np.asarray(Q.sum(axis=1)).ravel() - 1).max() < 1e-12
    assert np.abs(Q.data).min() >= 1e-2 - 1e-15
    assert Q.nnz < P.nnz


def _hat(n, nodes, i, J):
    """1D piecewise-linear hat of node J evaluated at cell i."""
    x = nodes
    if i <= x[0]:
        return 1.0 if J == 0 else 0.0
    if i >= x[-1]:
        return 1.0 if J == len(x) - 1 else 0.0
    k = np.searchsorted(x, i, side="right") - 1
    w = (i - x[k]) / (x[k + 1] - x[k])
    if J == k:
        return 1 - w
    if J == k + 1:
        return w
    return 0.0


def test_homogeneous_basis_is_tensor_product_hat():
    """In a homogeneous fracture-free medium the local problems are discrete
    Laplace problems whose solutions are the bilinear (trilinear) interpolants
    between node lines, so P is the tensor product of 1D hats."""
    for dim, shape, C in ((2, (20, 13, 1), (4, 5, 1)), (3, (9, 10, 7), (4, 3, 3))):
        nx, ny, nz = shape
        p = inputs.Problem(dim=dim, nx=nx, ny=ny, nz=nz, perm=np.ones(nx * ny * nz),
                           fracs=np.zeros((0, 4 if dim == 2 else 6)), kf=np.zeros(0),
                           coarsen=C)
        g, s, c = _setup(p)
        P = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, 0).toarray()
        _, ndx, nbx = coarsen.axis_blocks(nx, C[0])
        _, ndy, nby = coarsen.axis_blocks(ny, C[1])
        _, ndz, nbz = coarsen.axis_blocks(nz, C[2] if dim == 3 else 1)
        want = np.zeros_like(P)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    for K in range(nbz):
                        for J in range(nby):
                            for I in range(nbx):
                                want[x + nx * (y + ny * z), I + nbx * (J + nby * K)] = (
                                    _hat(nx, ndx, x, I) * _hat(ny, ndy, y, J)
                                    * (_hat(nz, ndz, z, K) if dim == 3 else 1.0))
        np.testing.assert_allclose(P, want, rtol=0, atol=1e-13)


def test_truncation_example():
    P = sp.csr_matrix(np.array([[0.5, 0.495, 0.005], [0.004, 0.006, 0.99], [0.3, 0.3, 0.4]]))
    Q = basis.truncate(P, 1e-2).toarray()
    np.testing.assert_allclose(Q[0], [0.5 / 0.995, 0.495 / 0.995, 0.0])
    np.testing.assert_allclose(Q[1], [0.0, 0.0, 1.0])
    np.testing.assert_allclose(Q[2], [0.3, 0.3, 0.4])
    # a row whose every entry is below alpha keeps its largest one
    R = basis.truncate(sp.csr_matrix(np.array([[0.3, 0.3, 0.4]])), 0.5).toarray()
    np.testing.assert_allclose(R, [[0.0, 0.0, 1.0]])


def _plate_cases():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "coarse3d_plates.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, val = line.partition(" ")
        if key == "case":
            cur = {"name": val, "plates": [], "rank": [], "block": []}
        elif key == "end":
            cases.append(cur)
        elif key == "plate":
            cur["plates"].append([float(t) for t in val.split()])
        elif key in ("rank", "block"):
            cur[key].extend(int(t) for t in val.split())
        elif key in ("grid", "coarsen", "nodes"):
            cur[key] = [int(t) for t in val.split()]
        else:
            cur[key] = int(val)
    return cases


@pytest.mark.parametrize("case", _plate_cases(), ids=lambda c: c["name"])
def test_3d_plate_coarsening_golden(case):
    """Ranks, fracture coarse blocks and node cells of every plate cell
    against hand-worked cases (a wrong vertical node layer, an E/F swap or a
    misnumbered block turns this red)."""
    nx, ny, nz = case["grid"]
    pl = np.array(case["plates"])
    p = inputs.Problem(dim=3, nx=nx, ny=ny, nz=nz, perm=np.ones(nx * ny * nz), fracs=pl,
                       kf=np.full(len(pl), 1e3), coarsen=tuple(case["coarsen"]),
                       frac_dmin=case["dmin"], frac_cz=case["cz"])
    g = geometry.build_geometry(p)
    c = coarsen.build_coarse(p, g)
    nm = g.n_matrix
    assert g.n_frac == len(case["rank"])
    assert c.n_coarse == case["ncoarse"]
    assert list(c.rank[nm:]) == case["rank"]
    assert list(c.primal[nm:] - c.n_coarse_matrix) == case["block"]
    assert list(c.node_cell[c.n_coarse_matrix:] - nm) == case["nodes"]


def _piece_cases():
    out, cur = [], None
    for line in open(os.path.join(GOLDEN, "oblique_pieces.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, val = line.partition(" ")
        if key == "case":
            cur = {"name": val, "pieces": {}}
        elif key == "end":
            out.append(cur)
        elif key == "seg":
            cur["seg"] = [float(t) for t in val.split()]
        elif key == "piece":
            s, ix, iy, num, den = (int(t) for t in val.split())
            cur["pieces"].setdefault(s, []).append((ix, iy, num / den))
        else:
            cur[key] = [int(t) for t in val.split()]
    return out


@pytest.mark.parametrize("case", _piece_cases(), ids=lambda c: c["name"])
def test_oblique_pieces_golden(case):
    """Matrix cells and lengths of the pieces of oblique fracture cells (Eqs.
    4-6: A_ij is the overlap length times the depth) against hand-worked
    parameter crossings."""
    ax, ay, bx, by = case["seg"]
    n = case["n"][0]
    nx, ny = case["grid"]
    L = float(np.hypot(bx - ax, by - ay))
    for s in range(n):
        got = geometry.piece_overlaps(ax, ay, bx, by, n, s, 1.0, 1.0, nx, ny)
        want = case["pieces"][s]
        assert [(i, j) for i, j, _ in got] == [(i, j) for i, j, _ in want]
        np.testing.assert_allclose([ln for _, _, ln in got], [f * L for _, _, f in want],
                                   rtol=1e-14, atol=0)


def test_merge_capped_by_hand():
    """Eight cells: same-medium blocks {0,1,2} {3} {4,5} {6,7}; cross-medium
    links in order (2,3) (1,4) (3,6) (5,7).  Cap 4: (2,3) gives {0,1,2,3}
    (4 cells); (1,4) would give 6 > 4, cut; (3,6) would give 6, cut; (5,7)
    gives {4,5,6,7}.  Cap 6: (2,3) -> 4 cells, (1,4) -> 6, (3,6) -> 8 cut,
    (5,7) -> {4,5} is already in the 6-cell block, {6,7} would give 8, cut."""
    same = [(0, 1), (1, 2), (4, 5), (6, 7)]
    cross = [(2, 3), (1, 4), (3, 6), (5, 7)]
    assert basis.merge_capped(8, same, cross, 4) == [0, 0, 0, 0, 4, 4, 4, 4]
    assert basis.merge_capped(8, same, cross, 6) == [0, 0, 0, 0, 0, 0, 6, 6]
    assert basis.merge_capped(8, same, cross, 8) == [0] * 8
    # a same-medium block above the cap merges with nothing
    assert basis.merge_capped(8, same, cross, 2) == [0, 0, 0, 3, 4, 4, 6, 6]


def _coupled_3d(cap):
    p = _crossing_plates(3)
    p.merge_cap = cap
    return p


@pytest.mark.parametrize("cap", [0, 8, 16])
def test_coupled_merge_cap(cap):
    """Coupled-AMS with a merge cap: the staged and Appendix A routes agree
    (cut links removed from the diagonal), partition of unity holds, and no
    block is larger than the cap unless one medium alone makes it so; with
    cap 0, or a cap above every merged block, nothing is cut."""
    p = _coupled_3d(cap)
    g, s, c = _setup(p)
    plate = np.concatenate([np.full(g.n_matrix, -1), g.cell_frac])
    P1 = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, cap)
    P2 = basis.prolongation_appendix(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net,
                                     cap)
    assert abs(P1 - P2).max() < 1e-12
    assert np.abs(np.asarray(P1.sum(axis=1)).ravel() - 1).max() < 1e-12
    blocks = basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, cap)
    free = basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, 0)
    cut = basis.cut_links(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, cap)
    if cap == 0:
        assert not cut
    else:
        assert cut and all(c.medium[r] != c.medium[q] for r, q in cut)
        big = max(len(b) for b in free)
        assert big > cap
        for cells in blocks:
            if len(cells) > cap:   # then one medium's cells alone exceed the cap
                sub = basis.stage_blocks(s.A0, c.rank, c.medium, c.node_cell, 0, plate,
                                         c.row_net)
                assert any(len(set(b) & set(cells)) > cap for b in sub)
    big = max(len(b) for b in free)
    assert not basis.cut_links(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, big)
    P3 = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, big)
    P0 = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, 0)
    assert abs(P3 - P0).max() == 0.0
