"""Pins of the oracle's coarse system, ILU(0), Table 1 iteration and flux
reconstruction (Sec. 3.2)."""
import copy

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle import assemble, basis, coarsen, geometry, solver
from paper_1705_05784_gb300 import inputs


def _small(variant=0, restriction=1, **kw):
    p = inputs.config_2d(24, 1.0, 4.0, 4, (6, 16), 1e2, 4, 4, seed=7, basis=variant,
                         restriction=restriction, **kw)
    return p


def test_ilu0_reproduces_a_on_its_pattern():
    p = _small()
    s = assemble.assemble(p)
    F = solver.ilu0(s.A)
    L = sp.tril(F, -1) + sp.identity(s.n)
    U = sp.triu(F)
    LU = (L @ U).tocsr()
    A = s.A.tocoo()
    d = np.asarray(LU[A.row, A.col]).ravel() - A.data
    assert np.abs(d).max() < 1e-12 * np.abs(A.data).max()


def test_ilu0_is_exact_lu_without_fill():
    n = 30
    rng = np.random.default_rng(1)
    off = -rng.uniform(0.5, 2, n - 1)
    diag = rng.uniform(5, 6, n)
    A = sp.diags([off, diag, off], [-1, 0, 1], format="csr")
    F = solver.ilu0(A)
    b = rng.standard_normal(n)
    x = solver.ilu0_apply(F, b)
    np.testing.assert_allclose(A @ x, b, rtol=0, atol=1e-12)


@pytest.mark.parametrize("restriction", [0, 1])
def test_coarse_operator_properties(restriction):
    p = _small(variant=3, restriction=restriction)
    g = geometry.build_geometry(p)
    s = assemble.assemble(p, g)
    c = coarsen.build_coarse(p, g)
    P = basis.prolongation_staged(s.A0, c.rank, c.medium, c.node_cell, 3)
    R = solver.restriction(P, c.primal, c.n_coarse, restriction)
    # zero row sums of R A0 P: A0 1 = 0 and P 1 = 1
    Ac0 = (R @ s.A0 @ P).toarray()
    assert np.abs(Ac0.sum(axis=1)).max() < 1e-10 * np.abs(Ac0).max()
    Ac = (R @ s.A @ P).toarray()
    if restriction == 1:
        assert np.abs(Ac - Ac.T).max() < 1e-12 * np.abs(Ac).max()
        assert np.linalg.eigvalsh(0.5 * (Ac + Ac.T)).min() > 0
    # after the multiscale stage the restricted residual vanishes:
    # R (r - A P (R A P)^-1 R r) = 0
    st = solver.setup(s, P, c.primal, c.n_coarse, restriction)
    r = s.q - s.A @ np.zeros(s.n)
    import scipy.linalg as sla
    dp = P @ sla.lu_solve(st.lu, R @ r)
    r1 = r - s.A @ dp
    assert np.abs(R @ r1).max() < 1e-11 * np.abs(R @ r).max()


def test_coarsening_ratio_one_is_a_direct_solve():
    p = inputs.config_2d(12, 1.0, 3.0, 0, (1, 2), 1.0, 1, 1, seed=2)
    r = oracle.run(p)
    assert r.iters == 1 and r.rel_res < 1e-13


@pytest.mark.parametrize("restriction", [0, 1])
def test_homogeneous_one_multiscale_step_is_exact(restriction):
    """With node lines on the boundary cells the coarse space contains the
    linear pressure of a homogeneous fracture-free W/E problem."""
    nx, ny = 40, 24
    p = inputs.Problem(dim=2, nx=nx, ny=ny, nz=1, perm=np.ones(nx * ny),
                       fracs=np.zeros((0, 4)), kf=np.zeros(0), coarsen=(8, 8, 1),
                       restriction=restriction)
    g, sysm, c, P, st = oracle.build(p)
    x, it, rr, ok, _ = solver.two_stage_solve(st, max_iter=1, smoother=False)
    np.testing.assert_allclose(x, np.tile(1 - (np.arange(nx) + 0.5) / nx, ny), atol=1e-13)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_converged_iterate_matches_direct_solve(variant):
    p = _small(variant=variant)
    r = oracle.run(p)
    assert r.converged
    x = spla.spsolve(r.sysm.A.tocsc(), r.sysm.q)
    assert np.linalg.norm(r.p - x) / np.linalg.norm(x) < 1e-6
    # the iteration count is the number of completed Table 1 sweeps
    assert len(r.history) == r.iters + 1


def test_zero_fracture_decoupled_is_plain_ams():
    """Decoupled-AMS with no fractures reduces to AMS on the matrix alone:
    every variant gives the same P and iterate."""
    p = inputs.config_2d(24, 1.0, 4.0, 0, (1, 2), 1.0, 4, 4, seed=3)
    res = []
    for v in range(4):
        p.basis = v
        res.append(oracle.run(p))
    for r in res[1:]:
        assert abs(r.P - res[0].P).max() == 0.0
        assert r.iters == res[0].iters


@pytest.mark.parametrize("variant", [0, 3])
def test_flux_reconstruction_is_conservative(variant):
    p = _small(variant=variant, restriction=1)
    p.tol = 1e-3          # stop early: the reconstruction works after any iteration
    r = oracle.run(p)
    g, sysm, c, P, st = oracle.build(p)
    st_fv = oracle.reconstruction_setup(p, g, sysm, c)
    flux, dflux, pp, pt = solver.reconstruct_flux(sysm, p, st_fv, r.p, c.primal, c.node_cell)
    bal = solver.cell_balance(sysm, p, flux, dflux)
    scale = np.abs(flux).max()
    assert np.abs(bal).max() < 1e-12 * max(scale, 1.0)
    # the W/E problem: total inflow at the west face equals outflow at the east
    dc, dT, dp, fid = sysm.dirichlet
    assert abs(dflux[fid == 0].sum() + dflux[fid == 1].sum()) < 1e-10 * scale


def test_flux_of_exact_solution_is_two_point_flux():
    p = _small(variant=0, restriction=1)
    g, sysm, c, P, st = oracle.build(p)
    x = spla.spsolve(sysm.A.tocsc(), sysm.q)
    st_fv = solver.setup(sysm, P, c.primal, c.n_coarse, solver.R_FV)
    flux, dflux, pp, pt = solver.reconstruct_flux(sysm, p, st_fv, x, c.primal, c.node_cell)
    ci, cj, cT = solver.connections(sysm, p)
    np.testing.assert_allclose(flux, cT * (x[ci] - x[cj]), rtol=0,
                               atol=1e-9 * np.abs(flux).max())


# --- GMRES with the two-stage step as right preconditioner (Sec. 4.5, 4.6) ---

def _minres_over_krylov(st, x0, k):
    """Brute force: min ||q - A (x0 + M^-1 K c)|| over the k-dimensional Krylov
    space K = span{r0, (A M^-1) r0, ...} (the defining property of GMRES),
    from explicit power vectors and an SVD least-squares solve."""
    A, q = st.A, st.q
    r0 = q - A @ x0
    cols, v = [], r0 / np.linalg.norm(r0)
    for _ in range(k):
        cols.append(v)
        v = A @ solver.precondition(st, v)
        v = v / np.linalg.norm(v)
    Z = np.stack([solver.precondition(st, c) for c in cols], axis=1)
    AZ = A @ Z
    c, *_ = np.linalg.lstsq(AZ, r0, rcond=None)
    return np.linalg.norm(r0 - AZ @ c)


@pytest.mark.parametrize("variant", [0, 3])
def test_gmres_minimises_the_residual_over_the_krylov_space(variant):
    p = _small(variant=variant)
    g, sysm, c, P, st = oracle.build(p)
    x0 = np.random.default_rng(3).uniform(0, 1, sysm.n)
    qn = np.linalg.norm(sysm.q)
    for k in range(1, 6):
        x, it, rr, ok, hist = solver.gmres_solve(st, x0=x0, tol=0.0, max_iter=k, restart=30,
                                                 history=True)
        assert it == k and len(hist) == k + 1
        best = _minres_over_krylov(st, x0, k)
        assert abs(rr * qn - best) <= 1e-7 * best
        # the least-squares estimate inside the cycle is the true residual too
        assert abs(np.linalg.norm(sysm.q - sysm.A @ x) / qn - rr) <= 1e-12


def test_gmres_residuals_do_not_increase_within_a_cycle():
    p = _small(variant=1)
    g, sysm, c, P, st = oracle.build(p)
    x, it, rr, ok, hist = solver.gmres_solve(st, tol=1e-10, max_iter=25, restart=25, history=True)
    assert np.all(np.diff(hist) <= 1e-14)


def test_gmres_with_exact_preconditioner_takes_one_iteration():
    # coarsening ratio 1: P = I and the coarse solve is a direct solve of A
    p = inputs.config_2d(12, 1.0, 3.0, 0, (1, 2), 1.0, 1, 1, seed=2, krylov=1)
    r = oracle.run(p)
    assert r.iters == 1 and r.rel_res < 1e-13


def test_gmres_terminates_on_a_tiny_system():
    """Without restarts GMRES finds the solution in at most n steps."""
    p = inputs.config_2d(6, 1.0, 2.0, 1, (2, 4), 1e2, 3, 3, seed=5)
    g, sysm, c, P, st = oracle.build(p)
    n = sysm.n
    x, it, rr, ok, hist = solver.gmres_solve(st, tol=1e-11, max_iter=n, restart=n, history=True)
    assert ok and it <= n
    xd = spla.spsolve(sysm.A.tocsc(), sysm.q)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8


@pytest.mark.parametrize("restart", [5, 30])
def test_gmres_converges_to_the_direct_solution_with_restarts(restart):
    p = _small(variant=2, krylov=1, restart=restart)
    r = oracle.run(p)
    assert r.converged
    # every cycle ends on a true residual, so the history's last entry is one
    assert abs(np.linalg.norm(r.sysm.q - r.sysm.A @ r.p) / np.linalg.norm(r.sysm.q)
               - r.rel_res) < 1e-14
    x = spla.spsolve(r.sysm.A.tocsc(), r.sysm.q)
    assert np.linalg.norm(r.p - x) / np.linalg.norm(x) < 1e-6
    rich = oracle.run(_small(variant=2))
    assert r.iters < rich.iters


# --- time-step update: mobility scales on the transmissibilities, P reused ---

def test_mobility_update_pins():
    p = _small(variant=1)
    g, sysm, c, P, st = oracle.build(p)
    n = sysm.n
    # scale 1: the same system
    u1 = assemble.update_mobility(sysm, np.ones(n))
    assert abs(u1.A - sysm.A).max() <= 1e-12 * abs(sysm.A).max()
    # a uniform scale c: A and the Dirichlet terms scale by c, the solution is
    # unchanged (no sources)
    uc = assemble.update_mobility(sysm, np.full(n, 3.0))
    assert abs(uc.A - 3.0 * sysm.A).max() <= 1e-12 * abs(sysm.A).max()
    x0 = spla.spsolve(sysm.A.tocsc(), sysm.q)
    x3 = spla.spsolve(uc.A.tocsc(), uc.q)
    assert np.linalg.norm(x3 - x0) <= 1e-10 * np.linalg.norm(x0)
    # a random scale: symmetric, zero row sums of A0, and one connection by hand
    sc = np.random.default_rng(2).uniform(0.5, 2.0, n)
    ur = assemble.update_mobility(sysm, sc)
    assert abs(ur.A - ur.A.T).max() <= 1e-14 * abs(ur.A).max()
    assert np.abs(np.asarray(ur.A0.sum(axis=1)).ravel()).max() <= 1e-12 * abs(ur.A0).max()
    i, j = 5, 6                                   # x-neighbours in the first row
    hm = 2 * sc[i] * sc[j] / (sc[i] + sc[j])
    assert abs(ur.A[i, j] - sysm.A[i, j] * hm) <= 1e-14 * abs(sysm.A[i, j])
    # the updated system with the old P: converges to its own direct solution,
    # and its flux field stays conservative
    su = solver.setup(ur, P, c.primal, c.n_coarse, solver.R_FE)
    x, it, rr, ok, _ = solver.gmres_solve(su, tol=1e-10, max_iter=200)
    xd = spla.spsolve(ur.A.tocsc(), ur.q)
    assert ok and np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    sfv = solver.setup(ur, P, c.primal, c.n_coarse, solver.R_FV)
    flux, dflux, _, _ = solver.reconstruct_flux(ur, p, sfv, x, c.primal, c.node_cell)
    bal = solver.cell_balance(ur, p, flux, dflux)
    # each cell sums a few fluxes T (p_i - p_j) of up to max T |p| in size
    bound = 64 * np.finfo(float).eps * abs(ur.A).max() * np.abs(x).max()
    assert np.abs(bal).max() <= bound


# --- numerically singular coarse systems (reading: scaled pivot test) ---

def test_singular_step_pins():
    rng = np.random.default_rng(11)
    M = rng.standard_normal((7, 7)) + 7 * np.eye(7)
    assert solver.singular_step(M) == -1
    Z = M.copy()
    Z[:, 3] = 0.0                                   # zero column
    assert solver.singular_step(Z) >= 0
    R = M.copy()
    R[4] = -2.5 * R[1]                              # dependent rows
    assert solver.singular_step(R) >= 0
    # invariant under row scaling: entries over 16 decades stay regular
    D = np.diag(10.0 ** np.linspace(-8, 8, 7))
    assert solver.singular_step(D) == -1
    assert solver.singular_step(D @ M) == -1
    assert solver.singular_step(D @ R) >= 0
    # nearly dependent rows (1e-6 apart) are ill-conditioned, not singular
    N = M.copy()
    N[4] = N[1] * (1 + 1e-6 * rng.standard_normal(7))
    assert solver.singular_step(N) == -1
    assert solver.singular_step(np.zeros((0, 0))) == -1


def _block_bound_basis():
    """A 64 x 64 instance (sigma 2, Rock-AMS, alpha 1e-2) in which a truncated
    basis function lies inside its own primal block."""
    return inputs.config_2d(64, 2.0, 8.0, 4, (10, 30), 1e4, 8, 8, seed=86, basis=2,
                            restriction=1, alpha=1e-2)


def test_truncated_fv_system_singular_and_the_reconstruction():
    """Truncation can make R^FV A P singular: a basis function whose
    truncated support stays inside its own primal block, off the block's
    boundary, sends no flux out of any block (a zero column; 13 of the 304
    instances of the 256 x 256 workload), and here a numerically singular
    pivot appears.  The reconstruction's finite-volume stage uses the basis
    functions before truncation: regular, and the reconstructed field
    conserves mass in every cell to round-off (64 eps T_max |p|_max)."""
    p = _block_bound_basis()
    g, sysm, c, P, st = oracle.build(p)
    Afv = solver.coarse_operator(solver.restriction(P, c.primal, c.n_coarse, solver.R_FV),
                                 sysm.A, P)
    assert solver.singular_step(Afv) >= 0
    rs = oracle.reconstruction_setup(p, g, sysm, c)
    assert rs.P.nnz > P.nnz
    assert solver.singular_step(rs.Ac) == -1
    x = oracle.run(p).p
    flux, dflux, _, _ = solver.reconstruct_flux(sysm, p, rs, x, c.primal, c.node_cell)
    bal = solver.cell_balance(sysm, p, flux, dflux)
    _, _, cT = solver.connections(sysm, p)
    assert np.abs(bal).max() < 64 * np.finfo(float).eps * cT.max() * max(np.abs(x).max(), 1.0)


def test_a_basis_function_inside_its_block_gives_a_zero_fv_column():
    """The structural case by hand: on a homogeneous 24 x 24 grid with 8 x 8
    coarsening, replace column j of P by the unit vector of its node cell
    (a support inside the block, off its boundary): the column of R^FV A P
    is zero (A0 has zero row sums, so A's column summed over the block is
    the flux out of the block, zero); with the untruncated column it is not."""
    p = inputs.config_2d(24, 0.0, 4.0, 0, (1, 2), 1.0, 8, 8, seed=1, restriction=0)
    p.coarsen = (8, 8, 1)
    g, sysm, c, P, st = oracle.build(p)
    nodes = c.node_cell
    # the node cell of an interior-ish block: one not on the domain boundary
    nx = p.nx
    j = next(k for k, v in enumerate(nodes) if 0 < v % nx < nx - 1 and 0 < v // nx < p.ny - 1)
    Q = P.tolil()
    Q[:, j] = 0.0
    Q[nodes[j], j] = 1.0
    Q = sp.csr_matrix(Q)
    R = solver.restriction(Q, c.primal, c.n_coarse, solver.R_FV)
    A0c = solver.coarse_operator(R, sysm.A0, Q)
    assert np.abs(A0c[:, j]).max() == 0.0
    Ac = solver.coarse_operator(R, sysm.A0, P)
    assert np.abs(Ac[:, j]).max() > 0.0


def test_sealed_node_and_the_reconstruction():
    """A node cell 1e-10 times less permeable than its neighbours: truncation
    reduces its basis function to the node cell, whose R^FV column is then
    zero.  Before truncation its basis function is about 1e-10 outside the
    node cell: the reconstruction's system is regular and its field
    conservative.  Sealed to 1e-300, even that system is singular by the
    scaled pivot test."""
    p = inputs.config_2d_sealed_node(restriction=solver.R_FV)
    g, sysm, c, P, st = oracle.build(p)
    node = 22 + 32 * 6
    J = int(np.nonzero(c.node_cell == node)[0][0])
    col = P.tocsc()[:, J]
    assert col.nnz == 1 and col.indices[0] == node and col.data[0] == 1.0
    assert np.abs(st.Ac[:, J]).max() <= 1e-14 * np.abs(st.Ac).max()
    assert solver.singular_step(st.Ac) >= 0
    sfe = solver.setup(sysm, P, c.primal, c.n_coarse, solver.R_FE)
    assert solver.singular_step(sfe.Ac) == -1
    rs = oracle.reconstruction_setup(p, g, sysm, c)
    assert solver.singular_step(rs.Ac) == -1
    q = copy.copy(p)
    q.restriction = solver.R_FE
    x = oracle.run(q).p
    flux, dflux, _, _ = solver.reconstruct_flux(sysm, p, rs, x, c.primal, c.node_cell)
    bal = solver.cell_balance(sysm, p, flux, dflux)
    _, _, cT = solver.connections(sysm, p)
    assert np.abs(bal).max() < 64 * np.finfo(float).eps * cT.max() * max(np.abs(x).max(), 1.0)
    s300 = inputs.config_2d_sealed_node(restriction=solver.R_FV, factor=1e-300)
    g3, sys3, c3, _, _ = oracle.build(s300)
    assert solver.singular_step(oracle.reconstruction_setup(s300, g3, sys3, c3).Ac) >= 0


def test_basis_rebuilt_for_new_mobilities():
    """Rebuilding the basis from the updated operator: a uniform mobility
    scale leaves P unchanged (A0 scales, its local solutions do not); a
    non-uniform one changes it, keeps the partition of unity and the vertex
    rows, and (fracture-free, no truncation) the rebuilt P solves the updated
    operator's rows at the interior cells exactly: those rows keep all their
    links, so (A0' P) vanishes there."""
    p = _small(0, restriction=1)
    g, sysm, c, P, st = oracle.build(p)
    u = assemble.update_mobility(sysm, np.full(sysm.n, 3.0))
    Pu = oracle.prolongation(p, g, u, c)
    assert abs(Pu - P).max() < 1e-12
    sc = np.random.default_rng(5).uniform(0.25, 4.0, sysm.n)
    u = assemble.update_mobility(sysm, sc)
    Pu = oracle.prolongation(p, g, u, c)
    assert abs(Pu - P).max() > 1e-3
    assert np.abs(np.asarray(Pu.sum(axis=1)).ravel() - 1).max() < 1e-12
    for J, cell in enumerate(c.node_cell):
        row = Pu.getrow(cell)
        assert row.nnz == 1 and row.indices[0] == J and row.data[0] == 1.0
    q = inputs.config_2d(24, 1.0, 4.0, 0, (6, 16), 1e2, 4, 4, seed=7, basis=0, restriction=1)
    q.alpha = 0.0
    gq, sq, cq, Pq, _ = oracle.build(q)
    uq = assemble.update_mobility(sq, np.random.default_rng(6).uniform(0.5, 2.0, sq.n))
    Pr = oracle.prolongation(q, gq, uq, cq)
    interior = cq.rank == cq.rank.min()
    R = (uq.A0 @ Pr).toarray()[interior]
    assert np.abs(R).max() < 1e-12 * abs(uq.A0).max()
    assert abs(Pr - Pq).max() > 1e-3


def test_msmix_restriction():
    """MSMIX: matrix coarse rows of R A P are the R^FE ones, fracture coarse
    rows the R^FV ones; without fractures MSMIX is R^FE; the GMRES iteration
    with it reaches the direct solution."""
    p = _small(1, restriction=solver.R_MIX)
    g, sysm, c, P, st = oracle.build(p)
    fe = solver.setup(sysm, P, c.primal, c.n_coarse, solver.R_FE)
    fv = solver.setup(sysm, P, c.primal, c.n_coarse, solver.R_FV)
    ncm = c.n_coarse_matrix
    assert c.n_coarse > ncm
    np.testing.assert_array_equal(st.Ac[:ncm], fe.Ac[:ncm])
    np.testing.assert_array_equal(st.Ac[ncm:], fv.Ac[ncm:])
    x, it, rr, ok, _ = solver.gmres_solve(st, tol=1e-10, max_iter=200, restart=30)
    xd = spla.spsolve(sysm.A.tocsc(), sysm.q)
    assert ok and np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    q = inputs.config_2d(24, 1.0, 4.0, 0, (6, 16), 1e2, 4, 4, seed=7, basis=0,
                         restriction=solver.R_MIX)
    gq, sq, cq, Pq, stq = oracle.build(q)
    feq = solver.setup(sq, Pq, cq.primal, cq.n_coarse, solver.R_FE)
    assert abs(stq.R - feq.R).max() == 0.0


def test_sub_block_smoother_factors_are_the_media_blocks():
    """The stage's ILU(0) is that of A^mm and A^ff apart (each factored on its
    own, then placed in A's pattern), and zero on the cross-medium entries;
    without fractures it is ILU(0) of A itself."""
    p = _small(variant=0, restriction=1)
    p.subblock = 1
    g, sysm, c, P, st = oracle.build(p)
    nm = g.n_matrix
    A = sysm.A.tocsr()
    Fm = solver.ilu0(A[:nm, :nm]).toarray()
    Ff = solver.ilu0(A[nm:, nm:]).toarray()
    Fb = st.Fb.toarray()
    np.testing.assert_allclose(Fb[:nm, :nm], Fm, rtol=1e-14, atol=0)
    np.testing.assert_allclose(Fb[nm:, nm:], Ff, rtol=1e-14, atol=0)
    assert not Fb[:nm, nm:].any() and not Fb[nm:, :nm].any()
    q = inputs.config_2d(24, 1.0, 4.0, 0, (1, 2), 1.0, 4, 4, seed=3)
    q.subblock = 1
    _, _, _, _, sq = oracle.build(q)
    assert abs(sq.Fb - sq.F).max() == 0.0


@pytest.mark.parametrize("variant", [0, 3])
def test_sub_block_smoother_converges_to_the_direct_solution(variant):
    p = inputs.config_2d(32, 1.5, 6.0, 6, (8, 20), 1e6, 4, 5, seed=9, basis=variant,
                         restriction=1)
    p.subblock = 1
    p.tol, p.max_iter = 1e-10, 500
    r = oracle.run(p)
    g, sysm, c, P, st = oracle.build(p)
    xd = spla.spsolve(sysm.A.tocsc(), sysm.q)
    assert r.converged and np.linalg.norm(r.p - xd) < 1e-6 * np.linalg.norm(xd)


def _adaptive_case():
    p = _small(3, restriction=1)
    p.alpha = 0.0
    g, sysm, c, P, st = oracle.build(p)
    return p, g, sysm, c, P


def test_adaptive_update_extremes():
    """eps < 0 solves every dual block again: the full rebuild; eps = inf
    solves none: P unchanged."""
    p, g, sysm, c, P = _adaptive_case()
    sc = np.random.default_rng(8).uniform(0.5, 2.0, sysm.n)
    u = assemble.update_mobility(sysm, sc)
    ref = np.ones(sysm.n)
    Pa, Pf, ref2, solved = oracle.prolongation_update(p, g, u, c, P, ref, sc, -1.0)
    assert abs(Pa - oracle.prolongation(p, g, u, c)).max() < 1e-13
    assert solved == len(basis.stage_blocks(sysm.A0, c.rank, c.medium, c.node_cell, p.basis,
                                            np.concatenate([np.full(g.n_matrix, -1),
                                                            g.cell_frac]), c.row_net))
    Pn, _, ref3, solved = oracle.prolongation_update(p, g, u, c, P, ref, sc, np.inf)
    assert solved == 0 and abs(Pn - P).max() == 0.0 and (ref3 == 1.0).all()


def test_adaptive_update_solves_the_marked_blocks_and_their_downstream():
    """Scales moved by 10x in a 3x3 patch (eps 0.5): the recomputed rows are
    exactly the blocks holding a marked cell plus, stage by stage, the blocks
    that read a recomputed row (an independent closure over the dual-block
    graph); every other row is the old one; every recomputed row solves its
    local problem (Eq. 18 with the dropped links on the diagonal) against
    the final values of the rows it reads; partition of unity holds."""
    p, g, sysm, c, P = _adaptive_case()
    nx = p.nx
    sc = np.ones(sysm.n)
    patch = [x + nx * y for x in range(9, 12) for y in range(13, 16)]
    sc[patch] = 10.0
    u = assemble.update_mobility(sysm, sc)
    Pa, Pf, ref2, solved = oracle.prolongation_update(p, g, u, c, P, np.ones(sysm.n), sc, 0.5)
    plate = np.concatenate([np.full(g.n_matrix, -1), g.cell_frac])
    blocks = basis.stage_blocks(sysm.A0, c.rank, c.medium, c.node_cell, p.basis, plate,
                                c.row_net, 0, True)
    A0 = sysm.A0.tocsr()

    def keep(r, q):
        return basis.keep_link(p.basis, c.medium[r], c.rank[r], c.medium[q], c.rank[q],
                               basis._cross(plate, c.row_net, r, q))
    stage_of = {}
    for si, cells in blocks:
        for r in cells:
            stage_of[r] = si
    rec = np.zeros(sysm.n, bool)
    for si, cells in blocks:
        hit = any(r in patch for r in cells) or any(
            rec[q] and keep(r, q) and stage_of.get(q, -1) != si
            for r in cells for q in A0.indices[A0.indptr[r]:A0.indptr[r + 1]] if q != r)
        if hit:
            rec[cells] = True
    assert solved > 0 and (ref2 == np.where(rec, sc, 1.0)).all()
    Pd, Po = Pa.toarray(), P.toarray()
    np.testing.assert_array_equal(Pd[~rec], Po[~rec])
    assert abs(Pd[rec] - Po[rec]).max() > 1e-3
    # each recomputed row solves its local equation with the updated operator
    U = u.A0.tocsr()
    for r in np.nonzero(rec)[0]:
        acc = np.zeros(Pd.shape[1])
        d = 0.0
        for k in range(U.indptr[r], U.indptr[r + 1]):
            q = U.indices[k]
            a = U.data[k]
            if q == r:
                d += a
            elif keep(r, q):
                acc += a * Pd[q]
            else:
                d += a   # a dropped link leaves the diagonal: A0 row sums are zero
        np.testing.assert_allclose(d * Pd[r] + acc, 0.0, atol=1e-12 * abs(U).max())
    np.testing.assert_allclose(Pd.sum(axis=1), 1.0, atol=1e-12)
