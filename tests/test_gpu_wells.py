"""Peaceman wells on the device against the oracle (Sec. 2 well terms,
Sec. 3.1 well basis functions with P^ww = I): the fine system with its well
rows, the well coarse nodes, P, GMRES trajectories, the conservative fluxes
with the perforation fluxes, a time-step update, and the whole-GPU path."""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import assemble as oasm
from oracle import solver as osolver
from paper_1705_05784_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fams():
    from paper_1705_05784_gb300 import fams
    return fams


def _case(name, variant=0, restriction=1):
    if name == "2d":
        p = inputs.config_2d(24, 1.0, 4.0, 3, (6, 16), 1e3, 4, 4, seed=7, basis=variant,
                             restriction=restriction)
        g = oracle.geometry.build_geometry(p)
        cell = int(g.nnc_m[len(g.nnc_m) // 2])
        p.wells = [inputs.Well(cells=np.array([cell]), pi=np.array([2.0]),
                               control=inputs.WELL_RATE, value=5.0),
                   inputs.column_well(24, 24, 1, 20, 3, 1.5, inputs.WELL_PRESSURE, 0.25),
                   inputs.Well(cells=np.array([3 + 24 * 17, 4 + 24 * 17]), pi=np.array([1.0, 0.5]),
                               control=inputs.WELL_RATE, value=-2.0)]
    else:
        # 3D: two full-height plates; an injector column through 6 of 8
        # layers and a producer column held at a pressure
        p = inputs.config_3d(16, 16, 8, 1.0, (4, 4, 2), 0, (4, 9), 1e3, (4, 4, 4), 4, 4, seed=5,
                             basis=variant, restriction=restriction)
        p.fracs = np.array([[1.5, 8.3, 14.5, 8.3, 0.0, 8.0], [8.3, 1.5, 8.3, 14.5, 0.0, 8.0]])
        p.kf = np.array([1e3, 1e3])
        p.wells = [inputs.column_well(16, 16, 8, 4, 11, 1.0, inputs.WELL_RATE, 3.0, 1, 7),
                   inputs.column_well(16, 16, 8, 12, 4, 2.0, inputs.WELL_PRESSURE, 0.0)]
    return p


def _gmres(p, restart, max_iter):
    q = copy.copy(p)
    q.krylov, q.restart, q.max_iter = 1, restart, max_iter
    return q


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_fine_system_and_coarse_grids_with_wells(name):
    fams = _fams()
    p = _case(name)
    g, sysm, c, P, st = oracle.build(p)
    with fams.Context(p) as ctx:
        S = ctx.sizes()
        assert S["n"] == sysm.n and S["n_well"] == sysm.n_well
        assert S["n_perf"] == sum(len(w.cells) for w in p.wells)
        np.testing.assert_array_equal(ctx.query("A_ROWPTR"), sysm.A.indptr)
        np.testing.assert_array_equal(ctx.query("A_COL"), sysm.A.indices)
        np.testing.assert_allclose(ctx.query("A_VAL"), sysm.A.data, rtol=1e-13,
                                   atol=1e-15 * abs(sysm.A).max())
        np.testing.assert_allclose(ctx.query("Q"), sysm.q, rtol=1e-13, atol=1e-15)
        np.testing.assert_array_equal(ctx.query("RANK"), c.rank)
        np.testing.assert_array_equal(ctx.query("PRIMAL"), c.primal)
        np.testing.assert_array_equal(ctx.query("NODE_CELL"), c.node_cell)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["2d", "3d"])
def test_prolongation_with_wells(name, variant):
    fams = _fams()
    p = _case(name, variant)
    g, sysm, c, P, st = oracle.build(p)
    with fams.Context(p) as ctx:
        Pg = sp.csr_matrix((ctx.query("P_VAL"), ctx.query("P_COL"), ctx.query("P_ROWPTR")),
                           shape=P.shape)
        np.testing.assert_array_equal(Pg.indptr, P.indptr)
        np.testing.assert_array_equal(Pg.indices, P.indices)
        np.testing.assert_allclose(Pg.data, P.data, rtol=0, atol=1e-12)


@pytest.mark.parametrize("restriction", [0, 1, 2])
@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("name", ["2d", "3d"])
def test_gmres_trajectory_with_wells(name, variant, restriction):
    """13 GMRES(8) iterations (a restart inside) against the oracle, 1e-10."""
    fams = _fams()
    p = _gmres(_case(name, variant, restriction), 8, 13)
    g, sysm, c, P, st = oracle.build(p)
    xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=13, restart=8)
    with fams.Context(p) as ctx:
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 13 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("name", ["2d", "3d"])
def test_fluxes_with_wells(name, variant):
    """The reconstruction from the same iterate equals the oracle's: face
    fluxes, fracture connections, rate-well perforations, pressure-well
    perforations (positive into the well); every cell and every rate well
    balances, and the injectors' perforations carry their rates."""
    fams = _fams()
    p = _gmres(_case(name, variant, 1), 30, 200)
    g, sysm, c, P, st = oracle.build(p)
    with fams.Context(p) as ctx:
        xs, stats = ctx.solve(tol=1e-9)
        assert stats[0]["converged"]
        face, nnc = ctx.flux(xs[0])
    rs = oracle.reconstruction_setup(p, g, sysm, c)
    flux, dflux, pp, pt = osolver.reconstruct_flux(sysm, p, rs, xs[0], c.primal, c.node_cell)
    nx, ny = p.nx, p.ny
    nz = p.nz if p.dim == 3 else 1
    nfx, nfy = (nx + 1) * ny * nz, nx * (ny + 1) * nz
    parts = [face[:nfx].reshape(nz, ny, nx + 1)[:, :, 1:-1].ravel(),
             face[nfx:nfx + nfy].reshape(nz, ny + 1, nx)[:, 1:-1, :].ravel()]
    if p.dim == 3:
        parts.append(face[nfx + nfy:].reshape(nz + 1, ny, nx)[1:-1].ravel())
    nconn = len(flux) - sum(len(p_) for p_ in parts)
    conn = np.concatenate(parts + [nnc[:nconn]])
    scale = np.abs(flux).max()
    np.testing.assert_allclose(conn, flux, rtol=0, atol=1e-8 * scale)
    dc, dT, dp, fid = sysm.dirichlet
    wp = fid >= 6
    np.testing.assert_allclose(nnc[nconn:], dflux[wp], rtol=0, atol=1e-8 * scale)
    # balances: every unknown (cells and rate wells) from the device fluxes
    ci, cj, cT = osolver.connections(sysm, p)
    out = np.zeros(sysm.n)
    np.add.at(out, ci, conn)
    np.subtract.at(out, cj, conn)
    fx = face[:nfx].reshape(nz, ny, nx + 1)
    xm = np.arange(g.n_matrix) % nx
    out[np.nonzero(xm == 0)[0]] -= fx[:, :, 0].ravel()
    out[np.nonzero(xm == nx - 1)[0]] += fx[:, :, -1].ravel()
    np.add.at(out, dc[wp], nnc[nconn:])
    src = sysm.q - sysm.q_dirichlet
    bound = 64 * np.finfo(float).eps * cT.max() * max(np.abs(pt).max(), 1.0)
    assert np.abs(out - src).max() < bound


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_time_step_update_with_wells(name):
    """fams_update with mobility scales of the matrix and fracture cells (the
    wells keep theirs): A and a GMRES trajectory against the oracle's update."""
    fams = _fams()
    p = _gmres(_case(name, 1, 1), 8, 13)
    g, sysm, c, P, st0 = oracle.build(p)
    nmf = g.n_matrix + g.n_frac
    sc = np.random.default_rng(4).uniform(0.3, 3.0, nmf)
    ur = oasm.update_mobility(sysm, np.concatenate([sc, np.ones(sysm.n_well)]))
    su = osolver.setup(ur, P, c.primal, c.n_coarse, p.restriction)
    with fams.Context(p) as ctx:
        ctx.update(sc)
        np.testing.assert_allclose(ctx.query("A_VAL"), ur.A.data, rtol=1e-13,
                                   atol=1e-15 * abs(ur.A).max())
        xo, ito, _, _, _ = osolver.gmres_solve(su, tol=0.0, max_iter=13, restart=8)
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 13 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_whole_gpu_solve_with_wells(name):
    fams = _fams()
    p = _gmres(_case(name, 3, 1), 10, 17)
    p.grid_solve = 1
    g, sysm, c, P, st = oracle.build(p)
    xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=17, restart=10)
    with fams.Context(p) as ctx:
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 17 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
