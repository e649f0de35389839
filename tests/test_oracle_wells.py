"""Pins of the oracle's Peaceman wells (Sec. 2: q^mw = PI lambda^m (p^w - p^m),
Sec. 3.1: each well one coarse node with P^ww = I and a locally computed
well basis function, Eq. 18's beta term in every coupling strategy)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle import assemble, basis, solver
from paper_1705_05784_gb300 import inputs


def _line(n, wells, bc_mask=inputs.BC_EAST):
    return inputs.Problem(dim=2, nx=n, ny=1, nz=1, perm=np.ones(n), fracs=np.zeros((0, 4)),
                          kf=np.zeros(0), bc_mask=bc_mask, bc_value=(1.0, 0.0, 0, 0, 0, 0),
                          coarsen=(4, 1, 1), frac_dmin=5, basis=0, restriction=1, wells=wells)


def test_rate_well_closed_form_on_a_line():
    """Ten unit cells (k = 1, face T = 1), east face at p = 0 (half-cell
    T_D = 2), an injector of rate Q = 2 perforating cell 0 with PI 3 (beta =
    3): the rate Q crosses every face, so p_9 = Q / T_D = 1, p_i = p_{i+1} +
    Q, and the well pressure is p_0 + Q / beta."""
    n, Q = 10, 2.0
    w = inputs.Well(cells=np.array([0]), pi=np.array([3.0]), control=inputs.WELL_RATE, value=Q)
    s = assemble.assemble(_line(n, [w]))
    assert s.n == n + 1 and s.n_well == 1
    x = spla.spsolve(s.A.tocsc(), s.q)
    want = 1.0 + Q * (n - 1 - np.arange(n))
    np.testing.assert_allclose(x[:n], want, rtol=1e-13)
    np.testing.assert_allclose(x[n], want[0] + Q / 3.0, rtol=1e-13)
    assert abs(s.A - s.A.T).max() == 0.0
    assert np.abs(np.asarray(s.A0.sum(axis=1)).ravel()).max() < 1e-14


def test_pressure_well_closed_form_on_a_line():
    """The same line with a pressure-controlled well at cell 0 (p_bhp = 1,
    beta = 3) and p = 0 on the east face: resistances 1/beta + 9/T + 1/T_D in
    series carry Q = 1 / (1/3 + 9 + 1/2); no well unknown."""
    n = 10
    w = inputs.Well(cells=np.array([0]), pi=np.array([3.0]), control=inputs.WELL_PRESSURE,
                    value=1.0)
    s = assemble.assemble(_line(n, [w]))
    assert s.n == n and s.n_well == 0
    x = spla.spsolve(s.A.tocsc(), s.q)
    Q = 1.0 / (1.0 / 3.0 + 9.0 + 0.5)
    np.testing.assert_allclose(x, 1.0 - Q / 3.0 - Q * np.arange(n), rtol=1e-13)


def _wells_case(variant, restriction=1):
    """24 x 24, six fractures, an injector (rate) through a cell next to a
    fracture and a producer held at a pressure; W/E Dirichlet faces too."""
    p = inputs.config_2d(24, 1.0, 4.0, 3, (6, 16), 1e3, 4, 4, seed=7, basis=variant,
                         restriction=restriction)
    g = oracle.geometry.build_geometry(p)
    cell = int(g.nnc_m[len(g.nnc_m) // 2])        # a matrix cell a fracture crosses
    p.wells = [inputs.Well(cells=np.array([cell]), pi=np.array([2.0]), control=inputs.WELL_RATE,
                           value=5.0),
               inputs.column_well(24, 24, 1, 20, 3, 1.5, inputs.WELL_PRESSURE, 0.25)]
    return p, cell


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_well_basis_functions(variant):
    """P^ww = I (the well row is the unit row of its coarse node), the rows of
    P sum to one, 0 <= P <= 1, the well column is nonzero at the perforated
    cell, and it reaches into the fractures only for Rock-AMS and Coupled-AMS
    (Sec. 3.1: fracture rows keep their matrix links only there)."""
    p, cell = _wells_case(variant)
    g, sysm, c, P, st = oracle.build(p)
    nm, nf = g.n_matrix, g.n_frac
    wrow = nm + nf
    jw = int(np.nonzero(c.node_cell == wrow)[0][0])
    assert jw == c.n_coarse - 1
    Pd = P.toarray()
    np.testing.assert_array_equal(Pd[wrow], np.eye(c.n_coarse)[jw])
    np.testing.assert_allclose(Pd.sum(axis=1), 1.0, atol=1e-12)
    assert Pd.min() > -1e-12 and Pd.max() < 1 + 1e-12
    col = Pd[:, jw]
    assert col[cell] > 0
    reaches_frac = np.abs(col[nm:nm + nf]).max() > 0
    assert reaches_frac == (variant in (2, 3))


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("restriction", [0, 1])
def test_wells_converge_and_conserve(variant, restriction):
    """GMRES with the two-stage preconditioner reaches the direct solution;
    the reconstructed flux field is conservative in every cell and the
    perforation fluxes of the injector add up to its rate."""
    p, cell = _wells_case(variant, restriction)
    p.krylov, p.restart, p.max_iter, p.tol = 1, 30, 300, 1e-10
    r = oracle.run(p)
    g, sysm, c, P, st = oracle.build(p)
    xd = spla.spsolve(sysm.A.tocsc(), sysm.q)
    assert r.converged and np.linalg.norm(r.p - xd) < 1e-6 * np.linalg.norm(xd)
    rs = oracle.reconstruction_setup(p, g, sysm, c)
    flux, dflux, _, _ = solver.reconstruct_flux(sysm, p, rs, r.p, c.primal, c.node_cell)
    bal = solver.cell_balance(sysm, p, flux, dflux)
    _, _, cT = solver.connections(sysm, p)
    assert np.abs(bal).max() < 64 * np.finfo(float).eps * cT.max() * np.abs(r.p).max()
    ci, cj, _ = solver.connections(sysm, p)
    wrow = g.n_matrix + g.n_frac
    into_well = flux[cj == wrow].sum()           # positive from the cell to the well
    np.testing.assert_allclose(-into_well, 5.0, rtol=1e-10)
