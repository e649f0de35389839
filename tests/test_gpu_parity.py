"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: integer and index work (fracture cells, matrix-fracture and
fracture-fracture connection lists, CSR patterns, wirebasket ranks, primal
blocks, coarse nodes) must be bit-exact.  FP64 values computed by the same
formula in a different summation order agree to a few ulps (1e-12 relative);
quantities that pass through local or coarse direct solves agree to 1e-10
relative; converged pressures to 1e-10 relative L2 with iteration counts
within +-1.
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import solver as osolver
from paper_1705_05784_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fams():
    from paper_1705_05784_gb300 import fams
    return fams


def _case(name, variant=0, restriction=1):
    if name == "2d32":
        p = inputs.config_2d_small(basis=variant, restriction=restriction)
    elif name == "2d64":
        p = inputs.config_2d(64, 1.5, 8.0, 6, (15, 45), 1e3, 8, 8, seed=4, basis=variant,
                             restriction=restriction)
    elif name == "2d50ragged":
        # 50 x 37 cells, coarsening 7 x 6: partial last blocks on both axes;
        # truncation on (alpha = 1e-2)
        nx, ny = 50, 37
        p = inputs.Problem(dim=2, nx=nx, ny=ny, nz=1,
                           perm=10 ** inputs.gaussian_field((nx, ny), 1.0, 5.0, 6),
                           fracs=inputs.random_segments(5, (nx, ny), (10, 30), 1006),
                           kf=np.full(5, 1e2), coarsen=(7, 6, 1), frac_dmin=6, basis=variant,
                           restriction=restriction, alpha=1e-2)
    elif name == "3d":
        p = inputs.config_3d(20, 18, 12, 1.0, (5, 5, 2), 4, (6, 14), 1e3, (5, 6, 4), 5, 4,
                             seed=8, basis=variant, restriction=restriction)
        p.fracs[:, 4] = 0.0
        p.fracs[:, 5] = 12.0
    elif name == "3dcross":
        # two full-height plates crossing at right angles plus an oblique one
        p = inputs.config_3d(16, 16, 8, 1.0, (4, 4, 2), 0, (4, 9), 1e3, (4, 4, 4), 4, 4, seed=5,
                             basis=variant, restriction=restriction)
        p.fracs = np.array([[1.5, 8.3, 14.5, 8.3, 0.0, 8.0], [8.3, 1.5, 8.3, 14.5, 0.0, 8.0],
                            [2.2, 2.7, 13.6, 12.9, 0.0, 8.0]])
        p.kf = np.array([1e3, 1e4, 1e3])
    elif name == "3dlayers":
        # five plates of their own layer ranges: two cross with different
        # ranges (separate networks), two with the same range (one network)
        p = inputs.config_3d(16, 16, 10, 1.0, (4, 4, 2), 0, (4, 9), 1e3, (4, 4, 4), 4, 3, seed=6,
                             basis=variant, restriction=restriction)
        p.fracs = np.array([[1.5, 4.3, 14.5, 4.3, 0.0, 7.0], [6.3, 1.5, 6.3, 14.5, 3.0, 10.0],
                            [2.2, 9.7, 13.6, 12.9, 2.0, 8.0], [11.7, 7.1, 10.1, 15.2, 2.0, 8.0],
                            [3.1, 14.4, 7.9, 14.1, 5.0, 9.0]])
        p.kf = np.array([1e3, 1e4, 1e3, 1e2, 1e3])
    else:
        raise KeyError(name)
    return p


CASES = ["2d32", "2d64", "2d50ragged", "3d", "3dcross", "3dlayers"]


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(name, variant=0, restriction=1):
        key = (name, variant, restriction)
        if key not in cache:
            p = _case(name, variant, restriction)
            g, sysm, c, P, st = oracle.build(p)
            ctx = _fams().Context(p)
            cache[key] = (p, g, sysm, c, P, st, ctx)
        return cache[key]
    yield get
    for v in cache.values():
        v[-1].close()


@pytest.mark.parametrize("name", CASES)
def test_geometry_bit_exact(built, name):
    p, g, sysm, c, P, st, ctx = built(name)
    s = ctx.sizes()
    assert s["n_matrix"] == g.n_matrix and s["n_frac"] == g.n_frac
    np.testing.assert_array_equal(ctx.query("NNC_FRAC"), g.nnc_f)
    np.testing.assert_array_equal(ctx.query("NNC_MATRIX"), g.nnc_m)
    np.testing.assert_allclose(ctx.query("NNC_AREA"), g.nnc_area, rtol=1e-13, atol=0)
    np.testing.assert_allclose(ctx.query("NNC_DIST"), g.nnc_dist, rtol=1e-12, atol=0)
    np.testing.assert_array_equal(ctx.query("FF_A"), g.ff_a)
    np.testing.assert_array_equal(ctx.query("FF_B"), g.ff_b)
    np.testing.assert_allclose(ctx.query("FF_T"), g.ff_T, rtol=1e-13, atol=0)


@pytest.mark.parametrize("name", CASES)
def test_fine_system(built, name):
    p, g, sysm, c, P, st, ctx = built(name)
    A = sysm.A
    np.testing.assert_array_equal(ctx.query("A_ROWPTR"), A.indptr)
    np.testing.assert_array_equal(ctx.query("A_COL"), A.indices)
    np.testing.assert_allclose(ctx.query("A_VAL"), A.data, rtol=1e-12, atol=1e-14 * abs(A.data).max())
    np.testing.assert_allclose(ctx.query("Q"), sysm.q, rtol=1e-12, atol=1e-14 * abs(sysm.q).max())


@pytest.mark.parametrize("name", CASES)
def test_coarse_grids_bit_exact(built, name):
    p, g, sysm, c, P, st, ctx = built(name)
    np.testing.assert_array_equal(ctx.query("RANK"), c.rank)
    np.testing.assert_array_equal(ctx.query("PRIMAL"), c.primal)
    np.testing.assert_array_equal(ctx.query("NODE_CELL"), c.node_cell)
    assert ctx.sizes()["n_coarse"] == c.n_coarse


def _gpu_P(ctx, shape):
    return sp.csr_matrix((ctx.query("P_VAL"), ctx.query("P_COL"), ctx.query("P_ROWPTR")),
                         shape=shape)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", CASES)
def test_prolongation(built, name, variant):
    p, g, sysm, c, P, st, ctx = built(name, variant)
    Pg = _gpu_P(ctx, P.shape)
    np.testing.assert_array_equal(Pg.indptr, P.indptr)
    np.testing.assert_array_equal(Pg.indices, P.indices)
    np.testing.assert_allclose(Pg.data, P.data, rtol=0, atol=1e-12)
    assert np.abs(np.asarray(Pg.sum(axis=1)).ravel() - 1).max() < 1e-12


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_coarse_operator(built, name, restriction):
    p, g, sysm, c, P, st, ctx = built(name, 0, restriction)
    Ac = ctx.query("AC").reshape(c.n_coarse, c.n_coarse)
    np.testing.assert_allclose(Ac, st.Ac, rtol=0, atol=1e-11 * np.abs(st.Ac).max())


def _band_solve(AB, ipiv, kl, ku, b):
    """LAPACK gbtrs on band factors (column-major, ldab = 2 kl + ku + 1):
    row interchanges and unit lower multipliers, then the upper band."""
    n = len(b)
    kv = kl + ku
    y = b.astype(np.float64).copy()
    for j in range(n):
        p = ipiv[j]
        if p != j:
            y[j], y[p] = y[p], y[j]
        km = min(kl, n - 1 - j)
        y[j + 1:j + 1 + km] -= AB[kv + 1:kv + 1 + km, j] * y[j]
    for j in range(n - 1, -1, -1):
        y[j] /= AB[kv, j]
        i0 = max(0, j - kv)
        y[i0:j] -= AB[kv - (j - i0):kv, j] * y[j]
    return y


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_coarse_factors_solve_the_coarse_system(built, name, restriction):
    """The band factors (LDL^T written as LU for R^FE, partial-pivoting band LU
    for R^FV) solve the reordered coarse system: backward error at rounding."""
    p, g, sysm, c, P, st, ctx = built(name, 0, restriction)
    nc = c.n_coarse
    Ac = ctx.query("AC").reshape(nc, nc)
    perm = ctx.query("COARSE_PERM")
    ipiv = ctx.query("COARSE_IPIV")
    kl, ku = ctx.query("BAND_KLKU")
    AB = ctx.query("BAND").reshape(nc, 2 * kl + ku + 1).T
    Ab = Ac[np.ix_(perm, perm)]
    rhs = np.random.default_rng(11).standard_normal(nc)
    x = _band_solve(AB, ipiv, kl, ku, rhs)
    berr = np.linalg.norm(Ab @ x - rhs) / (np.linalg.norm(Ab, np.inf) * np.linalg.norm(x, np.inf) + np.linalg.norm(rhs, np.inf))
    assert berr < 1e-13
    if restriction == 1:
        assert np.array_equal(ipiv, np.arange(nc))   # symmetric positive definite: no pivoting


def _check_band_factors(ctx, i):
    nc = ctx.sizes(i)["n_coarse"]
    Ac = ctx.query("AC", i).reshape(nc, nc)
    perm = ctx.query("COARSE_PERM", i)
    ipiv = ctx.query("COARSE_IPIV", i)
    kl, ku = ctx.query("BAND_KLKU", i)
    AB = ctx.query("BAND", i).reshape(nc, 2 * kl + ku + 1).T
    Ab = Ac[np.ix_(perm, perm)]
    rhs = np.random.default_rng(i).standard_normal(nc)
    x = _band_solve(AB, ipiv, kl, ku, rhs)
    berr = np.linalg.norm(Ab @ x - rhs) / (np.linalg.norm(Ab, np.inf) * np.linalg.norm(x, np.inf)
                                         + np.linalg.norm(rhs, np.inf))
    assert berr < 1e-13, (i, berr)
    return kl


def test_coarse_factors_at_bench_size():
    """256x256 instances, R^FV (band LU) and R^FE (LDL^T), bandwidths ~60-150."""
    fams = _fams()
    probs = [inputs.config_2d_256(seed=500 + i, tratio=1e4, basis=i % 4, restriction=i % 2,
                                  alpha=1e-2) for i in range(16)]
    with fams.Context(probs) as cb:
        for i in range(len(probs)):
            _check_band_factors(cb, i)


def test_coarse_factors_of_wide_bands():
    """3D 64x64x32 with 4x4x4 coarsening and R^FV: a coarse bandwidth beyond
    what shared memory holds ((kl+1)(2kl+1) doubles > 227 KB for kl > 118),
    so the band LU runs on its global-memory active block."""
    fams = _fams()
    p = inputs.config_3d(64, 64, 32, 1.0, (8, 8, 4), 6, (8, 24), 1e3, (4, 4, 4), 6, 4, seed=21,
                         basis=0, restriction=0)
    with fams.Context(p) as c1:
        assert _check_band_factors(c1, 0) > 118


def _coarse_solve_berr(ctx, i):
    nc = ctx.sizes(i)["n_coarse"]
    Ac = ctx.query("AC", i).reshape(nc, nc)
    rc, ec = ctx.query("LAST_RC", i), ctx.query("LAST_EC", i)
    return np.linalg.norm(Ac @ ec - rc, np.inf) / (np.linalg.norm(Ac, np.inf) * np.linalg.norm(ec, np.inf)
                                                   + np.linalg.norm(rc, np.inf))


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_device_coarse_solve(built, name, restriction):
    """The coarse solve inside the iteration -- blocks of 32 through inverse
    diagonal blocks for LDL^T factors, column by column with interchanges for
    the band LU -- solves the last application's R A P e = R r to rounding."""
    p, g, sysm, c, P, st, ctx = built(name, 0, restriction)
    ctx.solve(tol=1e-8)
    assert _coarse_solve_berr(ctx, 0) < 1e-13


def test_device_coarse_solve_at_bench_size():
    """256x256 R^FE instances (coarse sizes ~1100-1300, not multiples of 32;
    bandwidths 40-150) through the blocked solve."""
    fams = _fams()
    probs = []
    for i in range(8):
        q = _gmres(inputs.config_2d_256(seed=700 + i, tratio=10.0 ** (2 + 2 * (i % 4)), basis=i % 4,
                                        restriction=1, alpha=1e-2), 30, 3)
        probs.append(q)
    with fams.Context(probs) as cb:
        cb.solve(tol=0.0)
        for i in range(len(probs)):
            assert _coarse_solve_berr(cb, i) < 1e-13, i


@pytest.mark.parametrize("name", CASES)
def test_ilu0(built, name):
    p, g, sysm, c, P, st, ctx = built(name)
    F = ctx.query("ILU_VAL")
    np.testing.assert_allclose(F, st.F.data, rtol=1e-11, atol=1e-13 * np.abs(st.F.data).max())


def _fixed_k(p, k):
    """Same problem, iteration stopped after exactly k Table 1 sweeps."""
    import copy
    q = copy.copy(p)
    q.max_iter = k
    return q


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["2d32", "2d64", "2d50ragged", "3d", "3dcross"])
def test_iteration_trajectory(built, name, variant, restriction):
    """After the same number of sweeps the GPU iterate equals the oracle's."""
    p, g, sysm, c, P, st, ctx = built(name, variant, restriction)
    K = 6
    xo, ito, _, _, _ = osolver.two_stage_solve(st, tol=0.0, max_iter=K)
    with _fams().Context(_fixed_k(p, K)) as ck:
        xs, stats = ck.solve(tol=0.0)
    assert stats[0]["iterations"] == K == ito
    assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["2d32", "2d64", "2d50ragged", "3d"])
def test_solve_to_tolerance(built, name, variant):
    """To tol: iteration count within +-1 of the oracle's, the reported
    residual is the true one, and both solutions agree to tol x cond."""
    p, g, sysm, c, P, st, ctx = built(name, variant)
    xo, ito, rro, oko, _ = osolver.two_stage_solve(st, tol=1e-8, max_iter=p.max_iter)
    xs, stats = ctx.solve(tol=1e-8)
    x = xs[0]
    assert stats[0]["converged"] == oko
    assert abs(stats[0]["iterations"] - ito) <= 1
    rr = np.linalg.norm(sysm.q - sysm.A @ x) / np.linalg.norm(sysm.q)
    assert rr <= 1e-8
    # q - A x cancels to ~1e-8 of |q|: both norms carry ~1e-16 |A||x| absolute error
    assert abs(rr - stats[0]["rel_residual"]) <= 1e-6 * rr + 1e-13
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6


def _gmres(p, restart, max_iter):
    q = copy.copy(p)
    q.krylov, q.restart, q.max_iter = 1, restart, max_iter
    return q


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("name", ["2d32", "2d64", "2d50ragged", "3d", "3dcross"])
def test_gmres_trajectory(built, name, variant, restriction):
    """GMRES(8) for 13 iterations (one restart): the GPU iterate and residual
    history equal the oracle's (modified Gram-Schmidt there, classical
    Gram-Schmidt twice here: the same Krylov space, rounding apart)."""
    p, g, sysm, c, P, st, ctx = built(name, variant, restriction)
    K, m = 13, 8
    xo, ito, rro, _, ho = osolver.gmres_solve(st, tol=0.0, max_iter=K, restart=m, history=True)
    with _fams().Context(_gmres(p, m, K)) as ck:
        xs, stats = ck.solve(tol=0.0)
        hg = ck.query("HISTORY")
    assert stats[0]["iterations"] == K == ito
    assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
    # entries that end a cycle are true residuals ||q - A x|| / ||q||: their
    # rounding is absolute, about eps ||A|| ||x|| / ||q||
    np.testing.assert_allclose(hg[:K + 1], ho, rtol=1e-8, atol=1e-12)
    assert abs(stats[0]["rel_residual"] - rro) <= 1e-8 * rro + 1e-12


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["2d32", "2d64", "2d50ragged", "3d"])
def test_gmres_solve_to_tolerance(built, name, variant):
    p, g, sysm, c, P, st, ctx = built(name, variant)
    xo, ito, rro, oko, _ = osolver.gmres_solve(st, tol=1e-8, max_iter=p.max_iter, restart=30)
    with _fams().Context(_gmres(p, 30, p.max_iter)) as ck:
        xs, stats = ck.solve(tol=1e-8)
    x = xs[0]
    assert stats[0]["converged"] and oko
    assert abs(stats[0]["iterations"] - ito) <= 1
    rr = np.linalg.norm(sysm.q - sysm.A @ x) / np.linalg.norm(sysm.q)
    assert rr <= 1e-8
    assert abs(rr - stats[0]["rel_residual"]) <= 1e-6 * rr + 1e-13
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6


def _mixed(p, krylov, restart=30):
    q = copy.copy(p)
    q.precision, q.krylov, q.restart = 1, krylov, restart
    return q


@pytest.mark.parametrize("krylov", [0, 1])
@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("name", ["2d32", "2d64", "2d50ragged", "3d"])
def test_mixed_precision_reaches_the_fp64_tolerance(built, name, variant, krylov):
    """FP32 inner stages with FP64 residuals and refinement: the true FP64
    residual reaches tol, the solution matches the FP64 oracle's to tol x
    cond, and the iteration count stays close to the FP64 path's."""
    p, g, sysm, c, P, st, ctx = built(name, variant)
    if krylov:
        xo, ito, _, oko, _ = osolver.gmres_solve(st, tol=1e-8, max_iter=p.max_iter, restart=30)
    else:
        xo, ito, _, oko, _ = osolver.two_stage_solve(st, tol=1e-8, max_iter=p.max_iter)
    with _fams().Context(_mixed(p, krylov)) as cm:
        xs, stats = cm.solve(tol=1e-8)
    x = xs[0]
    rr = np.linalg.norm(sysm.q - sysm.A @ x) / np.linalg.norm(sysm.q)
    assert oko and stats[0]["converged"] and rr <= 1e-8
    assert abs(rr - stats[0]["rel_residual"]) <= 1e-6 * rr + 1e-13
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6
    assert stats[0]["iterations"] <= ito + max(3, ito // 4)


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("name", ["2d64", "2d50ragged", "3d"])
def test_bf16_stored_p_reaches_the_fp64_tolerance(built, name, variant):
    """fams_opts.bf16_p (P and P^T values of the FP32 restriction and
    prolongation stored in BF16): GMRES still reaches the FP64 tolerance, the
    solution matches the FP64 oracle's to tol x cond, and BF16 storage may
    cost iterations but not convergence; bf16_p without FAMS_MIXED is
    rejected."""
    p, g, sysm, c, P, st, ctx = built(name, variant)
    xo, ito, _, oko, _ = osolver.gmres_solve(st, tol=1e-8, max_iter=p.max_iter, restart=30)
    q = _mixed(p, 1)
    q.bf16_p, q.max_iter = 1, 400
    with _fams().Context(q) as cm:
        xs, stats = cm.solve(tol=1e-8)
    x = xs[0]
    rr = np.linalg.norm(sysm.q - sysm.A @ x) / np.linalg.norm(sysm.q)
    assert oko and stats[0]["converged"] and rr <= 1e-8
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6
    assert stats[0]["iterations"] <= 2 * ito + 10
    r = copy.copy(p)
    r.bf16_p = 1
    with pytest.raises(_fams().FamsError):
        _fams().Context(r)


def test_gmres_and_richardson_instances_share_a_batch(built):
    """A batch mixing both outer iterations gives each instance its own result."""
    pa = _gmres(built("2d32", 0)[0], 30, 200)
    pb = built("2d64", 3)[0]
    with _fams().Context([pa, pb]) as cab, _fams().Context(pa) as ca, \
            _fams().Context(pb) as cb:
        xs, st = cab.solve(tol=1e-8)
        xa, sa = ca.solve(tol=1e-8)
        xb, sb = cb.solve(tol=1e-8)
    assert st[0]["iterations"] == sa[0]["iterations"] and st[1]["iterations"] == sb[0]["iterations"]
    assert np.linalg.norm(xs[0] - xa[0]) / np.linalg.norm(xa[0]) < 1e-10
    assert np.linalg.norm(xs[1] - xb[0]) / np.linalg.norm(xb[0]) < 1e-10


def _interior_connections(p, face, nnc):
    """The device's fluxes in the oracle's connection order: interior x, y (z)
    faces, then the matrix-fracture and fracture-fracture connections."""
    nx, ny = p.nx, p.ny
    nz = p.nz if p.dim == 3 else 1
    nfx, nfy = (nx + 1) * ny * nz, nx * (ny + 1) * nz
    fx = face[:nfx].reshape(nz, ny, nx + 1)
    fy = face[nfx:nfx + nfy].reshape(nz, ny + 1, nx)
    parts = [fx[:, :, 1:-1].ravel(), fy[:, 1:-1, :].ravel()]
    if p.dim == 3:
        fz = face[nfx + nfy:].reshape(nz + 1, ny, nx)
        parts.append(fz[1:-1].ravel())
    return np.concatenate(parts + [nnc])


def _balance(sysm, p, face, conn):
    """Net outflow of every cell of a W/E problem without sources, from the
    device's face fluxes and connection fluxes."""
    nx, ny = p.nx, p.ny
    nz = p.nz if p.dim == 3 else 1
    fx = face[:(nx + 1) * ny * nz].reshape(nz, ny, nx + 1)
    ci, cj, _ = osolver.connections(sysm, p)
    out = np.zeros(sysm.n)
    np.add.at(out, ci, conn)
    np.subtract.at(out, cj, conn)
    xm = np.arange(sysm.n_matrix) % nx
    out[np.nonzero(xm == 0)[0]] -= fx[:, :, 0].ravel()
    out[np.nonzero(xm == nx - 1)[0]] += fx[:, :, -1].ravel()
    return out


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", ["2d32", "2d64", "3d"])
def test_flux_conservative_and_matches_oracle(built, name, restriction):
    p, g, sysm, c, P, st, ctx = built(name, 0, restriction)
    p.tol = 1e-4
    xs, stats = ctx.solve(tol=1e-4)
    x = xs[0]
    face, nnc = ctx.flux(x)
    # oracle reconstruction from the same iterate
    st_fv = oracle.reconstruction_setup(p, g, sysm, c)
    flux, dflux, pp, pt = osolver.reconstruct_flux(sysm, p, st_fv, x, c.primal, c.node_cell)
    gpu_conn = _interior_connections(p, face, nnc)
    scale = np.abs(flux).max()
    np.testing.assert_allclose(gpu_conn, flux, rtol=0, atol=1e-8 * scale)
    # cell-by-cell mass balance of the GPU field: conservative to round-off
    # (every flux is T (p_i - p_j), so a balance carries errors of order
    # eps T_max |p|_max; the oracle's own imbalance is of the same size)
    out = _balance(sysm, p, face, gpu_conn)
    _, _, cT = osolver.connections(sysm, p)
    bound = 64 * np.finfo(float).eps * cT.max() * max(np.abs(pt).max(), 1.0)
    assert np.abs(out).max() < bound
    nx, ny = p.nx, p.ny
    nz = p.nz if p.dim == 3 else 1
    fx = face[:(nx + 1) * ny * nz].reshape(nz, ny, nx + 1)
    assert abs(fx[:, :, 0].sum() - fx[:, :, -1].sum()) < sysm.n * bound


def test_batch_matches_single(built):
    """A batch of different instances gives each instance's single result
    (one CTA per instance, fixed reduction order in the iteration; the coarse
    operator is summed with atomic additions, so results agree to rounding)."""
    fams = _fams()
    probs = [_case("2d32", 0), _case("2d64", 0), _case("2d50ragged", 3)]
    with fams.Context(probs) as cb:
        xb, sb = cb.solve(tol=1e-8)
    for i, p in enumerate(probs):
        with fams.Context(p) as c1:
            x1, s1 = c1.solve(tol=1e-8)
        assert s1[0]["iterations"] == sb[i]["iterations"]
        assert np.linalg.norm(x1[0] - xb[i]) / np.linalg.norm(x1[0]) < 1e-10


def test_flux_batch_matches_single():
    """fams_flux_batch over a batch equals fams_flux of each instance alone."""
    fams = _fams()
    probs = [_case("2d32", 0, 1), _case("2d64", 3, 1), _case("3d", 1, 1)]
    with fams.Context(probs) as cb:
        xs, _ = cb.solve(tol=1e-6)
        S = [cb.sizes(i) for i in range(len(probs))]
        F = [np.zeros(s["n_faces"]) for s in S]
        N = [np.zeros(max(1, s["n_nnc"])) for s in S]
        st = cb.flux_batch_ptr([x.ctypes.data for x in xs], [f.ctypes.data for f in F],
                               [m.ctypes.data for m in N])
        assert st == [0, 0, 0]
        for i in range(len(probs)):
            f1, n1 = cb.flux(xs[i], i)
            np.testing.assert_array_equal(F[i], f1)
            np.testing.assert_array_equal(N[i][: S[i]["n_nnc"]], n1)


def _rows(ctx, i):
    s = ctx.sizes(i)
    return s["n_matrix"] + s["n_frac"]


def test_flux_prepared_beside_the_solve():
    """prepare_flux = 1 builds the R^FV coarse system on a second stream while
    the solve runs; the fluxes equal those of the system built on the first
    fams_flux call (to the rounding of the atomically summed coarse operator),
    also after a time-step update, which rebuilds it beside the next solve."""
    fams = _fams()

    def run(prep):
        probs = [_gmres(_case("2d64", 0, 1), 30, 200), _gmres(_case("3dcross", 1, 1), 30, 200),
                 _gmres(_case("2d50ragged", 2, 0), 30, 200)]
        for q in probs:
            q.prepare_flux = prep
        out = []
        with fams.Context(probs) as c:
            for sc_seed in (None, 5):
                if sc_seed is not None:
                    c.update([np.random.default_rng(sc_seed + i).uniform(0.5, 2.0, _rows(c, i))
                              for i in range(len(probs))])
                xs, st = c.solve(tol=1e-8)
                assert all(s["converged"] for s in st)
                out.append([(x,) + tuple(c.flux(x, i)) for i, x in enumerate(xs)])
        return out

    a, b = run(1), run(0)
    for ra, rb in zip(a, b):
        for (xa, fa, na), (xb, fb, nb) in zip(ra, rb):
            assert np.linalg.norm(xa - xb) / np.linalg.norm(xb) < 1e-10
            sc = max(np.abs(fb).max(), np.abs(nb).max() if len(nb) else 0.0)
            np.testing.assert_allclose(fa, fb, rtol=0, atol=1e-9 * sc)
            np.testing.assert_allclose(na, nb, rtol=0, atol=1e-9 * sc)


def test_flux_of_instances_with_a_singular_truncated_fv_system():
    """Instances whose R^FV A P with the truncated P is singular (a sealed
    node cell whose truncated basis function is its own cell; a 64 x 64
    instance with a numerically singular pivot) next to a regular one: the
    reconstruction's finite-volume stage uses the basis functions before
    truncation, so every instance is reconstructed, matches the oracle's
    reconstruction from the same iterate and conserves mass in every cell."""
    fams = _fams()
    sealed = inputs.config_2d_sealed_node(restriction=0)
    plain = inputs.config_2d_small(restriction=0)
    plain.alpha = 1e-2
    # truncation makes this instance's R^FV A P numerically singular
    bound = inputs.config_2d(64, 2.0, 8.0, 4, (10, 30), 1e4, 8, 8, seed=86, basis=2,
                             restriction=1, alpha=1e-2)
    probs = []
    for q in (sealed, plain, bound):
        q = _gmres(copy.copy(q), 30, 200)
        q.restriction = 1
        probs.append(q)
    with fams.Context(probs) as c:
        xs, st = c.solve(tol=1e-8)
        assert all(s["converged"] for s in st)
        S = [c.sizes(i) for i in range(3)]
        F = [np.full(s["n_faces"], 7.0) for s in S]
        N = [np.full(max(1, s["n_nnc"]), 7.0) for s in S]
        status = c.flux_batch_ptr([x.ctypes.data for x in xs], [f.ctypes.data for f in F],
                                  [m.ctypes.data for m in N])
        assert status == [0, 0, 0]
        for i, q in enumerate(probs):
            g, sysm, co, P, _ = oracle.build(q)
            trunc = osolver.coarse_operator(
                osolver.restriction(P, co.primal, co.n_coarse, osolver.R_FV), sysm.A, P)
            assert (osolver.singular_step(trunc) >= 0) == (i != 1)
            st_fv = oracle.reconstruction_setup(q, g, sysm, co)
            assert osolver.singular_step(st_fv.Ac) == -1
            flux, dflux, pp, pt = osolver.reconstruct_flux(sysm, q, st_fv, xs[i], co.primal,
                                                           co.node_cell)
            gpu_conn = _interior_connections(q, F[i], N[i][: S[i]["n_nnc"]])
            np.testing.assert_allclose(gpu_conn, flux, rtol=0, atol=1e-8 * np.abs(flux).max())
            _, _, cT = osolver.connections(sysm, q)
            bound = 64 * np.finfo(float).eps * cT.max() * max(np.abs(pt).max(), 1.0)
            assert np.abs(_balance(sysm, q, F[i], gpu_conn)).max() < bound


def test_flux_reports_a_singular_fv_coarse_system():
    """A node cell sealed to 1e-300: its basis function is 1e-300 outside the
    node cell and R^FV A P is singular by the oracle's scaled pivot test.  The
    R^FV iteration reports FAMS_EBREAKDOWN from the solve, and the
    reconstruction of that instance reports FAMS_EBREAKDOWN and leaves its
    buffers untouched, while a regular instance of the same batch is
    reconstructed as alone."""
    fams = _fams()
    sealed = inputs.config_2d_sealed_node(restriction=0, factor=1e-300)
    plain = inputs.config_2d_small(restriction=0)
    plain.alpha = 1e-2
    assert osolver.singular_step(oracle.build(sealed)[4].Ac) >= 0
    assert osolver.singular_step(oracle.build(plain)[4].Ac) == -1
    with fams.Context(sealed) as c:
        with pytest.raises(fams.FamsError) as e:
            c.solve(tol=1e-8)
        assert e.value.status == fams.EBREAKDOWN
    x_plain = oracle.run(plain).p
    with fams.Context([sealed, plain]) as c:
        S = [c.sizes(i) for i in range(2)]
        xs = [np.zeros(S[0]["n_matrix"] + S[0]["n_frac"]), x_plain]
        F = [np.full(s["n_faces"], 7.0) for s in S]
        N = [np.full(max(1, s["n_nnc"]), 7.0) for s in S]
        status = c.flux_batch_ptr([x.ctypes.data for x in xs], [f.ctypes.data for f in F],
                                  [m.ctypes.data for m in N])
        assert status == [fams.EBREAKDOWN, 0]
        assert (F[0] == 7.0).all() and (N[0] == 7.0).all()
        f1, n1 = c.flux(x_plain, 1)
        np.testing.assert_array_equal(F[1], f1)
        np.testing.assert_array_equal(N[1][: S[1]["n_nnc"]], n1)


def _degenerate(dim, nx, ny, nz, coarsen, seed=3):
    shape = (nx, ny) if dim == 2 else (nx, ny, nz)
    perm = (10 ** inputs.gaussian_field(shape, 1.0, 3.0, seed)).reshape(-1)
    return inputs.Problem(dim=dim, nx=nx, ny=ny, nz=nz, perm=perm,
                          fracs=np.zeros((0, 4 if dim == 2 else 6)), kf=np.zeros(0),
                          coarsen=coarsen, frac_dmin=5, basis=0, restriction=1, alpha=0.0)


@pytest.mark.parametrize("args", [(2, 16, 16, 1, (4, 4, 1)),    # no fractures
                                  (2, 16, 16, 1, (1, 1, 1)),    # every cell a coarse node
                                  (2, 1, 12, 1, (4, 4, 1)),     # one column of cells
                                  (2, 5, 3, 1, (8, 8, 1)),      # one partial primal block
                                  (3, 6, 5, 4, (2, 2, 2))])     # 3D without plates
def test_degenerate_inputs_match_the_oracle(args):
    """Inputs at the edges of the method: the GMRES trajectory, the converged
    pressure and the conservative fluxes equal the oracle's."""
    fams = _fams()
    p = _gmres(_degenerate(*args), 30, 200)
    g, sysm, c, P, st = oracle.build(p)
    xo, ito, _, oko, _ = osolver.gmres_solve(st, tol=1e-10, max_iter=200, restart=30)
    with fams.Context(p) as ctx:
        assert ctx.sizes()["n_coarse"] == c.n_coarse
        Pg = _gpu_P(ctx, P.shape)
        np.testing.assert_array_equal(Pg.indptr, P.indptr)
        np.testing.assert_array_equal(Pg.indices, P.indices)
        np.testing.assert_allclose(Pg.data, P.data, rtol=0, atol=1e-12)
        xs, stats = ctx.solve(tol=1e-10)
        assert stats[0]["converged"] and oko
        assert abs(stats[0]["iterations"] - ito) <= 1
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-8
        face, nnc = ctx.flux(xs[0])
    sfv = oracle.reconstruction_setup(p, g, sysm, c)
    flux, dflux, _, _ = osolver.reconstruct_flux(sysm, p, sfv, xs[0], c.primal, c.node_cell)
    nz = p.nz if p.dim == 3 else 1
    nfx, nfy = (p.nx + 1) * p.ny * nz, p.nx * (p.ny + 1) * nz
    parts = [face[:nfx].reshape(nz, p.ny, p.nx + 1)[:, :, 1:-1].ravel(),
             face[nfx:nfx + nfy].reshape(nz, p.ny + 1, p.nx)[:, 1:-1, :].ravel()]
    if p.dim == 3:
        parts.append(face[nfx + nfy:].reshape(nz + 1, p.ny, p.nx)[1:-1].ravel())
    conn = np.concatenate(parts + [nnc])
    # scale: the largest flux including the Dirichlet faces (in a single
    # column every internal flux is rounding noise)
    scale = max(np.abs(flux).max(), np.abs(dflux).max())
    np.testing.assert_allclose(conn, flux, rtol=0, atol=1e-9 * scale)


def test_rejects_bad_input():
    fams = _fams()
    p = _case("2d32")
    p.bc_mask = 0
    with pytest.raises(fams.FamsError) as e:
        fams.Context(p)
    assert e.value.status == fams.EINVAL
    # permeability not positive and finite (checked on the device)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        q = _case("2d32")
        q.perm = q.perm.copy()
        q.perm[37] = bad
        with pytest.raises(fams.FamsError) as e:
            fams.Context([_case("2d64"), q])
        assert e.value.status == fams.EINVAL and "permeability" in str(e.value)


# --- time-step update (fams_update): mobility scales, P reused ---

@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", ["2d64", "2d50ragged", "3dcross"])
def test_time_step_update_matches_oracle(name, restriction):
    """After fams_update the fine system, the coarse operator, ILU(0), a
    GMRES trajectory and the conservative fluxes equal the oracle's for the
    scaled system with the setup-time P; a second update replaces the first
    (scales are relative to the setup), and no scale restores the setup."""
    from oracle import assemble as oasm
    fams = _fams()
    p = _gmres(_case(name, 0, restriction), 8, 13)
    g, sysm, c, P, st0 = oracle.build(p)
    Pf = oracle.prolongation(p, g, sysm, c, truncated=False)   # the reconstruction's P
    n = sysm.n
    with fams.Context(p) as ctx:
        for seed in (3, 4):
            sc = np.random.default_rng(seed).uniform(0.25, 4.0, n)
            ur = oasm.update_mobility(sysm, sc)
            su = osolver.setup(ur, P, c.primal, c.n_coarse, p.restriction)
            ctx.update(sc)
            np.testing.assert_allclose(ctx.query("A_VAL"), ur.A.data, rtol=1e-13,
                                       atol=1e-15 * abs(ur.A).max())
            Ac = ctx.query("AC").reshape(c.n_coarse, c.n_coarse)
            np.testing.assert_allclose(Ac, su.Ac, rtol=0, atol=1e-11 * np.abs(su.Ac).max())
            F = ctx.query("ILU_VAL")
            np.testing.assert_allclose(F, su.F.data, rtol=1e-11, atol=1e-13 * np.abs(su.F.data).max())
            xo, ito, _, _, _ = osolver.gmres_solve(su, tol=0.0, max_iter=13, restart=8)
            xs, stats = ctx.solve(tol=0.0)
            assert stats[0]["iterations"] == 13 == ito
            assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
            face, nnc = ctx.flux(xs[0])
            sfv = osolver.setup(ur, Pf, c.primal, c.n_coarse, osolver.R_FV)
            flux, dflux, _, _ = osolver.reconstruct_flux(ur, p, sfv, xs[0], c.primal, c.node_cell)
            nz = p.nz if p.dim == 3 else 1
            nfx, nfy = (p.nx + 1) * p.ny * nz, p.nx * (p.ny + 1) * nz
            fx = face[:nfx].reshape(nz, p.ny, p.nx + 1)
            fy = face[nfx:nfx + nfy].reshape(nz, p.ny + 1, p.nx)
            parts = [fx[:, :, 1:-1].ravel(), fy[:, 1:-1, :].ravel()]
            if p.dim == 3:
                parts.append(face[nfx + nfy:].reshape(nz + 1, p.ny, p.nx)[1:-1].ravel())
            conn = np.concatenate(parts + [nnc])
            np.testing.assert_allclose(conn, flux, rtol=0, atol=1e-8 * np.abs(flux).max())
        ctx.update(None)
        np.testing.assert_allclose(ctx.query("A_VAL"), sysm.A.data, rtol=1e-13,
                                   atol=1e-15 * abs(sysm.A).max())


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", ["2d64", "2d50ragged", "3dcross"])
def test_basis_rebuild_matches_oracle(name, restriction):
    """fams_update_basis, the adaptive update of Sec. 3.1 per dual block:
    with a threshold above every change nothing is solved and P stays; with
    scales moved in a patch only the blocks holding a moved cell and their
    downstream blocks are solved again -- the same blocks as the oracle's
    (count bit-exact) -- and P, R A P, a GMRES trajectory and the fluxes
    equal the oracle's; the same scales again solve nothing; eps < 0 solves
    every block."""
    from oracle import assemble as oasm
    fams = _fams()
    p = _gmres(_case(name, 0, restriction), 8, 13)
    g, sysm, c, P, st0 = oracle.build(p)
    Pf = oracle.prolongation(p, g, sysm, c, truncated=False)
    rng = np.random.default_rng(7)
    sc = np.ones(sysm.n)
    patch = rng.choice(g.n_matrix, size=max(8, g.n_matrix // 20), replace=False)
    sc[patch] = rng.uniform(3.0, 6.0, len(patch))
    sc[g.n_matrix:] = rng.uniform(0.9, 1.1, g.n_frac)      # below the threshold
    with fams.Context(p) as ctx:
        assert ctx.update_basis(sc, 10.0) == 0
        Pg = _gpu_P(ctx, P.shape)
        np.testing.assert_array_equal(Pg.indices, P.indices)
        np.testing.assert_allclose(Pg.data, P.data, rtol=0, atol=1e-12)
        n_solved = ctx.update_basis(sc, 0.5)
        ur = oasm.update_mobility(sysm, sc)
        Pu, Puf, ref, solved = oracle.prolongation_update(p, g, ur, c, Pf, np.ones(sysm.n), sc,
                                                          0.5)
        total = len(oracle.basis.stage_blocks(
            sysm.A0, c.rank, c.medium, c.node_cell, p.basis,
            np.concatenate([np.full(g.n_matrix, -1), g.cell_frac]), c.row_net))
        assert n_solved == solved and 0 < solved < total
        Pg = _gpu_P(ctx, Pu.shape)
        np.testing.assert_array_equal(Pg.indptr, Pu.indptr)
        np.testing.assert_array_equal(Pg.indices, Pu.indices)
        np.testing.assert_allclose(Pg.data, Pu.data, rtol=0, atol=1e-12)
        su = osolver.setup(ur, Pu, c.primal, c.n_coarse, p.restriction)
        Ac = ctx.query("AC").reshape(c.n_coarse, c.n_coarse)
        np.testing.assert_allclose(Ac, su.Ac, rtol=0, atol=1e-11 * np.abs(su.Ac).max())
        xo, ito, _, _, _ = osolver.gmres_solve(su, tol=0.0, max_iter=13, restart=8)
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 13 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
        face, nnc = ctx.flux(xs[0])
        sfv = osolver.setup(ur, Puf, c.primal, c.n_coarse, osolver.R_FV)
        flux, dflux, _, _ = osolver.reconstruct_flux(ur, p, sfv, xs[0], c.primal, c.node_cell)
        conn = _interior_connections(p, face, nnc)
        np.testing.assert_allclose(conn, flux, rtol=0, atol=1e-8 * np.abs(flux).max())
        assert ctx.update_basis(sc, 0.5) == 0
        assert ctx.update_basis(sc, -1.0) == total


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("name", ["2d64", "2d50ragged", "3dcross"])
def test_msmix_matches_oracle(name, variant):
    """MSMIX restriction (P^T rows for matrix coarse nodes, indicators for
    fracture coarse nodes): R A P, a GMRES trajectory and the converged
    solution equal the oracle's."""
    fams = _fams()
    p = _gmres(_case(name, variant, osolver.R_MIX), 8, 13)
    g, sysm, c, P, st = oracle.build(p)
    with fams.Context(p) as ctx:
        Ac = ctx.query("AC").reshape(c.n_coarse, c.n_coarse)
        np.testing.assert_allclose(Ac, st.Ac, rtol=0, atol=1e-11 * np.abs(st.Ac).max())
        xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=13, restart=8)
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 13 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
    q = _gmres(_case(name, variant, osolver.R_MIX), 30, 300)
    with fams.Context(q) as ctx:
        xs, stats = ctx.solve(tol=1e-8)
        assert stats[0]["converged"]
    xd, _, _, okd, _ = osolver.gmres_solve(st, tol=1e-8, max_iter=300, restart=30)
    assert okd and np.linalg.norm(xs[0] - xd) / np.linalg.norm(xd) < 1e-6


def test_bench_workload_instances_match_the_oracle():
    """The bench workload at full size (256x256, GMRES(30), R^FE, reconstruction
    prepared beside the solve) in a batch of 16: two sampled instances against
    the oracle, both converged to 1e-8 -- pressure and conservative fluxes."""
    import bench
    fams = _fams()
    probs = bench.problems(16, bench.ORACLE_SEED)
    with fams.Context(probs) as c:
        xs, st = c.solve(tol=bench.TOL)
        assert all(s["converged"] for s in st)
        for i in (0, 1):
            p = probs[i]
            g, sysm, co, P, so = oracle.build(p)
            xo, _, _, oko, _ = osolver.gmres_solve(so, tol=bench.TOL, max_iter=p.max_iter,
                                                   restart=p.restart)
            assert oko
            assert np.linalg.norm(xs[i] - xo) / np.linalg.norm(xo) < 1e-6
            sfv = oracle.reconstruction_setup(p, g, sysm, co)
            fo, _, _, _ = osolver.reconstruct_flux(sysm, p, sfv, xo, co.primal, co.node_cell)
            face, nnc = c.flux(xs[i], i)
            assert np.abs(bench.conn_fluxes(p, face, nnc) - fo).max() < 1e-6 * np.abs(fo).max()


def _bench_oracle(i):
    """Pool worker: the oracle on instance i of the 16-instance bench batch --
    its GMRES(30) iteration count to 1e-8, the iterate after exactly that many
    iterations, and the trajectory's own rounding sensitivity: the relative
    change of that iterate when the initial guess 0 is replaced by 1e-14
    times a seeded normal vector (a perturbation at the rounding level of a
    pressure of order one)."""
    import warnings
    warnings.simplefilter("ignore")
    import bench
    p = bench.problems(16, bench.ORACLE_SEED)[i]
    g, sysm, co, P, so = oracle.build(p)
    xo, ito, rro, oko, _ = osolver.gmres_solve(so, tol=bench.TOL, max_iter=p.max_iter,
                                               restart=p.restart)
    x0 = 1e-14 * np.random.default_rng(100 + i).standard_normal(sysm.n)
    x1, _, _, _, _ = osolver.gmres_solve(so, x0=x0, tol=0.0, max_iter=ito, restart=p.restart)
    sens = np.linalg.norm(x1 - xo) / np.linalg.norm(xo)
    return i, xo, ito, oko, sens


def _bench_oracle_flux(args):
    """Pool worker: the oracle's reconstruction of bench instance i from an
    iterate x, and its own rounding sensitivity: the largest change of a flux
    when x is perturbed by 1e-14 times a seeded normal vector."""
    import warnings
    warnings.simplefilter("ignore")
    import bench
    i, x = args
    p = bench.problems(16, bench.ORACLE_SEED)[i]
    g, sysm, co, P, so = oracle.build(p)
    sfv = oracle.reconstruction_setup(p, g, sysm, co)
    fo, _, _, _ = osolver.reconstruct_flux(sysm, p, sfv, x, co.primal, co.node_cell)
    xp = x + 1e-14 * np.random.default_rng(200 + i).standard_normal(len(x))
    f1, _, _, _ = osolver.reconstruct_flux(sysm, p, sfv, xp, co.primal, co.node_cell)
    return i, fo, np.abs(f1 - fo).max()


def test_bench_workload_trajectories_at_full_size():
    """Every kind of instance of the bench workload at full size (256x256,
    the four coupling strategies x T_ratio 1e2, 1e4, 1e6, 1e8: a batch of
    16 with the bench's options): each instance converges in the oracle's
    iteration count, after exactly that many GMRES iterations its pressure
    equals the oracle's to 1e-10 relative L2 -- or, where the oracle's own
    trajectory moves by more under a rounding-level change of its initial
    guess (T_ratio 1e6 and 1e8 reach 1e-9..3e-7: the systems' conditioning
    amplifies rounding), to 10 times that sensitivity -- and its conservative
    fluxes from that iterate equal the oracle's reconstruction to 1e-8 of the
    largest flux, or to 10 times the oracle reconstruction's own change under
    a 1e-14 perturbation of the iterate.  The oracle runs on the host cores in
    spawned processes."""
    import multiprocessing as mp
    import bench
    fams = _fams()
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        ref = {i: (xo, ito, oko, sens) for i, xo, ito, oko, sens in
               pool.imap_unordered(_bench_oracle, range(16))}
        assert all(ref[i][2] for i in range(16))
        probs = bench.problems(16, bench.ORACLE_SEED)
        with fams.Context(probs) as c:
            xs, st = c.solve(tol=bench.TOL)
        its = [s["iterations"] for s in st]
        assert all(s["converged"] for s in st)
        assert its == [ref[i][1] for i in range(16)], (its, [ref[i][1] for i in range(16)])
        # the same batch with each instance stopped after the oracle's count
        for i, p in enumerate(probs):
            p.max_iter = ref[i][1]
        with fams.Context(probs) as c:
            xk, stk = c.solve(tol=0.0)
            assert [s["iterations"] for s in stk] == [ref[i][1] for i in range(16)]
            errs = [np.linalg.norm(xk[i] - ref[i][0]) / np.linalg.norm(ref[i][0])
                    for i in range(16)]
            bounds = [max(1e-10, 10.0 * ref[i][3]) for i in range(16)]
            assert all(e <= b for e, b in zip(errs, bounds)), list(zip(errs, bounds))
            fl = [c.flux(xk[i], i) for i in range(16)]
        for i, fo, fs in pool.imap_unordered(_bench_oracle_flux, [(i, xk[i]) for i in range(16)]):
            got = bench.conn_fluxes(probs[i], *fl[i])
            bound = max(1e-8 * np.abs(fo).max(), 10.0 * fs)
            assert np.abs(got - fo).max() < bound, (i, np.abs(got - fo).max(), bound)


def _class_case(variant):
    """3D, coarsening 8 x 8 x 8: interior dual blocks of 343 cells and primal
    blocks of 512 cells exceed shared memory as banded systems, so both the
    basis and the reconstruction take the global-workspace size class."""
    p = inputs.config_3d(24, 24, 16, 1.0, (6, 6, 3), 0, (6, 14), 1e3, (8, 8, 8), 8, 8, seed=12,
                         basis=variant, restriction=1)
    p.fracs = np.array([[2.5, 9.3, 21.5, 14.1, 0.0, 16.0], [12.3, 1.5, 11.1, 22.5, 0.0, 16.0]])
    p.kf = np.array([1e3, 1e4])
    return p


@pytest.mark.parametrize("variant", [0, 3])
def test_global_workspace_size_class_matches_the_oracle(variant):
    """The size class that solves local problems on a global-memory
    workspace: the query shows it was taken for dual blocks and primal
    blocks; P, a fixed-count GMRES trajectory and the fluxes equal the
    oracle's."""
    fams = _fams()
    p = _gmres(_class_case(variant), 30, 12)
    g, sysm, c, P, st = oracle.build(p)
    with fams.Context(p) as ctx:
        Pg = _gpu_P(ctx, P.shape)
        np.testing.assert_array_equal(Pg.indptr, P.indptr)
        np.testing.assert_array_equal(Pg.indices, P.indices)
        np.testing.assert_allclose(Pg.data, P.data, rtol=0, atol=1e-12)
        xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=12, restart=30)
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 12 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
        face, nnc = ctx.flux(xs[0])
        cc = ctx.query("CLASS_COUNTS")
        assert cc[3] > 0 and cc[7] > 0, cc
    sfv = oracle.reconstruction_setup(p, g, sysm, c)
    flux, _, _, pt = osolver.reconstruct_flux(sysm, p, sfv, xs[0], c.primal, c.node_cell)
    conn = _interior_connections(p, face, nnc)
    np.testing.assert_allclose(conn, flux, rtol=0, atol=1e-8 * np.abs(flux).max())
    # conservative to the rounding of the local solves: their residual grows
    # with the block size m (Wilkinson's n eps bound of a backward-stable
    # elimination), so the per-cell bound is max(64, 4 m) eps T_max |p|_max
    _, _, cT = osolver.connections(sysm, p)
    m = np.bincount(c.primal).max()
    bound = max(64, 4 * m) * np.finfo(float).eps * cT.max() * max(np.abs(pt).max(), 1.0)
    assert np.abs(_balance(sysm, p, face, conn)).max() < bound


@pytest.mark.parametrize("cap", [8, 16])
@pytest.mark.parametrize("name", ["3dcross", "3dlayers"])
def test_coupled_merge_cap_matches_the_oracle(name, cap):
    """Coupled-AMS with a merge cap (fams_opts.merge_cap): P bit-for-bit in
    pattern and to 1e-12 in value, and a fixed-count GMRES trajectory to
    1e-10, against the oracle's capped merge."""
    fams = _fams()
    p = _gmres(_case(name, 3, 1), 30, 12)
    p.merge_cap = cap
    g, sysm, c, P, st = oracle.build(p)
    plate = np.concatenate([np.full(g.n_matrix, -1), g.cell_frac])
    from oracle import basis as obasis
    assert obasis.cut_links(sysm.A0, c.rank, c.medium, c.node_cell, 3, plate, c.row_net, cap)
    with fams.Context(p) as ctx:
        Pg = _gpu_P(ctx, P.shape)
        np.testing.assert_array_equal(Pg.indptr, P.indptr)
        np.testing.assert_array_equal(Pg.indices, P.indices)
        np.testing.assert_allclose(Pg.data, P.data, rtol=0, atol=1e-12)
        xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=12, restart=30)
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 12 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10


@pytest.mark.parametrize("coarse_mode", [1, 2])
@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", ["2d64", "2d50ragged", "3d", "3dlayers"])
def test_whole_gpu_solve_matches_the_oracle(name, restriction, coarse_mode):
    """The iteration of a single instance on every SM (fams_opts.grid_solve =
    1: one cooperative kernel, grid barriers per ILU level; the coarse solve
    by A_c^-1 formed from the band factors or by the band factors on one CTA):
    a fixed-count GMRES trajectory to 1e-10 against the oracle, and the
    converged solve in the same iteration count (+-1) as the one-CTA kernel."""
    fams = _fams()
    p = _gmres(_case(name, 3 if name.startswith("3d") else 1, restriction), 10, 17)
    p.grid_solve, p.coarse_mode = 1, coarse_mode
    g, sysm, c, P, st = oracle.build(p)
    xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=17, restart=10)
    with fams.Context(p) as ctx:
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 17 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
    q = _gmres(p, 30, 300)
    res = []
    for mode in (1, -1):
        q.grid_solve = mode
        with fams.Context(q) as ctx:
            xs, stats = ctx.solve(tol=1e-9)
            assert stats[0]["converged"]
            res.append((xs[0], stats[0]["iterations"]))
    assert abs(res[0][1] - res[1][1]) <= 1
    assert np.linalg.norm(res[0][0] - res[1][0]) / np.linalg.norm(res[1][0]) < 1e-6


@pytest.mark.parametrize("grid", [-1, 1])
@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("name", ["2d64", "3dcross"])
def test_sub_block_smoothing_stage_matches_the_oracle(name, restriction, grid):
    """fams_opts.subblock: the extra smoothing stage on the media blocks
    (Sec. 3.2) in the GMRES preconditioner, on one CTA and on every SM: a
    fixed-count trajectory to 1e-10; the Table 1 loop with it too."""
    fams = _fams()
    p = _gmres(_case(name, 0, restriction), 10, 15)
    p.subblock, p.grid_solve = 1, grid
    g, sysm, c, P, st = oracle.build(p)
    assert st.Fb is not None
    xo, ito, _, _, _ = osolver.gmres_solve(st, tol=0.0, max_iter=15, restart=10)
    with fams.Context(p) as ctx:
        xs, stats = ctx.solve(tol=0.0)
        assert stats[0]["iterations"] == 15 == ito
        assert np.linalg.norm(xs[0] - xo) / np.linalg.norm(xo) < 1e-10
    if grid < 0 and restriction == 1:
        q = copy.copy(p)
        q.krylov, q.max_iter = 0, 9
        xt, itt, _, _, _ = osolver.two_stage_solve(st, tol=0.0, max_iter=9)
        with fams.Context(q) as ctx:
            xs, stats = ctx.solve(tol=0.0)
            assert stats[0]["iterations"] == 9 == itt
            assert np.linalg.norm(xs[0] - xt) / np.linalg.norm(xt) < 1e-10


def test_oversize_coarse_band_goes_to_the_whole_gpu():
    """A single instance below the automatic whole-GPU size whose coarse
    band is wider than the one-CTA kernels' band chunks (a 40^3 cube with
    189 plates at coarsening 4-8) is solved on the whole GPU when the caller
    leaves the choice to the library, as when it asks for it; with the
    one-CTA path forced it fails with FAMS_ECAPACITY."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    fams = _fams()
    p = bench.serve_stream(7, 4)[6][1]
    assert p.dim == 3 and p.nx == 40 and len(p.fracs) == 189
    with fams.Context(p) as c:
        kl, ku = c.query("BAND_KLKU")
        assert kl + ku + 1 > 3072 and c.sizes()["n"] < (1 << 18)
        xa, sa = c.solve(tol=1e-8)
        assert sa[0]["converged"]
    q = copy.copy(p)
    q.grid_solve = 1
    with fams.Context(q) as c:
        xg, sg = c.solve(tol=1e-8)
    assert sg[0]["iterations"] == sa[0]["iterations"]
    assert np.linalg.norm(xa[0] - xg[0]) / np.linalg.norm(xg[0]) < 1e-10
    q.grid_solve = -1
    with fams.Context(q) as c:
        with pytest.raises(fams.FamsError) as e:
            c.solve(tol=1e-8)
        assert e.value.status == fams.ECAPACITY


def test_whole_gpu_coarse_modes_agree_on_a_large_coarse_system():
    """7396 coarse unknowns (256^2 cells at coarsening 3): solving with the
    band factors on one CTA and with A_c^-1 gives the same iterations and
    solution to 1e-10."""
    fams = _fams()
    p = inputs.config_2d(256, 2.0, 16.0, 20, (20, 80), 1e4, 3, 6, seed=12, basis=1, restriction=1,
                         alpha=1e-2, krylov=1, restart=30, max_iter=200)
    p.grid_solve = 1
    res = []
    for mode in (2, 1):
        p.coarse_mode = mode
        with fams.Context(p) as c:
            assert c.sizes()["n_coarse"] > 6000
            xs, st = c.solve(tol=1e-9)
            assert st[0]["converged"]
            res.append((xs[0], st[0]["iterations"]))
    assert res[0][1] == res[1][1]
    assert np.linalg.norm(res[0][0] - res[1][0]) / np.linalg.norm(res[1][0]) < 1e-10
