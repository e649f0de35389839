"""Pins of the oracle's EDFM geometry and fine system (Sec. 2, Eqs. 1-8)
against closed forms, invariants and brute force."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import assemble, geometry
from paper_1705_05784_gb300 import inputs


def _prob(fracs, nx=16, ny=16, kf=100.0, perm=None, dim=2, nz=1, **kw):
    fr = np.asarray(fracs, float).reshape(-1, 4 if dim == 2 else 6)
    n = nx * ny * (nz if dim == 3 else 1)
    return inputs.Problem(dim=dim, nx=nx, ny=ny, nz=nz,
                          perm=np.ones(n) if perm is None else perm,
                          fracs=fr, kf=np.full(len(fr), kf), **kw)


def test_clip_segment():
    assert geometry.clip_segment(1, 1, 3, 2, 10, 10) == (1, 1, 3, 2)
    c = geometry.clip_segment(-2, 5, 12, 5, 10, 10)
    assert c == (0.0, 5.0, 10.0, 5.0)
    assert geometry.clip_segment(-5, -5, -1, -1, 10, 10) is None


def test_axis_aligned_fracture_cells_and_overlaps():
    # a horizontal fracture along y = 5.5 from x = 2 to 12: ten unit cells,
    # each overlapping exactly the matrix cell it lies in
    g = geometry.build_geometry(_prob([2, 5.5, 12, 5.5]))
    assert g.n_frac == 10
    assert list(g.nnc_f) == list(range(10))
    assert list(g.nnc_m) == [2 + s + 16 * 5 for s in range(10)]
    np.testing.assert_allclose(g.nnc_area, 1.0, rtol=0, atol=1e-14)
    # the line runs through the cell middle: <d> = 1/4 exactly
    np.testing.assert_allclose(g.nnc_dist, 0.25, rtol=0, atol=1e-15)


def test_overlap_lengths_sum_to_fracture_length():
    rng = np.random.default_rng(0)
    for _ in range(20):
        seg = rng.uniform(1, 15, 4)
        g = geometry.build_geometry(_prob(seg))
        if g.n_frac == 0:
            continue
        L = math.hypot(seg[2] - seg[0], seg[3] - seg[1])
        assert abs(g.nnc_area.sum() - L) < 1e-12 * max(L, 1)
        # every fracture cell overlaps at least one matrix cell
        assert set(g.nnc_f) == set(range(g.n_frac))
        # cell count = floor(L/h + 1/2)
        assert g.n_frac == max(1, int(math.floor(L + 0.5)))


def test_mean_distance_closed_forms():
    # a line clear of the cell: the distance is linear over the cell, so its
    # mean is the distance to the cell centre
    d = geometry.mean_distance(0, 10.0, 20, 10.0, 3, 2, 1.0, 1.0)
    assert abs(d - (10.0 - 2.5)) < 1e-14
    d = geometry.mean_distance(0, -4.0, 20, -4.0, 3, 2, 1.0, 1.0)
    assert abs(d - (2.5 + 4.0)) < 1e-14
    # the diagonal through a unit cell: mean |x - y| / sqrt(2) = 1 / (3 sqrt 2)
    d = geometry.mean_distance(0, 0, 8, 8, 3, 3, 1.0, 1.0)
    assert abs(d - 1.0 / (3 * math.sqrt(2))) < 1e-15
    # an axis-parallel line through the centre of a dx x dy cell: dx / 4
    d = geometry.mean_distance(3.5 * 2.0, -5.0, 3.5 * 2.0, 30.0, 3, 1, 2.0, 0.5)
    assert abs(d - 0.5) < 1e-15
    # a line at distance a < dx/2 from the centre, parallel to y:
    # mean |x - c| over [0, dx] = ((dx/2 + a)^2 + (dx/2 - a)^2) / (2 dx)
    a, w = 0.3, 2.0
    d = geometry.mean_distance(3 * w + w / 2 + a, 0.0, 3 * w + w / 2 + a, 9.0, 3, 1, w, 1.0)
    assert abs(d - ((w / 2 + a) ** 2 + (w / 2 - a) ** 2) / (2 * w)) < 1e-15


def test_mean_distance_against_brute_force_sampling():
    """A fine midpoint rule (1024^2 points) on random lines and cells: the
    exact mean differs from it by the rule's O(h^2) error only."""
    rng = np.random.default_rng(4)
    m = 1024
    u = (np.arange(m) + 0.5) / m
    for _ in range(20):
        ax, ay, bx, by = rng.uniform(0, 8, 4)
        ix, iy = rng.integers(0, 8, 2)
        dx, dy = rng.uniform(0.5, 2.0, 2)
        X, Y = np.meshgrid(ix * dx + u * dx, iy * dy + u * dy, indexing="ij")
        ex, ey = bx - ax, by - ay
        L = math.hypot(ex, ey)
        ref = np.abs((ex * (Y - ay) - ey * (X - ax)) / L).mean()
        d = geometry.mean_distance(ax, ay, bx, by, ix, iy, dx, dy)
        assert abs(d - ref) < 1e-6 * max(dx, dy)


def test_segment_intersection():
    t, u = geometry.segment_intersection((0, 0, 4, 4), (0, 4, 4, 0))
    assert abs(t - 0.5) < 1e-15 and abs(u - 0.5) < 1e-15
    assert geometry.segment_intersection((0, 0, 1, 0), (0, 1, 1, 1)) is None
    assert geometry.segment_intersection((0, 0, 1, 1), (2, 0, 3, -1)) is None


def test_system_symmetry_and_row_sums():
    p = inputs.config_2d(24, 1.0, 4.0, 4, (6, 14), 1e3, 4, 4, seed=5)
    s = assemble.assemble(p)
    A, A0 = s.A, s.A0
    assert abs(A - A.T).max() == 0.0
    assert np.abs(np.asarray(A0.sum(axis=1)).ravel()).max() < 1e-12 * abs(A0).max()
    # matrix-fracture connections: equal and opposite total flux (Eq. 6)
    nm = s.n_matrix
    g = s.geom
    for m, f in zip(g.nnc_m[:10], g.nnc_f[:10]):
        assert A[m, nm + f] == A[nm + f, m] < 0
    # off-diagonals non-positive, diagonal dominance
    off = A - sp.diags(A.diagonal())
    assert off.max() <= 0
    assert (A.diagonal() + np.asarray(off.sum(axis=1)).ravel() >= -1e-12).all()


def test_tpfa_two_cell_brute_force():
    p = inputs.Problem(dim=2, nx=2, ny=1, nz=1, perm=np.array([1.0, 4.0]),
                       fracs=np.zeros((0, 4)), kf=np.zeros(0), dx=2.0, dy=3.0, dz=0.5)
    s = assemble.assemble(p)
    area = 3.0 * 0.5
    T = area / (2.0 / 2 / 1.0 + 2.0 / 2 / 4.0)
    TDw = 2 * 1.0 * area / 2.0
    TDe = 2 * 4.0 * area / 2.0
    want = np.array([[T + TDw, -T], [-T, T + TDe]])
    np.testing.assert_allclose(s.A.toarray(), want, rtol=1e-15)
    np.testing.assert_allclose(s.q, [TDw * 1.0, 0.0], rtol=1e-15)


def test_linear_pressure_closed_form():
    # homogeneous, fracture-free, Dirichlet W=1 / E=0 with half-cell T_D:
    # p_i = 1 - (i + 1/2)/nx exactly
    for dim, shape in ((2, (20, 7, 1)), (3, (9, 4, 3))):
        nx, ny, nz = shape
        p = inputs.Problem(dim=dim, nx=nx, ny=ny, nz=nz, perm=np.ones(nx * ny * nz),
                           fracs=np.zeros((0, 4 if dim == 2 else 6)), kf=np.zeros(0))
        s = assemble.assemble(p)
        x = spla.spsolve(s.A.tocsc(), s.q)
        want = np.tile(1 - (np.arange(nx) + 0.5) / nx, ny * nz)
        np.testing.assert_allclose(x, want, rtol=0, atol=1e-12)


def test_star_delta_equals_explicit_intersection_dof():
    """Two crossing fractures: eliminating the intersection pressure by the
    star-delta rule gives the same fracture pressures as keeping it as an
    explicit unknown with its own flux balance (Sec. 4.1)."""
    p = _prob([[2.2, 3.1, 13.7, 11.9], [3.3, 12.6, 12.9, 2.4]], kf=50.0,
              perm=10 ** inputs.gaussian_field((16, 16), 1.0, 3.0, 11))
    s = assemble.assemble(p)
    g = s.geom
    x = spla.spsolve(s.A.tocsc(), s.q)
    # explicit system: drop the eliminated link, add one unknown
    k = int(np.nonzero(g.ff_kind == 2)[0][0])
    a, b = g.ff_a[k], g.ff_b[k]
    (fa, fb, t, u) = g.intersections[0]
    na, nb = g.frac_ns[fa], g.frac_ns[fb]
    sa, sb = min(int(t * na), na - 1), min(int(u * nb), nb - 1)
    La = math.hypot(*(g.seg[fa][2:] - g.seg[fa][:2]))
    Lb = math.hypot(*(g.seg[fb][2:] - g.seg[fb][:2]))
    Ta = 50.0 / max(abs(t - (sa + 0.5) / na) * La, 1e-3)
    Tb = 50.0 / max(abs(u - (sb + 0.5) / nb) * Lb, 1e-3)
    nm, n = s.n_matrix, s.n
    Tab = -s.A[nm + a, nm + b]
    A = s.A.tolil()
    A.resize((n + 1, n + 1))
    for c in (nm + a, nm + b):
        A[c, c] -= Tab
    A[nm + a, nm + b] = 0.0
    A[nm + b, nm + a] = 0.0
    for c, T in ((nm + a, Ta), (nm + b, Tb)):
        A[c, c] += T
        A[c, n] = -T
        A[n, c] = -T
        A[n, n] += T
    y = spla.spsolve(A.tocsc(), np.concatenate([s.q, [0.0]]))
    np.testing.assert_allclose(y[:n], x, rtol=0, atol=1e-12)


def test_3d_plate_connections():
    # a vertical plate spanning layers 1..3 of a 6x6x5 grid, along x at y = 3.5
    p = _prob([[1, 3.5, 5, 3.5, 1.0, 4.0]], nx=6, ny=6, nz=5, dim=3, kf=10.0)
    s = assemble.assemble(p)
    g = s.geom
    assert g.n_frac == 4 * 3
    assert len(g.nnc_f) == 12
    # vertical links carry k_f a_f h_s / dz, strike links k_f a_f dz / h_s
    assert set(g.ff_kind) == {0, 1}
    np.testing.assert_allclose(g.ff_T, 10.0)
    assert abs(s.A - s.A.T).max() == 0.0
