"""fams_solve_static (the allocation-free solve) against fams_solve.

The library's fixed work array keeps the previous call's contents, so the
entry point is called twice in a row, on two instances of different size and
then again on the first one; each result must match the allocating entry
point's on the same context to the tolerance of the trajectory tests (same
iteration count, 1e-10 relative L2).  The file is named to be collected last
and must pass alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1705_05784_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problems():
    a = inputs.config_2d_small(basis=3, restriction=1)
    b = inputs.config_2d(64, 1.5, 8.0, 6, (15, 45), 1e3, 8, 8, seed=4, basis=1, restriction=1)
    return a, b


def _agree(xs, ss, xr, sr):
    assert ss["iterations"] == sr["iterations"]
    assert ss["converged"] == sr["converged"]
    assert abs(ss["rel_residual"] - sr["rel_residual"]) <= 1e-10 * sr["rel_residual"] + 1e-15
    assert np.linalg.norm(xs - xr) / np.linalg.norm(xr) <= 1e-10


def test_static_matches_solve_on_consecutive_calls():
    from paper_1705_05784_gb300 import fams
    pa, pb = _problems()
    with fams.Context(pa) as ca, fams.Context(pb) as cb:
        na = ca.sizes()["n_matrix"] + ca.sizes()["n_frac"]
        rhs = np.random.default_rng(5).standard_normal(na) * 1e-3
        ref_a = ca.solve(rhs=rhs, tol=1e-8)
        ref_b = cb.solve(tol=1e-8)
        # three calls in a row through the shared array: a, b (larger), a
        # again; none of them allocates device memory
        n_alloc = fams.alloc_count()
        xa1, sa1 = ca.solve_static(rhs=rhs, tol=1e-8)
        _agree(xa1, sa1, ref_a[0][0], ref_a[1][0])
        xb, sb = cb.solve_static(tol=1e-8)
        _agree(xb, sb, ref_b[0][0], ref_b[1][0])
        xa2, sa2 = ca.solve_static(rhs=rhs, tol=1e-8)
        _agree(xa2, sa2, ref_a[0][0], ref_a[1][0])
        assert sa1["converged"] and sb["converged"]
        assert fams.alloc_count() == n_alloc
        # a setup allocates (the counter counts)
        with fams.Context(pa):
            pass
        assert fams.alloc_count() > n_alloc


def test_static_from_a_warm_start_and_device_buffers():
    """Device-resident x and rhs, and a nonzero initial guess, twice in a row."""
    import torch
    from paper_1705_05784_gb300 import fams
    pa, _ = _problems()
    with fams.Context(pa) as ca:
        n = ca.sizes()["n_matrix"] + ca.sizes()["n_frac"]
        rng = np.random.default_rng(9)
        x0 = rng.uniform(0.0, 1.0, n)
        rhs = rng.standard_normal(n) * 1e-3
        ref = ca.solve(rhs=rhs, x0=x0, tol=1e-9)
        for _ in range(2):
            xd = torch.tensor(x0, dtype=torch.float64, device="cuda")
            rd = torch.tensor(rhs, dtype=torch.float64, device="cuda")
            st = fams.fams_stats()
            s = fams.lib.fams_solve_static(ca.h, fams.C.c_void_p(rd.data_ptr()),
                                           fams.C.c_void_p(xd.data_ptr()), 1e-9,
                                           fams.C.byref(st))
            assert s == fams.OK
            got = dict(iterations=st.iterations, rel_residual=st.rel_residual,
                       converged=bool(st.converged))
            _agree(xd.cpu().numpy(), got, ref[0][0], ref[1][0])


def test_static_rejects_batch_and_oversize():
    from paper_1705_05784_gb300 import fams
    pa, pb = _problems()
    with fams.Context([pa, pb]) as cab:
        x = np.zeros(10)
        s = fams.lib.fams_solve_static(cab.h, None, x.ctypes.data_as(fams.C.c_void_p), 1e-8, None)
        assert s == fams.EINVAL
    big = inputs.config_2d_small(basis=0, restriction=1)
    big.max_iter = 20000
    with fams.Context(big) as cbig:
        n = cbig.sizes()["n_matrix"] + cbig.sizes()["n_frac"]
        x = np.zeros(n)
        s = fams.lib.fams_solve_static(cbig.h, None, x.ctypes.data_as(fams.C.c_void_p), 1e-8, None)
        assert s == fams.ECAPACITY
        assert b"max_iter" in fams.lib.fams_last_error()


def _line(n, cx):
    """A one-row 2D grid of n cells, coarsening cx along it (cheap to set up
    at the sizes of the static limits)."""
    perm = 10.0 ** inputs.gaussian_field((n, 1), 1.0, 8.0, 11)
    return inputs.Problem(dim=2, nx=n, ny=1, nz=1, perm=perm, fracs=np.zeros((0, 4)),
                          kf=np.zeros(0), coarsen=(cx, 1, 1), frac_dmin=5, basis=0,
                          restriction=1, alpha=0.0)


def test_static_rejects_instances_above_its_limits():
    """One unknown above FAMS_STATIC_MAX_ROWS, and one coarse unknown above
    FAMS_STATIC_MAX_COARSE: FAMS_ECAPACITY with the limit named, nothing run."""
    from paper_1705_05784_gb300 import fams
    cases = [(_line(262144 + 1, 64), b"unknowns; fams_solve_static holds at most 262144"),
             (_line(2 * 16384 + 2, 2), b"coarse unknowns; fams_solve_static holds at most 16384")]
    for p, msg in cases:
        with fams.Context(p) as c:
            S = c.sizes()
            assert (S["n_matrix"] > 262144) == (b"at most 262144" in msg)
            x = np.zeros(S["n_matrix"] + S["n_frac"])
            n_launch = fams.launch_count()
            s = fams.lib.fams_solve_static(c.h, None, x.ctypes.data_as(fams.C.c_void_p), 1e-8,
                                           None)
            assert s == fams.ECAPACITY
            assert msg in fams.lib.fams_last_error()
            assert fams.launch_count() == n_launch


def test_static_reports_a_singular_coarse_system_like_the_solve():
    """A node cell sealed to 1e-300 makes R^FV A P singular: fams_solve_static
    returns FAMS_EBREAKDOWN (the binding hands back the status, as for the
    batch solve) and fams_solve reports the same."""
    from paper_1705_05784_gb300 import fams
    p = inputs.config_2d_sealed_node(restriction=0, factor=1e-300)
    with fams.Context(p) as c:
        x, st = c.solve_static(tol=1e-8)
        assert st["status"] == fams.EBREAKDOWN
        with pytest.raises(fams.FamsError) as e:
            c.solve(tol=1e-8)
        assert e.value.status == fams.EBREAKDOWN
