"""The request server (continuous batching) against standalone solves.

Each served result -- pressure, fluxes, iteration count -- must match what
the same problem gives in a context of its own, whatever it was batched
with (to the rounding of the coarse operator's atomic sums: 1e-10 relative),
and a problem the method rejects must fail alone."""
import numpy as np
import pytest

from paper_1705_05784_gb300 import inputs

pytestmark = pytest.mark.gpu


def _mix():
    out = []
    for i in range(10):
        if i % 3 == 2:
            p = inputs.config_3d(16 + 2 * i, 14, 10, 1.0, (5, 5, 2), 3, (5, 10), 1e3, (4, 4, 2), 4,
                                 2, seed=40 + i, basis=i % 4, restriction=1)
            p.fracs[:, 4] = 0.0
            p.fracs[:, 5] = 10.0
        else:
            # R^FV only under GMRES: the FV Table 1 loop need not converge on
            # rough fields (Sec. 3.2)
            p = inputs.config_2d(24 + 8 * i, 1.5, 6.0, 4, (8, 20), 1e4, 4 + i % 3, 5, seed=60 + i,
                                 basis=i % 4, restriction=1 - (i % 4 == 1), alpha=1e-2)
        p.krylov = i % 2
        out.append(p)
    return out


def _alone(fams, p):
    with fams.Context(p) as c:
        xs, st = c.solve(tol=1e-8)
        face, nnc = c.flux(xs[0])
        s = c.sizes()
    assert st[0]["converged"]
    return xs[0], face, nnc, st[0], s


@pytest.mark.parametrize("max_batch,pipelines", [(4, 2), (16, 1), (1, 3)])
def test_served_results_match_standalone_solves(max_batch, pipelines):
    from paper_1705_05784_gb300 import fams
    probs = _mix()
    ref = [_alone(fams, p) for p in probs]
    with fams.Server(max_batch=max_batch, pipelines=pipelines, hbm_budget=8 << 30,
                     tol=1e-8) as srv:
        tickets = [srv.submit(p) for p in probs]
        for t, (x0, f0, n0, s0, sz) in zip(tickets, ref):
            assert srv.wait(t, 120000.0)
            n = sz["n_matrix"] + sz["n_frac"]
            x, face, nnc, st = srv.result(t, n, sz["n_faces"], sz["n_nnc"])
            assert st["status"] == 0 and st["converged"]
            assert st["iterations"] == s0["iterations"]
            assert np.linalg.norm(x - x0) / np.linalg.norm(x0) < 1e-10
            scale = max(np.abs(f0).max(), 1e-300)
            np.testing.assert_allclose(face, f0, rtol=0, atol=1e-9 * scale)
            np.testing.assert_allclose(nnc, n0, rtol=0, atol=1e-9 * scale)
            assert st["latency_ms"] > 0
            srv.release(t)


def test_a_rejected_problem_fails_alone():
    from paper_1705_05784_gb300 import fams
    good = _mix()[:3]
    bad = inputs.config_3d(20, 18, 12, 1.0, (5, 5, 2), 2, (6, 14), 1e3, (5, 6, 4), 5, 4, seed=8)
    # a negative permeability: the device's input check rejects the instance
    # during setup, inside the micro-batch
    bad.perm = bad.perm.copy()
    bad.perm[37] = -1.0
    with fams.Server(max_batch=8, pipelines=1, hbm_budget=8 << 30) as srv:
        tg = [srv.submit(p) for p in good]
        tb = srv.submit(bad)
        for t in tg + [tb]:
            assert srv.wait(t, 120000.0)
        assert srv.status(tb) == fams.EINVAL
        for t in tg:
            assert srv.status(t) == fams.OK


def test_small_budget_still_serves_one_at_a_time():
    from paper_1705_05784_gb300 import fams
    probs = _mix()[:4]
    with fams.Server(max_batch=8, pipelines=2, hbm_budget=1, with_flux=False) as srv:
        ts = [srv.submit(p) for p in probs]
        for t in ts:
            assert srv.wait(t, 120000.0)
            assert srv.status(t) == fams.OK


def _update_alone(fams, p, x_base, scale):
    """The reference of a served time-step update: the base problem's own
    context, fams_update with the scale, solved from the base's pressure."""
    with fams.Context(p) as c:
        c.update([scale])
        xs, st = c.solve(tol=1e-8, x0=[x_base])
        face, nnc = c.flux(xs[0])
    assert st[0]["converged"]
    return xs[0], face, nnc, st[0]


@pytest.mark.parametrize("budget", [8 << 30, 1])
def test_time_step_updates_match_standalone_updates(budget):
    """fams_server_submit_update against a resident setup (budget 8 GiB) and,
    with a budget of 1 byte, after the base's setup was evicted (set up again
    first): each updated result -- pressure, fluxes, iterations -- equals
    fams_update + solve from the base's pressure in a context of its own."""
    from paper_1705_05784_gb300 import fams
    probs = _mix()[:6]
    rng = np.random.default_rng(7)
    with fams.Server(max_batch=4, pipelines=2, hbm_budget=budget, tol=1e-8) as srv:
        base = [srv.submit(p) for p in probs]
        xb = []
        for t in base:
            assert srv.wait(t, 120000.0)
            x, face, nnc, st = srv.fetch(t)
            assert st["status"] == 0
            xb.append(x)
        picks = [0, 2, 3, 3, 5]          # two updates of one base, in one stream
        scales = [rng.uniform(0.5, 2.0, len(xb[i])) for i in picks]
        ups = [srv.submit_update(base[i], sc) for i, sc in zip(picks, scales)]
        for t, i, sc in zip(ups, picks, scales):
            assert srv.wait(t, 120000.0)
            x, face, nnc, st = srv.fetch(t)
            assert st["status"] == 0 and st["converged"], st["error"]
            x0, f0, n0, s0 = _update_alone(fams, probs[i], xb[i], sc)
            assert abs(st["iterations"] - s0["iterations"]) <= 1
            assert np.linalg.norm(x - x0) / np.linalg.norm(x0) < 1e-9
            fs = max(np.abs(f0).max(), 1e-300)
            np.testing.assert_allclose(face, f0, rtol=0, atol=1e-8 * fs)
            np.testing.assert_allclose(nnc, n0, rtol=0, atol=1e-8 * fs)
        # an update whose scale does not match its base fails alone
        bad = srv.submit_update(base[1], np.ones(3))
        assert srv.wait(bad, 60000.0)
        assert srv.status(bad) == fams.EINVAL
        # releasing the base first: its later update fails
        srv.release(base[4])
        late = None
        try:
            late = srv.submit_update(base[4], np.ones(len(xb[4])))
        except fams.FamsError:
            pass                         # unknown ticket at submission
        if late is not None:
            assert srv.wait(late, 60000.0)
            assert srv.status(late) == fams.EINVAL


def test_subset_solve_leaves_the_other_instances_alone():
    """fams_solve_subset: the listed instances are solved exactly as in a
    full batch solve; the others launch nothing and keep their state."""
    from paper_1705_05784_gb300 import fams
    probs = _mix()[:4]
    with fams.Context(probs) as c:
        xs_all, st_all = c.solve(tol=1e-8)
        xs, st = c.solve_subset([3, 1], tol=1e-8)
        for k, i in enumerate([3, 1]):
            assert st[k]["iterations"] == st_all[i]["iterations"]
            assert np.linalg.norm(xs[k] - xs_all[i]) / np.linalg.norm(xs_all[i]) < 1e-12
        with pytest.raises(fams.FamsError):
            c.solve_subset([1, 1])
