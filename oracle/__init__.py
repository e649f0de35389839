"""Plain FP64 CPU oracle of F-AMS (Tene, Al Kobaisi, Hajibeygi; arXiv 1705.05784).

TEST INFRASTRUCTURE ONLY: a slow, obviously-correct statement of the method,
written from the paper, used by the tests, the smoke check and the CPU-baseline
arm of the benchmark to check the CUDA library.  The library never imports,
links or calls anything here, and nothing here imports the library.

Modules:
  geometry  - EDFM fracture cells, matrix-fracture connections, intersections
  assemble  - the fine system A p = q (TPFA + NNC, Dirichlet faces)
  coarsen   - primal/dual coarse grids, wirebasket ranks, Table 2 BFS
  basis     - prolongation P by the staged rule and by Appendix A's formulas,
              truncation
  solver    - R, A_c = R A P, LU, ILU(0), Table 1 iteration, GMRES with the
              two-stage step as preconditioner, flux reconstruction

Parity unpinned: the paper's printed numbers (single-step error norms of
Sec. 4.2, Table 3 timings) depend on permeability maps and fracture networks
that are not published, so no function here is pinned to them.  Every other
function is pinned by the tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import assemble as _asm
from . import basis as _basis
from . import coarsen as _coarsen
from . import geometry as _geom
from . import solver as _solver


@dataclass
class OracleResult:
    geom: object
    sysm: object
    coarse: object
    P: object
    setup: object
    p: np.ndarray
    iters: int
    rel_res: float
    converged: bool
    history: list


def prolongation(prob, g, sysm, c, route="staged", truncated=True):
    """P (truncated unless `truncated` is False) from the basis operator A0 of
    `sysm` (Sec. 3.1, App. A; truncation Sec. 4.3).  Called with an updated
    system it rebuilds the basis functions for new mobilities on the same
    coarse grids."""
    plate = np.concatenate([np.full(g.n_matrix, -1, np.int64), g.cell_frac,
                            np.full(getattr(sysm, "n_well", 0), -1, np.int64)])
    cap = getattr(prob, "merge_cap", 0)
    if route == "staged":
        P = _basis.prolongation_staged(sysm.A0, c.rank, c.medium, c.node_cell, prob.basis, plate,
                                       c.row_net, cap)
    else:
        P = _basis.prolongation_appendix(sysm.A0, c.rank, c.medium, c.node_cell, prob.basis,
                                         plate, c.row_net, cap)
    return _basis.truncate(P, prob.alpha) if truncated else P


def prolongation_update(prob, g, sysm, c, P_full, ref, scale, eps):
    """The adaptive basis update (Sec. 3.1: basis functions are recomputed
    only where the fine-scale properties change beyond a threshold; Table 1
    step 4): a cell is marked when its mobility scale moved by more than a
    factor 1 + eps from `ref`, the scale its basis row was last computed
    with (eps < 0 marks every cell); dual blocks holding a marked cell, and
    the blocks that read rows recomputed in an earlier stage, are solved
    again from the updated operator of `sysm`; the others keep their rows of
    P_full (the untruncated P of the last build).  Returns (P truncated,
    P untruncated, new ref, blocks solved)."""
    scale = np.asarray(scale, np.float64)
    ref = np.asarray(ref, np.float64)
    marked = np.ones(len(scale), bool) if eps < 0 else (
        (scale > (1.0 + eps) * ref) | (scale < ref / (1.0 + eps)))
    plate = np.concatenate([np.full(g.n_matrix, -1, np.int64), g.cell_frac,
                            np.full(getattr(sysm, "n_well", 0), -1, np.int64)])
    Pf, rec, solved = _basis.prolongation_staged(
        sysm.A0, c.rank, c.medium, c.node_cell, prob.basis, plate, c.row_net,
        getattr(prob, "merge_cap", 0), old=P_full, marked=marked)
    ref = np.where(rec, scale, ref)
    return _basis.truncate(Pf, prob.alpha), Pf, ref, solved


def reconstruction_setup(prob, g, sysm, c):
    """The finite-volume coarse system of the flux reconstruction (Sec. 3.2):
    R^FV A P with the basis functions before truncation.  Reading: truncation
    (Sec. 4.3) cuts the iteration's cost, and a truncated basis function can
    lie inside its own primal block, where its column of R^FV A P vanishes and
    the finite-volume stage has no solution; the reconstruction's single stage
    therefore uses the untruncated basis functions."""
    P = prolongation(prob, g, sysm, c, truncated=False)
    return _solver.setup(sysm, P, c.primal, c.n_coarse, _solver.R_FV)


def build(prob, route="staged"):
    """Geometry, system, coarse grids, P (truncated) and the solver setup."""
    g = _geom.build_geometry(prob)
    sysm = _asm.assemble(prob, g)
    c = _coarsen.build_coarse(prob, g)
    P = prolongation(prob, g, sysm, c, route)
    st = _solver.setup(sysm, P, c.primal, c.n_coarse, prob.restriction,
                       c.medium if getattr(prob, "subblock", 0) else None)
    return g, sysm, c, P, st


def run(prob, x0=None, history=True):
    g, sysm, c, P, st = build(prob)
    if getattr(prob, "krylov", 0) == 1:
        p, it, rr, ok, hist = _solver.gmres_solve(st, x0=x0, tol=prob.tol, max_iter=prob.max_iter,
                                                  restart=prob.restart, history=history)
    else:
        p, it, rr, ok, hist = _solver.two_stage_solve(st, x0=x0, tol=prob.tol,
                                                       max_iter=prob.max_iter, history=history)
    return OracleResult(g, sysm, c, P, st, p, it, rr, ok, hist)
