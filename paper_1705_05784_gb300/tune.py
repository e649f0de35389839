"""Autotuner of the solve schedule of a workload.

For a list of problems (one batch context), times setup + solve to tol +
flux reconstruction under each candidate schedule -- the arithmetic of the
two-stage step (FP64; FP32 restriction, prolongation and ILU(0) sweeps; the
same with P stored in BF16) and the GMRES restart length -- and returns the
fastest with the whole table.  Every candidate is held to the same FP64
residual, so the choice trades only time.  Results can be kept in a JSON
cache keyed by a signature of the workload (sizes and options), so that a
server or a time-step loop tunes once per kind of problem.

Timing is host wall time around the library calls after one untimed run of
each candidate (module loading, pool warm-up); buffers live in host memory
and are reused across runs.
"""
from __future__ import annotations

import copy
import hashlib
import json
import os
import time

import numpy as np

from . import fams

# (name, precision, bf16_p) x restart
PRECISION_VARIANTS = (("fp64", fams.FP64, 0), ("mixed", fams.MIXED, 0),
                      ("mixed_bf16p", fams.MIXED, 1))
RESTARTS = (20, 30, 40)


def signature(problems):
    """Workload key: grid sizes, fracture counts and solver options of every
    instance (not the permeability values)."""
    h = hashlib.sha1()
    for p in problems:
        h.update(json.dumps([p.dim, p.nx, p.ny, p.nz, len(p.fracs), list(p.coarsen), p.frac_dmin,
                             p.basis, p.restriction, p.alpha, getattr(p, "krylov", 0),
                             getattr(p, "merge_cap", 0)]).encode())
    return h.hexdigest()[:16]


def candidates(restarts=RESTARTS, variants=PRECISION_VARIANTS):
    return [{"precision": name, "restart": m} for name, _, _ in variants for m in restarts]


def _apply(problems, cand):
    name = cand["precision"]
    prec, bf = next((p, b) for n, p, b in PRECISION_VARIANTS if n == name)
    out = []
    for p in problems:
        q = copy.copy(p)
        q.precision, q.bf16_p = prec, bf
        q.krylov, q.restart = fams.KRYLOV_GMRES, cand["restart"]
        q.prepare_flux = 1
        out.append(q)
    return out


def _run(problems, tol, bufs):
    with fams.Context(problems) as c:
        for x in bufs["x"]:
            x[:] = 0.0
        st = c.solve_device([None] * len(problems), [x.ctypes.data for x in bufs["x"]], tol)
        fl = c.flux_batch_ptr([x.ctypes.data for x in bufs["x"]],
                              [f.ctypes.data for f in bufs["f"]],
                              [m.ctypes.data for m in bufs["n"]])
    return st, fl


def tune(problems, tol=1e-8, cands=None, reps=1, cache=None):
    """Time every candidate schedule on `problems`; returns (best candidate,
    table of measurements).  cache: path of a JSON file (read first when it
    holds this workload's signature, written after tuning), or None."""
    key = signature(problems)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            known = json.load(f)
        if key in known:
            return known[key]["best"], known[key]["table"]
    cands = cands or candidates()
    with fams.Context(problems) as c:
        sz = [c.sizes(i) for i in range(len(problems))]
    bufs = {"x": [np.zeros(s["n"]) for s in sz],
            "f": [np.zeros(max(s["n_faces"], 1)) for s in sz],
            "n": [np.zeros(max(s["n_nnc"], 1)) for s in sz]}
    table = []
    for cand in cands:
        probs = _apply(problems, cand)
        _run(probs, tol, bufs)                       # untimed
        t = time.perf_counter()
        for _ in range(reps):
            st, fl = _run(probs, tol, bufs)
        sec = (time.perf_counter() - t) / reps
        ok = sum(1 for s, f in zip(st, fl) if s["converged"] and f == 0)
        its = [s["iterations"] for s in st]
        table.append(dict(cand, solves_per_s=ok / sec, seconds=sec, converged=ok,
                          of=len(problems), kernel_ms=st[0]["solve_ms"],
                          iterations_median=float(np.median(its)), iterations_max=int(max(its))))
    full = [r for r in table if r["converged"] == r["of"]] or table
    best = max(full, key=lambda r: r["solves_per_s"])
    best = {"precision": best["precision"], "restart": best["restart"]}
    if cache:
        known = {}
        if os.path.exists(cache):
            with open(cache) as f:
                known = json.load(f)
        known[key] = {"best": best, "table": table}
        with open(cache, "w") as f:
            json.dump(known, f, indent=1)
    return best, table


def apply(problems, best):
    """The problems with the tuned schedule set."""
    return _apply(problems, best)
