"""Oracle: EDFM geometry (Sec. 2; Eqs. 4-7).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow FP64 CPU statement
of the method that the CUDA path is checked against.  Only the tests, the
package's smoke check and the CPU-baseline arm of the benchmark may import it;
the library never does.

Embedded discrete fractures on a structured matrix grid:

* each (clipped) fracture segment is cut into n = floor(L/h_f + 1/2) equal
  cells (3D: a vertical plate is cut the same way along strike and into the
  matrix layers whose centres lie in [z0, z1));
* each fracture cell is clipped against the matrix cells it crosses; every
  overlap gives one matrix-fracture connection with area A_ij (overlap length
  x depth) and average distance <d>_ij (Eq. 7, CI_ij = A_ij/<d>_ij);
* <d>_ij is the mean distance from the matrix cell to the fracture's line,
  integrated exactly (the cell clipped by the line; a vertical plate gives
  the 2D value in every layer);
* fracture-fracture intersections (Sec. 4.1: an explicit intersection
  pressure with a flux balance) are eliminated exactly: for the two cells that
  meet at the intersection point, T_ab = T_a T_b / (T_a + T_b) with
  T_a = k_f a_f depth / d_a, d_a the distance from the cell centre to the point
  (floored at 1e-3 h_f).

All floating-point expressions that decide an integer (which cell a piece
lies in, how many cells a fracture has) use only correctly rounded IEEE-754
operations (+ - * / sqrt floor), written out in one fixed order so that another IEEE-754 double
implementation without fused multiply-add reproduces them exactly.
"""
from __future__ import annotations

import math

import numpy as np

ZERO_PIECE = 1e-12       # pieces shorter than this x h_f are dropped
DIST_FLOOR = 1e-3        # intersection distance floor, x h_f


def clip_segment(x0, y0, x1, y1, lx, ly):
    """Liang-Barsky clip of a segment to [0,lx] x [0,ly]; None if nothing is left."""
    dx, dy = x1 - x0, y1 - y0
    t0, t1 = 0.0, 1.0
    for p, q in ((-dx, x0), (dx, lx - x0), (-dy, y0), (dy, ly - y0)):
        if p == 0.0:
            if q < 0.0:
                return None
            continue
        r = q / p
        if p < 0.0:
            if r > t1:
                return None
            if r > t0:
                t0 = r
        else:
            if r < t0:
                return None
            if r < t1:
                t1 = r
    ax, ay = x0 + t0 * dx, y0 + t0 * dy
    bx, by = x0 + t1 * dx, y0 + t1 * dy
    return ax, ay, bx, by


def _floor_div(v, h):
    return int(math.floor(v / h))


def _len(ex, ey):
    return math.sqrt(ex * ex + ey * ey)


def piece_overlaps(ax, ay, bx, by, n, s, dx, dy, nx, ny, hf=1.0):
    """Clip fracture cell s (parameter [s/n,(s+1)/n] of segment A->B) against
    the matrix columns.  Returns a list of (ix, iy, length) sorted by column
    index ix + nx iy, pieces in the same column merged."""
    ex, ey = bx - ax, by - ay
    L = _len(ex, ey)
    ts = s / n
    te = (s + 1) / n
    brk = [ts, te]
    xa, xb = ax + ts * ex, ax + te * ex
    ya, yb = ay + ts * ey, ay + te * ey
    if ex != 0.0:
        lo, hi = min(xa, xb), max(xa, xb)
        for i in range(_floor_div(lo, dx), _floor_div(hi, dx) + 2):
            t = (i * dx - ax) / ex
            if ts < t < te:
                brk.append(t)
    if ey != 0.0:
        lo, hi = min(ya, yb), max(ya, yb)
        for j in range(_floor_div(lo, dy), _floor_div(hi, dy) + 2):
            t = (j * dy - ay) / ey
            if ts < t < te:
                brk.append(t)
    brk = sorted(set(brk))
    out = []
    for k in range(len(brk) - 1):
        t0, t1 = brk[k], brk[k + 1]
        ln = (t1 - t0) * L
        if ln < ZERO_PIECE * hf:
            continue
        tm = 0.5 * (t0 + t1)
        px = ax + tm * ex
        py = ay + tm * ey
        ix = min(max(_floor_div(px, dx), 0), nx - 1)
        iy = min(max(_floor_div(py, dy), 0), ny - 1)
        out.append((ix, iy, ln))
    # one connection per matrix column: pieces in the same column are summed
    # (in the order they lie along the fracture), then sorted by column index
    merged = {}
    for ix, iy, ln in out:
        key = ix + nx * iy
        merged[key] = (ix, iy, merged[key][2] + ln) if key in merged else (ix, iy, ln)
    return [merged[k] for k in sorted(merged)]


def mean_distance(ax, ay, bx, by, ix, iy, dx, dy):
    """<d> (Eq. 7): mean distance from matrix cell (ix, iy) to the infinite
    line through A, B.

    The signed distance f(x) = n . (x - A) is linear, so its integral over a
    triangle is the area times the mean of f at the three corners.  With P+
    the part of the cell where f >= 0 (the cell rectangle clipped by that
    half-plane, a convex polygon), int_cell |f| = 2 int_{P+} f - int_cell f,
    and int_cell f = area * f(centre).  Coordinates are taken relative to the
    cell's lower-left corner."""
    ex, ey = bx - ax, by - ay
    L = _len(ex, ey)
    nx, ny = -ey / L, ex / L
    x0, y0 = ix * dx, iy * dy
    ox, oy = ax - x0, ay - y0          # A relative to the corner

    def f(x, y):
        return nx * (x - ox) + ny * (y - oy)

    rect = [(0.0, 0.0), (dx, 0.0), (dx, dy), (0.0, dy)]
    poly = []
    for k in range(4):                 # clip by f >= 0 (Sutherland-Hodgman)
        p, q = rect[k], rect[(k + 1) % 4]
        fp, fq = f(*p), f(*q)
        if fp >= 0.0:
            poly.append(p)
        if (fp >= 0.0) != (fq >= 0.0):
            t = fp / (fp - fq)
            poly.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    pos = 0.0                          # int over P+ of f, by a fan of triangles
    for k in range(1, len(poly) - 1):
        (x1, y1), (x2, y2), (x3, y3) = poly[0], poly[k], poly[k + 1]
        area = 0.5 * ((x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1))
        pos += area * (f(x1, y1) + f(x2, y2) + f(x3, y3)) / 3.0
    A = dx * dy
    return float((2.0 * pos - A * f(0.5 * dx, 0.5 * dy)) / A)


class Geometry:
    """Discretised fractures and their connections for one problem.

    Attributes (all numpy):
      n_matrix, n_frac
      frac_first[f], frac_ns[f], frac_k0[f], frac_nk[f]  per input fracture
      seg[f] = (ax, ay, bx, by) clipped segment (nan if empty)
      cell_frac[c], cell_s[c], cell_k[c]                 per fracture cell (local index)
      nnc_f, nnc_m, nnc_area, nnc_dist                   matrix-fracture connections,
                                                         sorted by (fracture cell, matrix cell)
      ff_a, ff_b, ff_T, ff_kind                          fracture-fracture connections a<b
                                                         (kind 0 along strike, 1 vertical,
                                                         2 intersection)
      strike_* : the x-y projection graph used by the coarsening (Sec. 4.3)
    """


def build_geometry(prob):
    dim = prob.dim
    nx, ny = prob.nx, prob.ny
    nz = prob.nz if dim == 3 else 1
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    lx, ly = nx * dx, ny * dy
    hf = prob.h_f
    af = prob.aperture
    fr = np.zeros((0, 6 if dim == 3 else 4)) if prob.fracs is None else np.asarray(prob.fracs, float)
    kf = np.zeros(0) if prob.kf is None else np.asarray(prob.kf, float)
    nf = len(fr)
    g = Geometry()
    g.dim = dim
    g.n_matrix = nx * ny * nz
    g.seg = np.full((nf, 4), np.nan)
    g.frac_first = np.zeros(nf, np.int64)
    g.frac_ns = np.zeros(nf, np.int64)
    g.frac_k0 = np.zeros(nf, np.int64)
    g.frac_nk = np.zeros(nf, np.int64)
    g.frac_kf = kf.copy()
    first = 0
    for f in range(nf):
        c = clip_segment(fr[f, 0], fr[f, 1], fr[f, 2], fr[f, 3], lx, ly)
        ns = 0
        if c is not None:
            L = _len(c[2] - c[0], c[3] - c[1])
            if L >= ZERO_PIECE * hf:
                ns = max(1, int(math.floor(L / hf + 0.5)))
                g.seg[f] = c
        k0, nk = 0, 1
        if dim == 3:
            # layers whose centre (k+1/2) dz lies in [z0, z1)
            z0, z1 = fr[f, 4], fr[f, 5]
            ks = [k for k in range(nz) if z0 <= (k + 0.5) * dz < z1]
            if ks:
                k0, nk = ks[0], len(ks)
            else:
                ns = 0
        if ns == 0:
            nk = 0 if dim == 3 else 1
        g.frac_first[f] = first
        g.frac_ns[f] = ns
        g.frac_k0[f] = k0
        g.frac_nk[f] = nk if ns else 0
        first += ns * (nk if ns else 0) if dim == 3 else ns
    g.n_frac = first
    g.cell_frac = np.zeros(first, np.int64)
    g.cell_s = np.zeros(first, np.int64)
    g.cell_k = np.zeros(first, np.int64)
    for f in range(nf):
        ns, nk = g.frac_ns[f], (g.frac_nk[f] if dim == 3 else 1)
        for kk in range(nk):
            for s in range(ns):
                c = g.frac_first[f] + s + ns * kk
                g.cell_frac[c] = f
                g.cell_s[c] = s
                g.cell_k[c] = g.frac_k0[f] + kk if dim == 3 else 0
    depth = dz  # 2D: unit-thickness slab of thickness dz; 3D: layer height

    # --- matrix-fracture connections (Eqs. 4-7) ---
    nnc = []
    for f in range(nf):
        ns = g.frac_ns[f]
        if ns == 0:
            continue
        ax, ay, bx, by = g.seg[f]
        for s in range(ns):
            ov = piece_overlaps(ax, ay, bx, by, ns, s, dx, dy, nx, ny, hf)
            for (ix, iy, ln) in ov:
                dmean = mean_distance(ax, ay, bx, by, ix, iy, dx, dy)
                if dim == 2:
                    nnc.append((g.frac_first[f] + s, ix + nx * iy, ln * depth, dmean))
                else:
                    for kk in range(g.frac_nk[f]):
                        k = g.frac_k0[f] + kk
                        nnc.append((g.frac_first[f] + s + ns * kk,
                                    ix + nx * (iy + ny * k), ln * depth, dmean))
    nnc.sort(key=lambda t: (t[0], t[1]))
    g.nnc_f = np.array([t[0] for t in nnc], np.int64)
    g.nnc_m = np.array([t[1] for t in nnc], np.int64)
    g.nnc_area = np.array([t[2] for t in nnc], np.float64)
    g.nnc_dist = np.array([t[3] for t in nnc], np.float64)

    # --- fracture-fracture connections ---
    ff = []
    for f in range(nf):
        ns = g.frac_ns[f]
        if ns == 0:
            continue
        ax, ay, bx, by = g.seg[f]
        h = _len(bx - ax, by - ay) / ns
        nk = g.frac_nk[f] if dim == 3 else 1
        for kk in range(nk):
            for s in range(ns - 1):
                a = g.frac_first[f] + s + ns * kk
                ff.append((a, a + 1, kf[f] * af * depth / h, 0))
            if dim == 3 and kk + 1 < nk:
                for s in range(ns):
                    a = g.frac_first[f] + s + ns * kk
                    ff.append((a, a + ns, kf[f] * af * h / dz, 1))
    inter = []
    for fa in range(nf):
        if g.frac_ns[fa] == 0:
            continue
        for fb in range(fa + 1, nf):
            if g.frac_ns[fb] == 0:
                continue
            hit = segment_intersection(g.seg[fa], g.seg[fb])
            if hit is None:
                continue
            t, u = hit
            inter.append((fa, fb, t, u))
            na, nb = g.frac_ns[fa], g.frac_ns[fb]
            sa = min(int(math.floor(t * na)), na - 1)
            sb = min(int(math.floor(u * nb)), nb - 1)
            La = _len(g.seg[fa][2] - g.seg[fa][0], g.seg[fa][3] - g.seg[fa][1])
            Lb = _len(g.seg[fb][2] - g.seg[fb][0], g.seg[fb][3] - g.seg[fb][1])
            da = max(abs(t - (sa + 0.5) / na) * La, DIST_FLOOR * hf)
            db = max(abs(u - (sb + 0.5) / nb) * Lb, DIST_FLOOR * hf)
            Ta = kf[fa] * af * depth / da
            Tb = kf[fb] * af * depth / db
            Tab = Ta * Tb / (Ta + Tb)
            if dim == 2:
                ff.append((g.frac_first[fa] + sa, g.frac_first[fb] + sb, Tab, 2))
            else:
                lo = max(g.frac_k0[fa], g.frac_k0[fb])
                hi = min(g.frac_k0[fa] + g.frac_nk[fa], g.frac_k0[fb] + g.frac_nk[fb])
                for k in range(lo, hi):
                    ca = g.frac_first[fa] + sa + na * (k - g.frac_k0[fa])
                    cb = g.frac_first[fb] + sb + nb * (k - g.frac_k0[fb])
                    ff.append((ca, cb, Tab, 2))
    g.intersections = inter
    ff = [(min(a, b), max(a, b), T, kd) for (a, b, T, kd) in ff]
    ff.sort(key=lambda t: (t[0], t[1], t[3]))
    g.ff_a = np.array([t[0] for t in ff], np.int64)
    g.ff_b = np.array([t[1] for t in ff], np.int64)
    g.ff_T = np.array([t[2] for t in ff], np.float64)
    g.ff_kind = np.array([t[3] for t in ff], np.int64)

    # --- the x-y projection ("strike") graph used by the fracture coarsening:
    # along-strike neighbours, and the crossing cells of two fractures (in 3D
    # of two plates with the same layer range) ---
    n_strike = int(g.frac_ns.sum())
    g.n_strike = n_strike
    sfirst = np.concatenate([[0], np.cumsum(g.frac_ns)[:-1]]) if nf else np.zeros(0, np.int64)
    g.strike_first = sfirst.astype(np.int64)
    adj = [set() for _ in range(n_strike)]
    for f in range(nf):
        for s in range(g.frac_ns[f] - 1):
            a = sfirst[f] + s
            adj[a].add(a + 1)
            adj[a + 1].add(a)
    for (fa, fb, t, u) in inter:
        na, nb = g.frac_ns[fa], g.frac_ns[fb]
        sa = min(int(math.floor(t * na)), na - 1)
        sb = min(int(math.floor(u * nb)), nb - 1)
        if dim == 3:
            # plates are coarsened together only where they share their layer
            # range (uniform vertical extrusion of the network, Sec. 4.3);
            # crossing plates of other ranges stay connected in A
            if g.frac_k0[fa] != g.frac_k0[fb] or g.frac_nk[fa] != g.frac_nk[fb]:
                continue
            if g.frac_nk[fa] <= 0:
                continue
        a, b = sfirst[fa] + sa, sfirst[fb] + sb
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    g.strike_adj = [sorted(s) for s in adj]
    return g


def segment_intersection(sa, sb):
    """Parameters (t,u) of the crossing of two closed segments, None if they miss
    or are parallel."""
    ax, ay, bx, by = sa
    cx, cy, ex, ey = sb
    d1x, d1y = bx - ax, by - ay
    d2x, d2y = ex - cx, ey - cy
    den = d1x * d2y - d1y * d2x
    n1 = _len(d1x, d1y)
    n2 = _len(d2x, d2y)
    if abs(den) <= 1e-14 * n1 * n2:
        return None
    wx, wy = cx - ax, cy - ay
    t = (wx * d2y - wy * d2x) / den
    u = (wx * d1y - wy * d1x) / den
    if 0.0 <= t <= 1.0 and 0.0 <= u <= 1.0:
        return t, u
    return None
