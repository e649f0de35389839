"""Seeded synthetic inputs shaped like the paper's 2D and 3D test cases.

This module only draws random numbers and lays out arrays: grids, log10
permeability fields and fracture geometry.  It holds none of the method's
arithmetic, so the CPU oracle tests and the CUDA path can both consume its
output without sharing any code of the method.

The paper's own permeability maps and fracture networks (Sec. 4, Figs. 8, 11,
16) are not available, so these generators stand in for them:

* log10 k: a stationary Gaussian field with exponential covariance, drawn by
  circulant embedding (FFT) on a padded torus, mean 0 so that the geometric mean
  of k is 1;
* 2D fractures: straight segments with uniform centre, length and angle;
* 3D fractures: vertical rectangular plates (a segment in the x-y plane and a
  layer range), the geometry class of the paper's 3D experiments (Sec. 4.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# face bits of the Dirichlet mask: west, east, south, north, bottom, top
BC_WEST, BC_EAST, BC_SOUTH, BC_NORTH, BC_BOTTOM, BC_TOP = 1, 2, 4, 8, 16, 32


WELL_RATE, WELL_PRESSURE = 0, 1


@dataclass
class Well:
    """A vertical (or any) well: the matrix cells it perforates, the geometric
    productivity index of each perforation, and its control: a total
    injection rate (the well pressure is an unknown) or a bottom-hole
    pressure."""
    cells: np.ndarray
    pi: np.ndarray
    control: int = WELL_RATE
    value: float = 0.0


@dataclass
class Problem:
    """One F-AMS problem instance (all arrays host numpy, float64 / int32)."""
    dim: int
    nx: int
    ny: int
    nz: int
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    bc_mask: int = BC_WEST | BC_EAST
    bc_value: tuple = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    perm: np.ndarray = None          # (n_matrix,), x fastest
    fracs: np.ndarray = None         # 2D: (n,4) x0,y0,x1,y1 ; 3D: (n,6) x0,y0,x1,y1,z0,z1
    kf: np.ndarray = None            # (n,) fracture permeability per fracture
    aperture: float = 1.0
    h_f: float = 1.0
    # method options
    coarsen: tuple = (4, 4, 1)
    frac_dmin: int = 5
    frac_cz: int = 1
    basis: int = 0                   # 0 Decoupled, 1 Frac, 2 Rock, 3 Coupled
    restriction: int = 0             # 0 FV, 1 FE, 2 MSMIX
    alpha: float = 0.0
    merge_cap: int = 0               # Coupled: largest block merged across the media (0: none)
    grid_solve: int = 0              # single instance on every SM: 0 auto (>= 2^18 unknowns), 1, -1
    subblock: int = 0                # 1: the sub-block smoothing stage after ILU(0)
    bf16_p: int = 0                  # mixed precision: P and P^T values stored in BF16
    coarse_mode: int = 0             # whole-GPU coarse solve: 0 auto, 1 A_c^-1, 2 band factors
    tol: float = 1e-8
    max_iter: int = 200
    krylov: int = 0                  # 0 the Table 1 loop, 1 GMRES(restart)
    restart: int = 30
    prepare_flux: int = 0            # 1: build the reconstruction's coarse system beside the solve
    precision: int = 0               # 0 FP64, 1 FP32 inner stages
    rhs: np.ndarray = None           # sources, length N (matrix then fracture); None = 0
    wells: list = None               # Well objects (None: no wells)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_matrix(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)


def gaussian_field(shape, sigma, corr, seed, mean=0.0):
    """Stationary Gaussian field with covariance sigma^2 exp(-|h/corr|) on a grid.

    shape: tuple of cell counts (x fastest in the returned flat array).
    corr: scalar or per-axis correlation length in cells.
    Circulant embedding on a torus twice the size; negative eigenvalues (rare
    for this covariance) are clipped to zero.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    corr = np.broadcast_to(np.asarray(corr, dtype=np.float64), (d,))
    big = tuple(2 * s for s in shape)
    axes = []
    for s, l in zip(big, corr):
        h = np.arange(s, dtype=np.float64)
        h = np.minimum(h, s - h)
        axes.append(h / max(l, 1e-12))
    mesh = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(sum(m * m for m in mesh))
    cov = sigma * sigma * np.exp(-r)
    lam = np.fft.fftn(cov).real
    lam = np.maximum(lam, 0.0)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(big) + 1j * rng.standard_normal(big)
    f = np.fft.ifftn(np.sqrt(lam) * noise) * math.sqrt(np.prod(big))
    sl = tuple(slice(0, s) for s in shape)
    out = f.real[sl] + mean
    # shape is (nx, ny[, nz]) in ij indexing -> flatten with x fastest
    return np.ascontiguousarray(out.transpose(tuple(range(d))[::-1])).reshape(-1)


def random_segments(n, domain, length_range, seed, angle_range=(0.0, 180.0)):
    """n straight 2D segments: uniform centre in the domain, uniform length and angle."""
    rng = np.random.default_rng(seed)
    lx, ly = domain
    cx = rng.uniform(0.0, lx, n)
    cy = rng.uniform(0.0, ly, n)
    ln = rng.uniform(length_range[0], length_range[1], n)
    th = np.deg2rad(rng.uniform(angle_range[0], angle_range[1], n))
    hx, hy = 0.5 * ln * np.cos(th), 0.5 * ln * np.sin(th)
    return np.stack([cx - hx, cy - hy, cx + hx, cy + hy], axis=1)


def random_plates(n, domain, side_range, nz, seed):
    """n vertical rectangular plates: strike segment and a layer range [z0, z1)."""
    rng = np.random.default_rng(seed)
    lx, ly = domain
    seg = random_segments(n, domain, side_range, seed + 7919)
    h = rng.integers(int(side_range[0]), int(side_range[1]) + 1, n)
    h = np.minimum(h, nz)
    z0 = rng.integers(0, np.maximum(nz - h, 0) + 1)
    return np.concatenate([seg, z0[:, None].astype(np.float64),
                           (z0 + h)[:, None].astype(np.float64)], axis=1)


def config_2d_small(seed=1, basis=0, restriction=0):
    """32x32 cells, sigma 1, corr 4; one 20-cell fracture at 30 deg through the centre,
    k_f = 1e4 x geometric mean k_m; Dirichlet W=1/E=0; coarsening 4x4, d_min 5."""
    nx = ny = 32
    perm = 10.0 ** gaussian_field((nx, ny), 1.0, 4.0, seed)
    th = math.radians(30.0)
    c = (16.0, 16.0)
    hl = 10.0
    fr = np.array([[c[0] - hl * math.cos(th), c[1] - hl * math.sin(th),
                    c[0] + hl * math.cos(th), c[1] + hl * math.sin(th)]])
    return Problem(dim=2, nx=nx, ny=ny, nz=1, perm=perm, fracs=fr, kf=np.array([1e4]),
                   coarsen=(4, 4, 1), frac_dmin=5, basis=basis, restriction=restriction,
                   alpha=0.0, name="2d-32x32-1frac")


def config_2d_sealed_node(basis=0, restriction=1, factor=1e-10):
    """config_2d_small with truncation (alpha 1e-2) and the cell at (22, 6), the
    coarse node of primal block (5, 1), `factor` times as permeable as before."""
    p = config_2d_small(basis=basis, restriction=restriction)
    p.perm = p.perm.copy()
    p.perm[22 + 32 * 6] *= factor
    p.alpha = 1e-2
    p.name = "2d-32x32-sealed-node"
    return p


def config_2d_256(seed=2, tratio=1e4, basis=0, restriction=0, n_fracs=30, alpha=0.0):
    """256x256 cells, sigma 2, corr 16; 30 random fractures, length U[20,120],
    angle U[0,180); k_f = tratio (geometric mean k_m = 1); coarsening 8x8, d_min 8."""
    nx = ny = 256
    perm = 10.0 ** gaussian_field((nx, ny), 2.0, 16.0, seed)
    fr = random_segments(n_fracs, (nx, ny), (20.0, 120.0), seed + 1000)
    return Problem(dim=2, nx=nx, ny=ny, nz=1, perm=perm, fracs=fr,
                   kf=np.full(n_fracs, float(tratio)), coarsen=(8, 8, 1), frac_dmin=8,
                   basis=basis, restriction=restriction, alpha=alpha,
                   name=f"2d-256x256-{n_fracs}frac-T{tratio:g}")


def config_2d(n, sigma, corr, n_fracs, flen, tratio, coarsen, dmin, seed, basis=0,
              restriction=0, alpha=0.0, **solver_opts):
    """Generic 2D instance of the same family at any size (tests use small ones);
    solver_opts sets further Problem fields (krylov, restart, precision, ...)."""
    perm = 10.0 ** gaussian_field((n, n), sigma, corr, seed)
    fr = random_segments(n_fracs, (n, n), flen, seed + 1000) if n_fracs else np.zeros((0, 4))
    return Problem(dim=2, nx=n, ny=n, nz=1, perm=perm, fracs=fr,
                   kf=np.full(len(fr), float(tratio)), coarsen=(coarsen, coarsen, 1),
                   frac_dmin=dmin, basis=basis, restriction=restriction, alpha=alpha,
                   name=f"2d-{n}-{n_fracs}frac-s{seed}", **solver_opts)


def config_3d(nx, ny, nz, sigma, corr, n_plates, side, tratio, coarsen, dmin, cz, seed,
              basis=0, restriction=0, alpha=0.0):
    """3D instance: layered log10 k field and vertical plates with random layer ranges."""
    perm = 10.0 ** gaussian_field((nx, ny, nz), sigma, corr, seed)
    fr = (random_plates(n_plates, (nx, ny), side, nz, seed + 1000) if n_plates
          else np.zeros((0, 6)))
    return Problem(dim=3, nx=nx, ny=ny, nz=nz, perm=perm, fracs=fr,
                   kf=np.full(len(fr), float(tratio)), coarsen=tuple(coarsen),
                   frac_dmin=dmin, frac_cz=cz, basis=basis, restriction=restriction,
                   alpha=alpha, name=f"3d-{nx}x{ny}x{nz}-{n_plates}pl-s{seed}")


def column_well(nx, ny, nz, ix, iy, pi, control, value, k0=0, k1=None):
    """A vertical well through the matrix column (ix, iy), layers k0..k1-1
    (all layers by default), the same productivity index per perforation."""
    k1 = nz if k1 is None else k1
    cells = np.array([ix + nx * (iy + ny * k) for k in range(k0, k1)], np.int64)
    return Well(cells=cells, pi=np.full(len(cells), float(pi)), control=control, value=value)
