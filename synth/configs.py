"""The synthetic workloads of the transport sweep, each scalable down for tests.

Every problem is seeded and synthetic; the recipes stand in for the paper's physics
test set-ups (which need chemistry and hydrodynamics) at the sizes the benchmark uses:

  plain32   32^3 lattice Voronoi mesh, vacuum, kappa*h = 0.1, unit source at cell (16,16,16),
            16 Fibonacci directions (rotation seed 0), 1 group
  column    n cube cells along +x, one direction +x with weight 4pi, unit inflow at x = 0
  batched   64 Poisson-Voronoi meshes (sizes log-uniform in [2^12, 2^17], 2^22 cells in all),
            lognormal density (P(k) ~ k^-3, sigma_ln = 1), kappa ~ rho, 8 sources per mesh ~ mass,
            128 directions, 2 groups
  scatter   2^20 cells with generators ~ rho, albedo 0.5, 64 sources, 96 directions, 4 groups
  periodic  2^22 cells with generators ~ rho (P(k) ~ k^-2.5, sigma_ln = 1.5), periodic box,
            10^4 sources with log-uniform emissivity over 4 decades, 128 directions, 1 group
  adjoint   2^18 Poisson cells, lognormal kappa, 32 sources, 64 directions, 2 groups
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import fields as F
from .mesh import Mesh, column_mesh, concat_meshes, lattice_mesh, voronoi_mesh


@dataclass
class Problem:
    name: str
    mesh: Mesh
    omega: np.ndarray
    weight: np.ndarray
    kappa_abs: np.ndarray
    emissivity: np.ndarray
    kappa_scat: np.ndarray | None = None
    boundary_inflow: np.ndarray | None = None
    tol_scat: float = 1e-6
    tol_pbc: float = 1e-6
    max_it: int = 100
    info: dict = field(default_factory=dict)

    @property
    def n_groups(self) -> int:
        return self.kappa_abs.shape[1]

    @property
    def n_dir(self) -> int:
        return self.omega.shape[0]


def plain32(n: int = 32, n_dir: int = 16) -> Problem:
    m = lattice_mesh(n)
    h = 1.0 / n
    kap = np.full((m.n_cells, 1), 0.1 / h)
    c = n // 2
    eps = np.zeros((m.n_cells, 1))
    eps[c + n * (c + n * c), 0] = 1.0
    om, w = F.fibonacci_directions(n_dir, seed=0)
    return Problem("plain%d" % n, m, om, w, kap, eps, info={"source_cell": c + n * (c + n * c)})


def column(n: int = 256, kappa: float = 3.2, h: float = 1.0 / 256, source: float = 0.0,
           reverse: bool = False) -> Problem:
    m = column_mesh(n, h)
    nb = int(np.count_nonzero(m.flags & 1))
    bc = np.zeros((nb, 1))
    bc[1 if reverse else 0, 0] = 1.0
    om = np.array([[-1.0 if reverse else 1.0, 0.0, 0.0]])
    return Problem("column", m, om, np.array([4 * math.pi]), np.full((n, 1), kappa), np.full((n, 1), source),
                   boundary_inflow=bc, info={"h": h})


def _sizes_loguniform(n_meshes: int, total: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Log-uniform sizes in [lo, hi], rescaled by a common factor so they sum to total."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), n_meshes))
    for _ in range(50):
        s = np.clip(s * (total / s.sum()), lo, hi)
    s = np.round(s).astype(np.int64)
    s[-1] += total - s.sum()
    s[-1] = int(np.clip(s[-1], lo, hi))
    return s


def batched(n_meshes: int = 64, total: int = 1 << 22, lo: int = 1 << 12, hi: int = 1 << 17, n_dir: int = 128,
            n_groups: int = 2, ngrid: int = 128, seed: int = 1, threads: int | None = None) -> Problem:
    sizes = _sizes_loguniform(n_meshes, total, lo, hi, seed)
    meshes, rhos = [], []
    for i, n in enumerate(sizes):
        pts = F.generators_poisson(int(n), seed * 1000 + i)
        pts = pts[F.hilbert_order(pts)]
        m = voronoi_mesh(pts, periodic=False, threads=threads)
        rho = F.sample_field(F.lognormal_field(ngrid, -3.0, 1.0, seed * 1000 + i), pts)
        meshes.append(m)
        rhos.append(rho)
    mesh = concat_meshes(meshes)
    rho = np.concatenate(rhos)
    kap = F.kappa_from_density(rho, mesh.volume, n_groups)
    eps = np.zeros((mesh.n_cells, n_groups))
    for i, m in enumerate(meshes):
        o = mesh.mesh_cell_offset[i]
        cells, em = F.point_sources(rhos[i] * m.volume, 8, seed * 1000 + 500 + i)
        eps[o + cells, :] = em[:, None]
    om, w = F.fibonacci_directions(n_dir, seed=seed)
    return Problem("batched", mesh, om, w, kap, eps, info={"sizes": sizes.tolist()})


def scatter(n_cells: int = 1 << 20, n_dir: int = 96, n_groups: int = 4, n_src: int = 64, ngrid: int = 128,
            seed: int = 3, threads: int | None = None) -> Problem:
    field_ = F.lognormal_field(ngrid, -3.0, 1.0, seed)
    pts = F.generators_from_density(field_, n_cells, seed + 1)
    pts = pts[F.hilbert_order(pts)]
    mesh = voronoi_mesh(pts, periodic=False, threads=threads)
    rho = F.sample_field(field_, pts)
    ka = F.kappa_from_density(rho, mesh.volume, n_groups)
    cells, em = F.point_sources(rho * mesh.volume, n_src, seed + 2)
    eps = F.emissivity_array(mesh.n_cells, n_groups, cells, em)
    om, w = F.fibonacci_directions(n_dir, seed=seed)
    return Problem("scatter", mesh, om, w, ka, eps, kappa_scat=ka.copy())


def periodic(n_cells: int = 1 << 22, n_dir: int = 128, n_src: int = 10_000, ngrid: int = 256, seed: int = 4,
             threads: int | None = None) -> Problem:
    field_ = F.lognormal_field(ngrid, -2.5, 1.5, seed)
    pts = F.generators_from_density(field_, n_cells, seed + 1)
    pts = pts[F.hilbert_order(pts)]
    mesh = voronoi_mesh(pts, periodic=True, threads=threads)
    rho = F.sample_field(field_, pts)
    ka = F.kappa_from_density(rho, mesh.volume, 1)
    cells, em = F.point_sources(rho * mesh.volume, n_src, seed + 2, log_range=4.0)
    eps = F.emissivity_array(mesh.n_cells, 1, cells, em)
    om, w = F.fibonacci_directions(n_dir, seed=seed)
    return Problem("periodic", mesh, om, w, ka, eps)


def adjoint(n_cells: int = 1 << 18, n_dir: int = 64, n_groups: int = 2, n_src: int = 32, ngrid: int = 128,
            seed: int = 5, threads: int | None = None) -> Problem:
    pts = F.generators_poisson(n_cells, seed)
    pts = pts[F.hilbert_order(pts)]
    mesh = voronoi_mesh(pts, periodic=False, threads=threads)
    rho = F.sample_field(F.lognormal_field(ngrid, -3.0, 1.0, seed), pts)
    ka = F.kappa_from_density(rho, mesh.volume, n_groups)
    cells, em = F.point_sources(rho * mesh.volume, n_src, seed + 1)
    eps = F.emissivity_array(mesh.n_cells, n_groups, cells, em)
    om, w = F.fibonacci_directions(n_dir, seed=seed)
    rng = np.random.default_rng(seed + 2)
    ka_target = ka * (1.0 + 0.1 * rng.normal(size=ka.shape))
    return Problem("adjoint", mesh, om, w, ka, eps, info={"kappa_target": np.abs(ka_target)})


def voronoi_small(n_cells: int, periodic_box: bool = False, n_dir: int = 8, n_groups: int = 1, seed: int = 0,
                  n_src: int = 4, scatter_albedo: float = 0.0, bc_inflow: bool = False) -> Problem:
    """Small random problem for parity tests: Poisson generators, random kappa, a few sources."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n_cells, 3))
    pts = pts[F.hilbert_order(pts)]
    mesh = voronoi_mesh(pts, periodic=periodic_box, threads=1)
    h = np.cbrt(mesh.volume)
    tau = np.exp(rng.uniform(math.log(0.01), math.log(10.0), (mesh.n_cells, n_groups)))
    ka = tau / h[:, None]
    eps = np.zeros((mesh.n_cells, n_groups))
    src = rng.choice(mesh.n_cells, size=min(n_src, mesh.n_cells), replace=False)
    eps[src, :] = rng.uniform(0.5, 2.0, (src.size, n_groups))
    ks = ka * scatter_albedo / max(1e-300, 1.0 - scatter_albedo) if scatter_albedo > 0 else None
    bc = None
    if bc_inflow:
        nb = int(np.count_nonzero(mesh.flags & 1))
        bc = rng.uniform(0.0, 1.0, (nb, n_groups))
    om, w = F.fibonacci_directions(n_dir, seed=seed)
    return Problem("voronoi%d" % n_cells, mesh, om, w, ka, eps, kappa_scat=ks, boundary_inflow=bc)
