"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (see the precision statement of the library):
  levels                         bit-exact
  FP64 sweeps (plain, batched)   1e-12 relative (max norm over the array)
  FP32 sweeps, FP64 tallies      mean intensity 1e-5 relative per cell (cells with J >= 1e-30 max J),
                                 photon-conservation defect 1e-6
"""
import math

import numpy as np
import pytest

import oracle
from synth import configs
from synth.mesh import FACE_PERIODIC, column_mesh, concat_meshes, lattice_mesh, voronoi_mesh
from synth.fields import fibonacci_directions

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
DEFECT_TOL = 1e-6


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def fp32_err(J, Jo):
    m = Jo >= 1e-30 * Jo.max()
    return float(np.max(np.abs(J[m] - Jo[m]) / Jo[m]))


def load(ctx, p):
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ctx.set_material(p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat, boundary_inflow=p.boundary_inflow)


def run_oracle(p, **kw):
    return oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                        bc_inflow=p.boundary_inflow, threads=8, **kw)


# ---- levels ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["lattice", "voronoi", "periodic", "batch"])
def test_levels_bit_exact(ctx, kind):
    if kind == "lattice":
        m = lattice_mesh(12)  # axis-aligned faces: exact ties for some directions
        om = np.concatenate([fibonacci_directions(10, seed=1)[0], np.eye(3), -np.eye(3)])
    elif kind == "batch":
        rng = np.random.default_rng(7)
        m = concat_meshes([voronoi_mesh(rng.random((n, 3)), threads=4) for n in (300, 1200, 77, 2500)])
        om = fibonacci_directions(24, seed=3)[0]
    else:
        rng = np.random.default_rng(5)
        m = voronoi_mesh(rng.random((5000, 3)), periodic=kind == "periodic", threads=4)
        om = fibonacci_directions(33, seed=2)[0]
    w = np.full(om.shape[0], 4 * math.pi / om.shape[0])
    ctx.set_mesh(m)
    ctx.set_directions(om, w)
    rc, lev, depth = oracle.levels(m, om, threads=8)
    assert rc == 0
    for d in range(om.shape[0]):
        gl, gd = ctx.levels(d)
        assert np.array_equal(gl, lev[d]), d
        assert gd == depth[d]


# ---- FP64: plain per-(direction, level) launches and the batched kernel ------------------------------
@pytest.mark.parametrize("schedule", ["plain", "level", "dataflow"])
def test_plain32_fp64(ctx, schedule):
    p = configs.plain32()
    load(ctx, p)
    J, G, st, s = ctx.solve(precision=64, schedule=schedule)
    r = run_oracle(p)
    assert rel_max(J, r["J"]) <= 1e-12
    assert rel_max(G, r["Gamma"]) <= 1e-12
    assert abs(st["defect"]) <= 1e-12
    assert st["emitted"] == pytest.approx(r["stats"]["emitted"], rel=1e-14)


@pytest.mark.parametrize("G", [1, 2, 3, 4])
def test_voronoi_fp64_intensities(ctx, G):
    p = configs.voronoi_small(3000, n_dir=12, n_groups=G, seed=G, bc_inflow=True)
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=64, schedule="dataflow")
    r = run_oracle(p, want_intensity=True)
    for d in range(p.n_dir):
        assert rel_max(ctx.intensity(d), r["I"][d]) <= 1e-12
    assert rel_max(J, r["J"]) <= 1e-12
    assert abs(st["defect"]) <= 1e-12


# ---- FP32 sweeps with FP64 tallies ----------------------------------------------------------------------
@pytest.mark.parametrize("geometry_only", [0, 1])
@pytest.mark.parametrize("schedule", ["level", "dataflow", "auto"])
@pytest.mark.parametrize("G", [1, 2, 4])
def test_voronoi_fp32(ctx, schedule, G, geometry_only):
    p = configs.voronoi_small(6000, n_dir=16, n_groups=G, seed=10 + G, n_src=12)
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=32, schedule=schedule, geometry_only=geometry_only)
    r = run_oracle(p)
    assert fp32_err(J, r["J"]) <= FP32_TOL
    assert fp32_err(Gm, r["Gamma"]) <= FP32_TOL
    assert abs(st["defect"]) <= DEFECT_TOL
    assert st["absorbed"] == pytest.approx(r["stats"]["absorbed"], rel=FP32_TOL)


@pytest.mark.parametrize("lanes,bpsm", [(1, 1), (1, 0), (2, 0), (4, 0), (8, 0), (16, 0)])
@pytest.mark.parametrize("G", [1, 3])
def test_operator_kernels(ctx, lanes, bpsm, G):
    # every form of the FP32 forward sweep over the assembled operator (and the periodic inflow path)
    p = configs.voronoi_small(5000, periodic_box=True, n_dir=16, n_groups=G, seed=20 + G, n_src=10)
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=32, schedule="dataflow", lanes_per_task=lanes, blocks_per_sm=bpsm,
                             tol_pbc=0.0, max_it_pbc=4)
    assert st["lanes_used"] == lanes
    if G == 1 and lanes in (8, 16):
        assert st["kernel_used"] == {8: 5, 16: 6}[lanes]  # the lean forms
    r = run_oracle(p, tol_pbc=0.0, max_it_pbc=4)
    assert fp32_err(J, r["J"]) <= FP32_TOL


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("reverse", [False, True])
def test_column_closed_form(ctx, precision, reverse):
    n, h, kap = 256, 1.0 / 256, 3.2
    p = configs.column(n, kappa=kap, h=h, reverse=reverse)
    load(ctx, p)
    ctx.solve(precision=precision, schedule="dataflow")
    I = ctx.intensity(0)[:, 0]
    k = np.arange(n) if not reverse else np.arange(n)[::-1]
    exact = (1.0 + kap * h) ** (-(k + 1.0))
    tol = 1e-14 if precision == 64 else 1e-5
    assert rel_max(I, exact) <= tol
    assert np.max(np.abs(I - exact) / exact) <= (1e-13 if precision == 64 else 2e-5)


# ---- the EXP absorption law ------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [64, 32])
def test_exp_law_column(ctx, precision):
    # the EXP update is the exact transport solution along a column of cubes: exp(-kappa x) at each
    # cell's exit, and J the chord average of exp(-kappa x) over the cell
    n, h, kap = 256, 1.0 / 256, 3.2
    p = configs.column(n, kappa=kap, h=h)
    load(ctx, p)
    J, _, st, _ = ctx.solve(precision=precision, law="exp")
    k = np.arange(n)
    tol = 1e-13 if precision == 64 else 1e-5
    assert rel_max(ctx.intensity(0)[:, 0], np.exp(-kap * h * (k + 1.0))) <= tol
    assert rel_max(J[:, 0], (np.exp(-kap * h * k) - np.exp(-kap * h * (k + 1.0))) / (kap * h)) <= tol
    assert st["kernel_used"] == (2 if precision == 64 else 7)  # the generic kernel, or the packed one in FP32


@pytest.mark.parametrize("precision,schedule", [(64, "dataflow"), (64, "plain"), (32, "dataflow"), (32, "level")])
@pytest.mark.parametrize("kind", ["vacuum", "scattering", "periodic"])
def test_exp_law_matches_oracle(ctx, precision, schedule, kind):
    p = configs.voronoi_small(4000, periodic_box=kind == "periodic", n_dir=12, n_groups=2, seed=63,
                              scatter_albedo=0.5 if kind != "vacuum" else 0.0, n_src=8,
                              bc_inflow=kind == "vacuum")
    load(ctx, p)
    it = dict(tol_scat=1e-10, max_it_scat=500, tol_pbc=1e-10, max_it_pbc=500)
    J, Gm, st, s = ctx.solve(precision=precision, schedule=schedule, law="exp", **it)
    r = run_oracle(p, law="exp", **it)
    assert s == 0
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-9 and rel_max(Gm, r["Gamma"]) <= 1e-9
    else:
        assert fp32_err(J, r["J"]) <= FP32_TOL
    assert abs(st["defect"]) <= (1e-9 if precision == 64 else DEFECT_TOL)
    # plain, generic (FP64) or packed (FP32) kernel
    assert st["kernel_used"] == (1 if schedule == "plain" else (2 if precision == 64 else 7))
    # the BALANCE answer on the same context is unchanged by an EXP solve in between
    Jb, _, _, _ = ctx.solve(precision=precision, **it)
    assert fp32_err(Jb, run_oracle(p, **it)["J"]) <= (1e-9 if precision == 64 else FP32_TOL)


def test_exp_law_rejected_by_the_adjoint(ctx):
    from paper_2207_12848_gb300 import SweepError
    p = configs.voronoi_small(500, n_dir=4, seed=65)
    load(ctx, p)
    with pytest.raises(SweepError) as e:
        ctx.adjoint(dl_dGamma=np.ones_like(p.kappa_abs), law="exp")
    assert e.value.status == 1


def test_column_deeper_than_the_level_tables(ctx):
    # 70000 levels of one cell: more than the direction-parallel levelisation's 65536-level tables, so the
    # level-synchronous form takes over; levels and the closed form must come out the same
    n, kap = 70000, 3.2
    h = 1.0 / n
    p = configs.column(n, kappa=kap, h=h)
    load(ctx, p)
    lev, depth = ctx.levels(0)
    assert depth == n and np.array_equal(lev, np.arange(n))
    ctx.solve(precision=64, schedule="dataflow")
    I = ctx.intensity(0)[:, 0]
    k = np.arange(n)
    exact = np.exp(-(k + 1.0) * np.log1p(kap * h))
    assert np.max(np.abs(I - exact) / exact) <= 1e-11


# ---- iterations: scattering (Alg. 1) and periodic boundaries (Sec. 2.7) -------------------------------
@pytest.mark.parametrize("precision", [32, 64])
def test_scattering_iteration(ctx, precision):
    p = configs.voronoi_small(4000, n_dir=12, n_groups=2, seed=41, scatter_albedo=0.5, n_src=8)
    load(ctx, p)
    # a fixed number of source iterations: both sides do exactly the same sweeps
    J, Gm, st, s = ctx.solve(precision=precision, schedule="dataflow", tol_scat=0.0, max_it_scat=6)
    r = run_oracle(p, tol_scat=0.0, max_it_scat=6)
    assert st["it_scat"] == r["stats"]["it_scat"] == 6
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-12
        assert st["res_scat"] == pytest.approx(r["stats"]["res_scat"], rel=1e-9)
    else:
        assert fp32_err(J, r["J"]) <= FP32_TOL
    # converged
    J, Gm, st, s = ctx.solve(precision=precision, tol_scat=1e-8, max_it_scat=200)
    r = run_oracle(p, tol_scat=1e-8, max_it_scat=200)
    assert s == 0 and st["res_scat"] <= 1e-8
    assert fp32_err(J, r["J"]) <= (1e-10 if precision == 64 else FP32_TOL)
    assert abs(st["defect"]) <= (1e-7 if precision == 64 else DEFECT_TOL)


@pytest.mark.parametrize("precision", [32, 64])
def test_periodic_iteration(ctx, precision):
    p = configs.voronoi_small(5000, periodic_box=True, n_dir=12, n_groups=1, seed=43, n_src=6)
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=precision, schedule="level", tol_pbc=0.0, max_it_pbc=5)
    r = run_oracle(p, tol_pbc=0.0, max_it_pbc=5)
    assert st["it_pbc"] == r["stats"]["it_pbc"] == 5
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-12
        assert st["res_pbc"] == pytest.approx(r["stats"]["res_pbc"], rel=1e-9)
    else:
        assert fp32_err(J, r["J"]) <= FP32_TOL
    J, Gm, st, s = ctx.solve(precision=precision, tol_pbc=1e-7, max_it_pbc=300)
    r = run_oracle(p, tol_pbc=1e-7, max_it_pbc=300)
    assert s == 0 and st["res_pbc"] < 1e-7
    assert fp32_err(J, r["J"]) <= (1e-9 if precision == 64 else FP32_TOL)
    assert abs(st["defect"]) <= 1e-6


def test_periodic_warm_start(ctx):
    p = configs.voronoi_small(3000, periodic_box=True, n_dir=8, seed=45)
    load(ctx, p)
    _, _, st1, _ = ctx.solve(precision=64, tol_pbc=1e-9)
    J2, _, st2, _ = ctx.solve(precision=64, tol_pbc=1e-9, warm_start=1)
    assert st2["it_pbc"] < st1["it_pbc"]
    r = run_oracle(p, tol_pbc=1e-12, max_it_pbc=500)
    assert rel_max(J2, r["J"]) <= 1e-7


def test_batched_meshes_fp32(ctx):
    p = configs.batched(n_meshes=6, total=20000, lo=1000, hi=8000, n_dir=16, n_groups=2, ngrid=32, threads=8)
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=32)
    r = run_oracle(p)
    assert fp32_err(J, r["J"]) <= FP32_TOL
    assert abs(st["defect"]) <= DEFECT_TOL


# ---- adjoint ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision,batch", [(64, 0), (64, 5), (32, 0), (32, 7)])
def test_adjoint_matches_oracle(ctx, precision, batch):
    p = configs.voronoi_small(3000, n_dir=16, n_groups=2, seed=51, n_src=6)
    load(ctx, p)
    rng = np.random.default_rng(52)
    dg = rng.normal(size=p.kappa_abs.shape)
    dj = rng.normal(size=p.kappa_abs.shape)
    gk, ge, st = ctx.adjoint(dl_dJ=dj, dl_dGamma=dg, precision=precision, dir_batch=batch, schedule="dataflow")
    rc, ok_, oe = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dl_dJ=dj, dl_dGamma=dg,
                                 threads=8)
    assert rc == 0
    tol = 1e-10 if precision == 64 else 1e-4
    assert rel_max(gk, ok_) <= tol
    assert rel_max(ge, oe) <= tol


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("albedo", [0.0, 0.5])
def test_adjoint_through_the_periodic_iteration(ctx, precision, albedo):
    # the transposed iteration with periodic faces (and scattering) against the oracle's: a fixed
    # number of forward sweeps and transposed passes, then converged
    p = configs.voronoi_small(3000, periodic_box=True, n_dir=12, n_groups=2, seed=59, scatter_albedo=albedo,
                              n_src=6)
    load(ctx, p)
    ks = p.kappa_scat if albedo else np.zeros_like(p.kappa_abs)
    rng = np.random.default_rng(60)
    dg = rng.normal(size=p.kappa_abs.shape)
    dj = rng.normal(size=p.kappa_abs.shape)
    fixed = dict(tol_scat=0.0, max_it_scat=3, tol_pbc=0.0, max_it_pbc=3)
    gk, ge, gs, st = ctx.adjoint(dl_dJ=dj, dl_dGamma=dg, precision=precision, schedule="dataflow",
                                 with_kappa_scat=True, allow_not_converged=True, **fixed)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, dl_dJ=dj,
                            dl_dGamma=dg, threads=8, **fixed)
    assert st["it_scat"] == r["it_forward"] == (9 if albedo else 3)
    assert st["it_pbc"] == r["it_adjoint"] == 3
    tol = 1e-10 if precision == 64 else 1e-4
    assert rel_max(gk, r["grad_kappa_abs"]) <= tol
    assert rel_max(ge, r["grad_emissivity"]) <= tol
    assert rel_max(gs, r["grad_kappa_scat"]) <= tol
    t = 1e-11 if precision == 64 else 1e-6
    conv = dict(tol_scat=t, max_it_scat=2000, tol_pbc=t, max_it_pbc=2000)
    gk, ge, gs, st = ctx.adjoint(dl_dJ=dj, dl_dGamma=dg, precision=precision, with_kappa_scat=True, **conv)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, dl_dJ=dj,
                            dl_dGamma=dg, threads=8, **conv)
    assert st["it_pbc"] > 3 and st["res_pbc"] <= t
    tol = 1e-9 if precision == 64 else 1e-4
    assert rel_max(gk, r["grad_kappa_abs"]) <= tol
    assert rel_max(ge, r["grad_emissivity"]) <= tol
    assert rel_max(gs, r["grad_kappa_scat"]) <= tol


def test_adjoint_periodic_plain_schedule(ctx):
    # the plain FP64 path's transposed periodic reads, against the batched FP64 adjoint
    p = configs.voronoi_small(2000, periodic_box=True, n_dir=6, n_groups=1, seed=61, n_src=4)
    load(ctx, p)
    dg = np.random.default_rng(62).normal(size=p.kappa_abs.shape)
    kw = dict(tol_scat=1e-12, max_it_scat=2000, tol_pbc=1e-12, max_it_pbc=2000)
    gk_p, ge_p, _ = ctx.adjoint(dl_dGamma=dg, schedule="plain", **kw)
    gk_b, ge_b, _ = ctx.adjoint(dl_dGamma=dg, precision=64, schedule="dataflow", **kw)
    assert rel_max(gk_p, gk_b) <= 1e-10 and rel_max(ge_p, ge_b) <= 1e-10


@pytest.mark.parametrize("precision", [64, 32])
def test_adjoint_through_the_source_iteration(ctx, precision):
    # the transposed source iteration against the oracle's: first sweep for sweep (a fixed number of
    # forward and transposed passes), then both converged, with the gradient in kappa_scat
    p = configs.voronoi_small(3000, n_dir=16, n_groups=2, seed=55, scatter_albedo=0.5, n_src=6)
    load(ctx, p)
    rng = np.random.default_rng(56)
    dg = rng.normal(size=p.kappa_abs.shape)
    dj = rng.normal(size=p.kappa_abs.shape)
    tol = 1e-10 if precision == 64 else 1e-4
    gk, ge, gs, st = ctx.adjoint(dl_dJ=dj, dl_dGamma=dg, precision=precision, schedule="dataflow", tol_scat=0.0,
                                 max_it_scat=5, with_kappa_scat=True, allow_not_converged=True)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                            dl_dJ=dj, dl_dGamma=dg, tol_scat=0.0, max_it_scat=5, threads=8)
    assert r["rc"] == oracle.NOT_CONVERGED  # a fixed count: both iterations stop at their maximum
    assert st["it_scat"] == r["it_forward"] == 5 and st["it_pbc"] == r["it_adjoint"] == 5
    assert rel_max(gk, r["grad_kappa_abs"]) <= tol
    assert rel_max(ge, r["grad_emissivity"]) <= tol
    assert rel_max(gs, r["grad_kappa_scat"]) <= tol
    kw = dict(tol_scat=1e-11 if precision == 64 else 1e-6, max_it_scat=500)
    gk, ge, gs, st = ctx.adjoint(dl_dJ=dj, dl_dGamma=dg, precision=precision, with_kappa_scat=True, **kw)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                            dl_dJ=dj, dl_dGamma=dg, threads=8, **kw)
    assert st["res_pbc"] <= kw["tol_scat"] and st["it_pbc"] > 5
    tol = 1e-9 if precision == 64 else 1e-4
    assert rel_max(gk, r["grad_kappa_abs"]) <= tol
    assert rel_max(ge, r["grad_emissivity"]) <= tol
    assert rel_max(gs, r["grad_kappa_scat"]) <= tol


def test_adjoint_kappa_scat_gradient_without_scattering(ctx):
    # the derivative at kappa_s = 0 needs J but no source iteration: one forward and one transposed sweep
    p = configs.voronoi_small(3000, n_dir=16, n_groups=2, seed=57, n_src=6)
    load(ctx, p)
    dg = np.random.default_rng(58).normal(size=p.kappa_abs.shape)
    gk, ge, gs, st = ctx.adjoint(dl_dGamma=dg, precision=64, dir_batch=5, with_kappa_scat=True)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity,
                            kappa_scat=np.zeros_like(p.kappa_abs), dl_dGamma=dg, threads=8)
    assert st["it_scat"] == st["it_pbc"] == 1
    assert rel_max(gk, r["grad_kappa_abs"]) <= 1e-10
    assert rel_max(gs, r["grad_kappa_scat"]) <= 1e-10


# ---- edge cases -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("geometry_only,lanes", [(0, 0), (1, 0), (0, 16)])
def test_high_degree_cell(ctx, geometry_only, lanes):
    # a generator at the centre of a sphere of 60 others: its cell has ~60 faces (rows longer than
    # 32 sides) and ~30 inflow sides per direction (more than an operator line holds)
    rng = np.random.default_rng(61)
    u = rng.normal(size=(60, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    inner = 0.5 + 0.08 * u
    outer = rng.random((1500, 3))
    outer = outer[np.linalg.norm(outer - 0.5, axis=1) > 0.16]
    pts = np.concatenate([[[0.5, 0.5, 0.5]], inner, outer])
    m = voronoi_mesh(pts, threads=4)
    assert m.neighbour_counts()[0] > 40
    om, w = fibonacci_directions(24, seed=5)
    ka = np.full((m.n_cells, 2), 3.0)
    ka[:, 1] = 0.5
    eps = np.zeros((m.n_cells, 2))
    eps[0] = 1.0
    eps[100] = 2.0
    ctx.set_mesh(m)
    ctx.set_directions(om, w)
    ctx.set_material(ka, eps)
    J, G, st, s = ctx.solve(precision=32, geometry_only=geometry_only, lanes_per_task=lanes,
                            schedule="dataflow" if lanes else "auto")
    r = oracle.solve(m, om, w, ka, eps, threads=8)
    assert fp32_err(J, r["J"]) <= FP32_TOL
    J64, _, _, _ = ctx.solve(precision=64)
    assert rel_max(J64, r["J"]) <= 1e-12



def test_single_cell_and_single_direction(ctx):
    m = lattice_mesh(1)
    ctx.set_mesh(m)
    ctx.set_directions(np.array([[0.0, 0.6, 0.8]]), np.array([4 * math.pi]))
    ctx.set_material(np.array([[2.0]]), np.array([[1.0]]))
    J, G, st, s = ctx.solve(precision=64)
    # one cube cell: P = 0.6 + 0.8 (projected outflow area), I = (eps/4pi) / (P + kappa V)
    I = (1.0 / (4 * math.pi)) / (1.4 + 2.0)
    assert J[0, 0] == pytest.approx(I, rel=1e-15)
    assert st["depth_max"] == 1


def test_mesh_without_faces(ctx):
    from synth.mesh import Mesh
    m = Mesh(volume=np.array([0.5, 0.25]), face_cells=np.zeros((0, 2), np.int32), area=np.zeros(0),
             normal=np.zeros((0, 3)), flags=np.zeros(0, np.uint8))
    ctx.set_mesh(m)
    om, w = fibonacci_directions(4, seed=0)
    ctx.set_directions(om, w)
    ctx.set_material(np.array([[1.0], [2.0]]), np.array([[1.0], [3.0]]))
    J, G, st, s = ctx.solve(precision=32)
    # no faces: every photon is absorbed in place, Gamma = eps
    assert np.allclose(G[:, 0], [1.0, 3.0], rtol=1e-6)


def test_zero_absorption_streaming(ctx):
    p = configs.voronoi_small(2000, n_dir=8, seed=55)
    load(ctx, p)
    ctx.set_material(np.zeros_like(p.kappa_abs), p.emissivity)
    J, G, st, s = ctx.solve(precision=64)
    assert st["absorbed"] == 0.0
    assert st["escaped"] == pytest.approx(st["emitted"], rel=1e-13)


def test_odd_group_count_and_many_directions(ctx):
    p = configs.voronoi_small(1500, n_dir=200, n_groups=5, seed=57)
    load(ctx, p)
    J, G, st, s = ctx.solve(precision=32)
    r = run_oracle(p)
    assert fp32_err(J, r["J"]) <= FP32_TOL


# ---- full-size workload in the benchmark's launch configuration: sampled parity and properties -------
@pytest.mark.slow
def test_periodic_headline_full_size(ctx):
    p = configs.periodic()
    load(ctx, p)
    J, G, st, s = ctx.solve(precision=32, relevel=1)
    assert s == 0 and st["res_pbc"] < 1e-6
    assert abs(st["defect"]) <= DEFECT_TOL
    # levels of sampled directions, bit-exact
    for d in (0, 77):
        rc, lev, depth = oracle.levels(p.mesh, p.omega[d:d + 1], threads=1)
        gl, gd = ctx.levels(d)
        assert np.array_equal(gl, lev[0]) and gd == depth[0]
    # per-task balance of the final sweep for a sampled direction, evaluated in FP64 from the
    # GPU's own intensities (the cell update must hold for every cell)
    d = 5
    I = ctx.intensity(d)[:, 0]
    m = p.mesh
    t = (m.normal[:, 0] * p.omega[d, 0] + m.normal[:, 1] * p.omega[d, 1]) + m.normal[:, 2] * p.omega[d, 2]
    a = m.area * np.abs(t)
    c0, c1 = m.face_cells[:, 0], m.face_cells[:, 1]
    per = (m.flags & FACE_PERIODIC) != 0
    up = np.where(t > 0, c0, c1)
    down = np.where(t > 0, c1, c0)
    P = np.bincount(up[t != 0], weights=a[t != 0], minlength=m.n_cells)
    inflow = np.bincount(down[(t != 0) & ~per], weights=(a * I[up])[(t != 0) & ~per], minlength=m.n_cells)
    q = p.emissivity[:, 0] / (4 * math.pi)
    lhs = (P + p.kappa_abs[:, 0] * m.volume) * I
    rhs = q + inflow
    # periodic inflow comes from the previous iteration: compare only cells without periodic faces
    has_p = np.zeros(m.n_cells, bool)
    has_p[c0[per]] = True
    has_p[c1[per]] = True
    ok = ~has_p & (rhs > 1e-30 * rhs.max())
    assert np.max(np.abs(lhs[ok] - rhs[ok]) / rhs[ok]) <= 1e-5


@pytest.mark.parametrize("precision", [64, 32])
def test_plain32_against_stored_golden(ctx, precision):
    # stored FP64 oracle values of the 32^3 lattice set-up (tests/golden/oracle_plain32.json)
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_plain32.json")) as f:
        g = json.load(f)
    p = configs.plain32()
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=precision)
    tol = 1e-12 if precision == 64 else FP32_TOL
    assert np.max(np.abs(J[g["cells"], 0] - g["J"]) / np.abs(g["J"])) <= tol
    assert np.max(np.abs(Gm[g["cells"], 0] - g["Gamma"]) / np.abs(g["Gamma"])) <= tol
    assert [ctx.levels(d)[1] for d in range(p.n_dir)] == g["depths"]


@pytest.mark.parametrize("kind", ["periodic", "scattering"])
def test_iteration_graphs_match_the_host_loop(ctx, kind):
    # the iterations replayed as CUDA graphs run the same kernels in the same order as the host loop,
    # and every reduction has a fixed order: the answers are bit-identical
    if kind == "periodic":
        p = configs.voronoi_small(4000, periodic_box=True, n_dir=12, n_groups=2, seed=91, n_src=8)
    else:
        p = configs.voronoi_small(4000, n_dir=12, n_groups=2, seed=92, scatter_albedo=0.5, n_src=8)
    load(ctx, p)
    Jg, Gg, sg, _ = ctx.solve(precision=32, schedule="dataflow", use_graph=1)
    Jh, Gh, sh, _ = ctx.solve(precision=32, schedule="dataflow", use_graph=0)
    assert sg["graph_used"] == 1 and sh["graph_used"] == 0
    assert sg["n_sweeps"] == sh["n_sweeps"] and sg["it_pbc"] == sh["it_pbc"] and sg["it_scat"] == sh["it_scat"]
    assert np.array_equal(Jg, Jh) and np.array_equal(Gg, Gh)
    assert sg["t_sweep_ms"] > 0  # sweep time from the event nodes inside the graphs
    r = run_oracle(p)
    assert fp32_err(Jg, r["J"]) <= FP32_TOL


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_fused_scattering_and_periodic_loops(ctx, precision, use_graph):
    # Sec. 2.7's fused loops: one source-iteration sweep per periodic iteration, against the oracle's
    # fused loop sweep for sweep, then converged against the nested loops' fixed point
    p = configs.voronoi_small(4000, periodic_box=True, n_dir=12, n_groups=2, seed=47, scatter_albedo=0.5, n_src=8)
    load(ctx, p)
    J, Gm, st, s = ctx.solve(precision=precision, schedule="dataflow", tol_pbc=0.0, tol_scat=0.0, max_it_pbc=5,
                             fused_loops=1, use_graph=use_graph)
    r = run_oracle(p, tol_pbc=0.0, tol_scat=0.0, max_it_pbc=5, fused=True)
    assert st["graph_used"] == use_graph
    assert st["it_pbc"] == st["it_scat"] == st["n_sweeps"] == r["stats"]["it_pbc"] == r["stats"]["it_scat"] == 5
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-12
        assert st["res_pbc"] == pytest.approx(r["stats"]["res_pbc"], rel=1e-9)
        assert st["res_scat"] == pytest.approx(r["stats"]["res_scat"], rel=1e-9)
    else:
        assert fp32_err(J, r["J"]) <= FP32_TOL
    kw = dict(tol_pbc=1e-7, tol_scat=1e-8, max_it_pbc=400, max_it_scat=400)
    Jf, Gf, sf, s = ctx.solve(precision=precision, fused_loops=1, use_graph=use_graph, **kw)
    assert s == 0 and sf["res_pbc"] < 1e-7 and sf["res_scat"] <= 1e-8
    r = run_oracle(p, fused=True, **kw)
    assert sf["it_pbc"] == sf["it_scat"]
    assert fp32_err(Jf, r["J"]) <= (1e-10 if precision == 64 else FP32_TOL)
    assert abs(sf["defect"]) <= (1e-7 if precision == 64 else DEFECT_TOL)
    Jn, _, sn, s = ctx.solve(precision=precision, fused_loops=0, **kw)
    assert s == 0 and sn["n_sweeps"] > sf["n_sweeps"]
    assert fp32_err(Jf, Jn) <= (1e-6 if precision == 64 else FP32_TOL)


def test_fused_loops_graph_matches_the_host_loop(ctx):
    p = configs.voronoi_small(4000, periodic_box=True, n_dir=12, n_groups=2, seed=93, scatter_albedo=0.5, n_src=8)
    load(ctx, p)
    Jg, Gg, sg, _ = ctx.solve(precision=32, schedule="dataflow", fused_loops=1, use_graph=1)
    Jh, Gh, sh, _ = ctx.solve(precision=32, schedule="dataflow", fused_loops=1, use_graph=0)
    assert sg["graph_used"] == 1 and sh["graph_used"] == 0
    assert sg["n_sweeps"] == sh["n_sweeps"] and sg["it_pbc"] == sh["it_pbc"] == sg["it_scat"]
    assert np.array_equal(Jg, Jh) and np.array_equal(Gg, Gh)
    # the nested loops stay on the host loop
    _, _, sn, _ = ctx.solve(precision=32, schedule="dataflow", fused_loops=0, use_graph=1)
    assert sn["graph_used"] == 0


def test_adjoint_against_central_differences(ctx):
    # the GPU's FP64 adjoint against FP64 central differences of the GPU's own solve, on the 2^12-cell
    # differentiation sub-mesh, loss sum (Gamma - T)^2
    p = configs.voronoi_small(4096, n_dir=8, n_groups=2, seed=36, n_src=6)
    load(ctx, p)
    T = np.random.default_rng(37).random(p.kappa_abs.shape) * 1e-3

    def loss(ka, em):
        ctx.set_material(ka, em)
        _, Gm, _, _ = ctx.solve(precision=64)
        return math.fsum(((Gm - T) ** 2).ravel()), Gm

    L0, G0 = loss(p.kappa_abs, p.emissivity)
    gk, ge, _ = ctx.adjoint(dl_dGamma=2 * (G0 - T), precision=64)
    rng = np.random.default_rng(38)
    big = np.argsort(np.abs(gk[:, 0]))[-40:]
    for c in rng.choice(big, 4, replace=False):
        for g in range(2):
            h = 1e-4 * p.kappa_abs[c, g]
            kp, km = p.kappa_abs.copy(), p.kappa_abs.copy()
            kp[c, g] += h
            km[c, g] -= h
            fd = (loss(kp, p.emissivity)[0] - loss(km, p.emissivity)[0]) / (2 * h)
            assert gk[c, g] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gk).max())
            # emissivity must stay >= 0 (most cells have none): the loss is quadratic in it (Gamma is
            # linear), so the one-sided three-point difference is exact up to rounding
            he = 1e-4 * max(p.emissivity[c, g], 1.0)
            e1, e2 = p.emissivity.copy(), p.emissivity.copy()
            e1[c, g] += he
            e2[c, g] += 2 * he
            fde = (-3 * L0 + 4 * loss(p.kappa_abs, e1)[0] - loss(p.kappa_abs, e2)[0]) / (2 * he)
            assert ge[c, g] == pytest.approx(fde, rel=1e-6, abs=1e-7 * np.abs(ge).max())


@pytest.mark.parametrize("precision", [64, 32])
def test_answers_reproducible_across_contexts(gpu_lib, precision):
    # every CSR row is sorted by face, and every reduction runs in a fixed order, so two contexts built
    # from the same inputs give bit-identical answers (a row left in the order its sides were scattered
    # by atomics would change the summation order from one build to the next)
    from paper_2207_12848_gb300 import Context
    p = configs.voronoi_small(20000, periodic_box=True, n_dir=16, n_groups=1, seed=101, n_src=8)
    out = []
    for _ in range(2):
        with Context(0) as c:
            load(c, p)
            J, G, st, s = c.solve(precision=precision, tol_pbc=0.0, max_it_pbc=3)
            out.append((J, G, c.intensity(7)))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
