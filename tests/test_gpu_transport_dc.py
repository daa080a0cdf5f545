"""GPU parity of direction-conserving transport (scheme (b) of Sec. 2.6, sweep_opts.transport = n)
against the FP64 oracle (oracle.solve / oracle.levels with dc_n = n): levels bit-exact, FP64 sweeps
within 1e-12 (every intensity), FP32 sweeps within 1e-5, photon conservation, with scattering, periodic
faces and boundary inflow."""
import math

import numpy as np
import pytest

import oracle
from synth import configs
from synth.fields import fibonacci_directions
from synth.mesh import concat_meshes, lattice_mesh, star_mesh, voronoi_mesh

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
DEFECT_TOL = 1e-6


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def fp32_err(x, ref):
    m = ref >= 1e-30 * ref.max()
    return float(np.max(np.abs(x[m] - ref[m]) / ref[m]))


def load(ctx, p):
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ctx.set_material(p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat, boundary_inflow=p.boundary_inflow)


def run_oracle(p, **kw):
    return oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                        bc_inflow=p.boundary_inflow, threads=8, **kw)


@pytest.mark.parametrize("n", [1, 3])
@pytest.mark.parametrize("kind", ["lattice", "voronoi", "periodic", "batch"])
def test_dc_levels_bit_exact(ctx, kind, n):
    if kind == "lattice":
        m = lattice_mesh(10)  # axis-aligned faces: exact ties among the outflow faces
        om = np.concatenate([fibonacci_directions(9, seed=1)[0], np.eye(3), -np.eye(3),
                             np.array([[1.0, 1.0, 1.0]]) / math.sqrt(3.0)])
    elif kind == "batch":
        rng = np.random.default_rng(8)
        m = concat_meshes([voronoi_mesh(rng.random((k, 3)), threads=4) for k in (300, 1500, 90)])
        om = fibonacci_directions(16, seed=3)[0]
    else:
        rng = np.random.default_rng(9)
        m = voronoi_mesh(rng.random((4000, 3)), periodic=kind == "periodic", threads=4)
        om = fibonacci_directions(24, seed=2)[0]
    w = np.full(om.shape[0], 4 * math.pi / om.shape[0])
    ctx.set_mesh(m)
    ctx.set_directions(om, w)
    ctx.set_material(np.ones((m.n_cells, 1)), np.ones((m.n_cells, 1)))
    _, _, st, _ = ctx.solve(precision=64, transport=n, max_it_pbc=1)
    rc, lev, depth = oracle.levels(m, om, threads=8, dc_n=n)
    assert rc == 0
    for d in range(om.shape[0]):
        gl, gd = ctx.levels(d)
        assert gd == depth[d] and np.array_equal(gl, lev[d]), d
    assert st["depth_max"] == depth.max()
    # the thinner graph is never deeper than scheme (a)'s
    _, _, sa, _ = ctx.solve(precision=64, transport=0, max_it_pbc=1)
    assert st["depth_max"] <= sa["depth_max"]


@pytest.mark.parametrize("schedule", ["dataflow", "level", "plain"])
@pytest.mark.parametrize("n", [1, 3])
@pytest.mark.parametrize("kind", ["inflow", "periodic", "scatter"])
def test_dc_fp64_every_intensity(ctx, kind, n, schedule):
    p = configs.voronoi_small(3000, periodic_box=kind == "periodic", n_dir=12, n_groups=2, seed=80 + n,
                              scatter_albedo=0.5 if kind == "scatter" else 0.0, n_src=8, bc_inflow=kind == "inflow")
    load(ctx, p)
    it = dict(tol_scat=0.0, max_it_scat=4, tol_pbc=0.0, max_it_pbc=3)
    J, Gm, st, s = ctx.solve(precision=64, schedule=schedule, transport=n, **it)
    r = run_oracle(p, dc_n=n, want_intensity=True, **it)
    assert r["rc"] in (0, 3)  # 3: the fixed iteration counts end before the tolerances
    for d in range(p.n_dir):
        assert rel_max(ctx.intensity(d), r["I"][d]) <= 1e-12, d
    assert rel_max(J, r["J"]) <= 1e-12 and rel_max(Gm, r["Gamma"]) <= 1e-12
    if kind == "inflow":
        assert abs(st["defect"]) <= 1e-12
        assert st["escaped"] == pytest.approx(r["stats"]["escaped"], rel=1e-12)
        assert st["injected"] == pytest.approx(r["stats"]["injected"], rel=1e-12)


@pytest.mark.parametrize("form", [dict(packets_per_step=2), dict(packets_per_step=1), dict(schedule="level"),
                                  dict(geometry_only=1)])
@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("kind", ["inflow", "periodic", "scatter"])
def test_dc_fp32(ctx, kind, G, form):
    # the packed operator (its entries carry the upwind cell's share) and the FP32 mesh-row kernel
    p = configs.voronoi_small(4000, periodic_box=kind == "periodic", n_dir=16, n_groups=G, seed=90 + G,
                              scatter_albedo=0.5 if kind == "scatter" else 0.0, n_src=10, bc_inflow=kind == "inflow")
    load(ctx, p)
    it = dict(tol_scat=0.0, max_it_scat=4, tol_pbc=0.0, max_it_pbc=3)
    kw = dict(schedule="dataflow")
    kw.update(form)
    J, Gm, st, s = ctx.solve(precision=32, transport=3, **kw, **it)
    assert st["kernel_used"] == (2 if form.get("geometry_only") else 7)
    r = run_oracle(p, dc_n=3, want_intensity=True, **it)
    for d in range(p.n_dir):
        assert fp32_err(ctx.intensity(d), r["I"][d]) <= FP32_TOL, d
    assert fp32_err(J, r["J"]) <= FP32_TOL and fp32_err(Gm, r["Gamma"]) <= FP32_TOL
    if kind == "inflow":
        assert abs(st["defect"]) <= DEFECT_TOL


@pytest.mark.parametrize("precision", [64, 32])
def test_dc_converged_conservation(ctx, precision):
    # periodic box with scattering, both iterations converged: against the oracle, and photons conserved
    p = configs.voronoi_small(3000, periodic_box=True, n_dir=12, n_groups=1, seed=95, scatter_albedo=0.5, n_src=8)
    load(ctx, p)
    it = dict(tol_scat=1e-10, max_it_scat=500, tol_pbc=1e-10, max_it_pbc=500)
    J, Gm, st, s = ctx.solve(precision=precision, transport=3, fused_loops=1, **it)
    assert s == 0
    r = run_oracle(p, dc_n=3, fused=True, **it)
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-9 and abs(st["defect"]) <= 1e-9
    else:
        assert fp32_err(J, r["J"]) <= FP32_TOL and abs(st["defect"]) <= DEFECT_TOL


@pytest.mark.parametrize("precision", [64, 32])
def test_dc_with_the_exp_law(ctx, precision):
    p = configs.voronoi_small(3000, n_dir=12, n_groups=2, seed=96, n_src=8, bc_inflow=True, scatter_albedo=0.3)
    load(ctx, p)
    it = dict(tol_scat=1e-10, max_it_scat=500)
    J, Gm, st, s = ctx.solve(precision=precision, transport=3, law="exp", **it)
    r = run_oracle(p, dc_n=3, law="exp", **it)
    assert s == 0
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-9 and abs(st["defect"]) <= 1e-9
    else:
        assert fp32_err(J, r["J"]) <= FP32_TOL and abs(st["defect"]) <= DEFECT_TOL


def test_dc_limits(ctx):
    from paper_2207_12848_gb300 import SweepError
    p = configs.voronoi_small(500, n_dir=4, seed=97)
    load(ctx, p)
    with pytest.raises(SweepError) as e:  # the adjoint takes scheme (a)
        ctx.adjoint(dl_dGamma=np.ones_like(p.kappa_abs), transport=3)
    assert e.value.status == 1
    with pytest.raises(SweepError) as e:
        ctx.solve(transport=9)
    assert e.value.status == 1
    # a cell with more than 64 face sides: scheme (b) refuses, scheme (a) still solves it
    m = star_mesh(80, seed=1)
    om, w = fibonacci_directions(4, seed=3)
    ctx.set_mesh(m)
    ctx.set_directions(om, w)
    ctx.set_material(np.full((m.n_cells, 1), 2.0), np.ones((m.n_cells, 1)))
    with pytest.raises(SweepError) as e:
        ctx.solve(transport=3)
    assert e.value.status == 1
    J, _, _, s = ctx.solve(transport=0)
    assert s == 0 and J.max() > 0


@pytest.fixture(scope="module")
def box18():
    return configs.periodic(n_cells=1 << 18)


def test_dc_on_a_2p18_box(ctx, box18):
    # the benchmark's periodic box at 2^18 cells x 128 directions under scheme (b): every direction's levels
    # bit-exact, J and Gamma after three periodic iterations against the oracle, depth below scheme (a)'s
    p = box18
    load(ctx, p)
    it = dict(tol_pbc=0.0, max_it_pbc=3)
    J, Gm, st, s = ctx.solve(precision=32, relevel=1, transport=3, **it)
    assert st["kernel_used"] == 7
    r = run_oracle(p, dc_n=3, **it)
    assert fp32_err(J, r["J"]) <= FP32_TOL and fp32_err(Gm, r["Gamma"]) <= FP32_TOL
    rc, lev, depth = oracle.levels(p.mesh, p.omega, threads=8, dc_n=3)
    for d in range(p.n_dir):
        gl, gd = ctx.levels(d)
        assert gd == depth[d] and np.array_equal(gl, lev[d]), d
    _, _, sa, _ = ctx.solve(precision=32, relevel=1, transport=0, **it)
    assert st["depth_max"] < sa["depth_max"]
