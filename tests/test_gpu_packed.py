"""GPU parity of the sweep over the packed operator (tasks packed back to back, within a wavefront
level, into 512-byte warp packets) against the FP64 oracle, element by element, including the
headline workload's kernel at a size where its wide levels run.

Tolerances as in test_gpu_parity: FP32 intensities within 1e-5 relative of the oracle (cells with a
value >= 1e-30 of the largest), photon-conservation defect within 1e-6, levels bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from synth import configs
from synth.fields import fibonacci_directions
from synth.mesh import star_mesh

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
DEFECT_TOL = 1e-6
PACKED = 7  # SWEEP_KERNEL_PACKED


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


@pytest.mark.parametrize("pps", [1, 2])
@pytest.mark.parametrize("schedule", ["dataflow", "level"])
@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("kind", ["periodic", "inflow"])
def test_packed_forms_every_intensity(ctx, kind, G, schedule, pps):
    # periodic entries (previous iteration's partner) and boundary-inflow entries, every task's value
    p = configs.voronoi_small(5000, periodic_box=kind == "periodic", n_dir=16, n_groups=G, seed=70 + G, n_src=10,
                              bc_inflow=kind == "inflow")
    load(ctx, p)
    it = dict(tol_pbc=0.0, max_it_pbc=3)
    J, Gm, st, s = ctx.solve(precision=32, schedule=schedule, op_format="packets", packets_per_step=pps, **it)
    assert st["kernel_used"] == PACKED and st["lanes_used"] == 32 * pps
    r = run_oracle(p, want_intensity=True, **it)
    for d in range(p.n_dir):
        assert fp32_err(ctx.intensity(d), r["I"][d]) <= FP32_TOL, d
    assert fp32_err(J, r["J"]) <= FP32_TOL
    assert fp32_err(Gm, r["Gamma"]) <= FP32_TOL
    if kind == "inflow":
        assert abs(st["defect"]) <= DEFECT_TOL


@pytest.mark.parametrize("use_graph", [1, 0])
def test_packed_scattering_iteration(ctx, use_graph):
    # the source iteration over the packed operator: six sweeps, sweep for sweep, then converged
    p = configs.voronoi_small(4000, n_dir=12, n_groups=2, seed=77, scatter_albedo=0.5, n_src=8)
    load(ctx, p)
    J, _, st, _ = ctx.solve(precision=32, tol_scat=0.0, max_it_scat=6, use_graph=use_graph)
    assert st["kernel_used"] == PACKED and st["it_scat"] == 6
    assert fp32_err(J, run_oracle(p, tol_scat=0.0, max_it_scat=6)["J"]) <= FP32_TOL
    J, _, st, s = ctx.solve(precision=32, tol_scat=1e-6, max_it_scat=200, use_graph=use_graph)
    assert s == 0 and abs(st["defect"]) <= DEFECT_TOL
    assert fp32_err(J, run_oracle(p, tol_scat=1e-6, max_it_scat=200)["J"]) <= 2 * FP32_TOL


@pytest.mark.parametrize("n_arms,packed", [(80, True), (160, False)])
def test_packed_long_rows(ctx, n_arms, packed):
    # a hub with 80 faces: rows longer than 32 sides and ~40 inflow sides (a task of more than 16 lanes,
    # whose packet takes the fifth scan step); with 160 faces ~80 inflow sides exceed what a packet
    # holds (63), and the solve falls back to the 128-byte line form
    m = star_mesh(n_arms, seed=n_arms)
    om, w = fibonacci_directions(12, seed=3)
    ka = np.full((m.n_cells, 1), 2.0)
    eps = np.zeros((m.n_cells, 1))
    eps[0] = 1.0
    bc = np.random.default_rng(1).uniform(0.1, 1.0, (n_arms, 1))
    ctx.set_mesh(m)
    ctx.set_directions(om, w)
    ctx.set_material(ka, eps, boundary_inflow=bc)
    J, _, st, s = ctx.solve(precision=32, op_format="packets")
    assert (st["kernel_used"] == PACKED) == packed
    r = oracle.solve(m, om, w, ka, eps, bc_inflow=bc, threads=4, want_intensity=True)
    assert fp32_err(J, r["J"]) <= FP32_TOL
    for d in range(om.shape[0]):
        assert fp32_err(ctx.intensity(d), r["I"][d]) <= FP32_TOL


def test_packed_and_line_forms_agree(ctx):
    # both assembled forms, and the mesh-row kernel, on one context: the operator is rebuilt in the
    # requested form each time, and every form matches the oracle
    p = configs.voronoi_small(6000, periodic_box=True, n_dir=24, seed=79, n_src=16)
    load(ctx, p)
    it = dict(tol_pbc=0.0, max_it_pbc=2)
    r = run_oracle(p, **it)
    for kw, kernel in ((dict(op_format="packets"), PACKED), (dict(op_format="lines", lanes_per_task=16), 6),
                       (dict(geometry_only=1), 3), (dict(op_format="packets", packets_per_step=1), PACKED)):
        J, _, st, _ = ctx.solve(precision=32, schedule="dataflow", **kw, **it)
        assert st["kernel_used"] == kernel, kw
        assert fp32_err(J, r["J"]) <= FP32_TOL, kw


# ---- the headline workload's kernel where its wide levels run -----------------------------------------
@pytest.fixture(scope="module")
def box18():
    return configs.periodic(n_cells=1 << 18)


@pytest.mark.parametrize("form", ["bench", "lines16"])
def test_headline_kernel_on_a_2p18_box(ctx, box18, form):
    # the periodic box of the benchmark at 2^18 cells x 128 directions (levels ~50x wider than the small
    # parity meshes): the benchmark's launch configuration (autotuned packed operator) and the 8-lane
    # pair form over 128-byte lines; every cell's J and Gamma after three periodic iterations against
    # the oracle's, every direction's levels bit-exact, conservation of the converged solve
    p = box18
    load(ctx, p)
    it = dict(tol_pbc=0.0, max_it_pbc=3)
    kw = dict(relevel=1) if form == "bench" else dict(relevel=1, op_format="lines", lanes_per_task=16,
                                                       schedule="dataflow")
    J, Gm, st, s = ctx.solve(precision=32, **kw, **it)
    assert st["kernel_used"] == (PACKED if form == "bench" else 6)
    r = run_oracle(p, **it)
    assert fp32_err(J, r["J"]) <= FP32_TOL
    assert fp32_err(Gm, r["Gamma"]) <= FP32_TOL
    if form == "bench":
        rc, lev, depth = oracle.levels(p.mesh, p.omega, threads=8)
        assert rc == 0
        for d in range(p.n_dir):
            gl, gd = ctx.levels(d)
            assert gd == depth[d] and np.array_equal(gl, lev[d]), d
    J, Gm, st, s = ctx.solve(precision=32, tol_pbc=1e-6, max_it_pbc=200, **kw)
    assert s == 0 and st["res_pbc"] < 1e-6
    assert abs(st["defect"]) <= DEFECT_TOL


# ---- the EXP law and the transposed (adjoint) sweep over packets -------------------------------------
@pytest.mark.parametrize("pps", [1, 2])
@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("kind", ["inflow", "periodic", "scatter"])
def test_packed_exp_law(ctx, kind, G, pps):
    # the EXP update in the packed kernel (intensity and cell mean per head lane): every intensity after
    # a fixed number of iterations, then J and conservation of the converged solve
    p = configs.voronoi_small(4000, periodic_box=kind == "periodic", n_dir=12, n_groups=G, seed=110 + G, n_src=8,
                              scatter_albedo=0.5 if kind == "scatter" else 0.0, bc_inflow=kind == "inflow")
    load(ctx, p)
    it = dict(tol_scat=0.0, max_it_scat=3, tol_pbc=0.0, max_it_pbc=3)
    J, Gm, st, _ = ctx.solve(precision=32, law="exp", packets_per_step=pps, **it)
    assert st["kernel_used"] == PACKED and st["lanes_used"] == 32 * pps
    r = run_oracle(p, law="exp", want_intensity=True, **it)
    for d in range(p.n_dir):
        assert fp32_err(ctx.intensity(d), r["I"][d]) <= FP32_TOL, d
    assert fp32_err(J, r["J"]) <= FP32_TOL and fp32_err(Gm, r["Gamma"]) <= FP32_TOL
    conv = dict(tol_scat=1e-7, max_it_scat=500, tol_pbc=1e-7, max_it_pbc=500)
    J, _, st, s = ctx.solve(precision=32, law="exp", packets_per_step=pps, **conv)
    assert s == 0 and abs(st["defect"]) <= DEFECT_TOL
    assert fp32_err(J, run_oracle(p, law="exp", **conv)["J"]) <= 2 * FP32_TOL


def _adjoint_pair(ctx, p, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=p.kappa_abs.shape), rng.normal(size=p.kappa_abs.shape)


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("pps", [1, 2])
@pytest.mark.parametrize("G", [1, 2])
@pytest.mark.parametrize("kind", ["vacuum", "periodic", "scatter"])
def test_packed_transposed_adjoint(ctx, kind, G, pps):
    # the transposed sweep over the packed transposed operator (outflow entries, levels streamed in
    # reverse, 2G split groups) against the oracle's adjoint, a fixed number of passes; and against the
    # FP32 mesh-row transposed sweep on the same context, which differs only in summation order
    p = configs.voronoi_small(4000, periodic_box=kind == "periodic", n_dir=12, n_groups=G, seed=120 + G, n_src=8,
                              scatter_albedo=0.5 if kind == "scatter" else 0.0)
    load(ctx, p)
    dj, dg = _adjoint_pair(ctx, p, 121)
    coupled = kind != "vacuum"
    fixed = dict(tol_scat=0.0, max_it_scat=3, tol_pbc=0.0, max_it_pbc=3, allow_not_converged=True) if coupled else {}
    kw = dict(dl_dJ=dj, dl_dGamma=dg, precision=32, schedule="dataflow", packets_per_step=pps, **fixed)
    out = ctx.adjoint(with_kappa_scat=coupled, **kw)
    st = out[-1]
    assert st["kernel_used"] == PACKED
    ks = p.kappa_scat if kind == "scatter" else np.zeros_like(p.kappa_abs)
    ofix = {k: v for k, v in fixed.items() if k != "allow_not_converged"}
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, dl_dJ=dj,
                            dl_dGamma=dg, threads=8, **ofix)
    # FP32 intensities, FP64 gradient accumulation: within 1e-6 of the largest gradient (measured: <= 2.4e-7)
    assert rel_max(out[0], r["grad_kappa_abs"]) <= 1e-6
    assert rel_max(out[1], r["grad_emissivity"]) <= 1e-6
    if coupled:
        assert rel_max(out[2], r["grad_kappa_scat"]) <= 1e-6
    ref = ctx.adjoint(with_kappa_scat=coupled, geometry_only=1, **kw)
    assert ref[-1]["kernel_used"] != PACKED
    for a, b in zip(out[:-1], ref[:-1]):
        assert rel_max(a, b) <= 1e-6
