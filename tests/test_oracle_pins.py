"""Pins of the FP64 oracle to facts other than itself (closed forms, identities, the paper's
Appendix A invariant, independent dense solves, brute force, finite differences)."""
import math

import numpy as np
import pytest

import oracle
from oracle import dense
from synth import configs
from synth.fields import fibonacci_directions
from synth.mesh import FACE_BOUNDARY, FACE_PERIODIC, column_mesh, lattice_mesh, voronoi_mesh

pytestmark = pytest.mark.filterwarnings("ignore")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---- (a) closed form of the discrete update along a 1-D column (Sec. 2.6 scheme (a)) ----------
@pytest.mark.parametrize("reverse", [False, True])
def test_column_closed_form_inflow(reverse):
    n, h, kap = 96, 1.0 / 64, 2.5
    p = configs.column(n, kappa=kap, h=h, reverse=reverse)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     want_intensity=True)
    assert r["rc"] == oracle.OK
    I = r["I"][0, :, 0]
    k = np.arange(n) if not reverse else np.arange(n)[::-1]
    exact = (1.0 + kap * h) ** (-(k + 1.0))  # each cell attenuates by 1/(1 + kappa h)
    assert rel(I, exact) <= 1e-14


def test_column_closed_form_source():
    n, h, kap, s = 80, 1.0 / 32, 1.7, 0.3
    p = configs.column(n, kappa=kap, h=h, source=s)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     want_intensity=True)
    I = r["I"][0, :, 0]
    A, tau = h * h, kap * h
    rr = 1.0 / (1.0 + tau)
    b = (s / (4 * math.pi)) / (A * (1.0 + tau))
    k = np.arange(n) + 1.0
    exact = rr ** k + b * (1.0 - rr ** k) / (1.0 - rr)
    assert rel(I, exact) <= 1e-14


def test_column_tie_faces_carry_no_flux():
    # the side faces have n.Omega = 0 exactly: neither upwind nor downwind (tie reading)
    p = configs.column(16, kappa=0.0)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     want_intensity=True)
    assert np.allclose(r["I"][0, :, 0], 1.0, rtol=0, atol=1e-15)
    rc, lev, depth = oracle.levels(p.mesh, p.omega)
    assert rc == 0 and depth[0] == 16 and np.array_equal(lev[0], np.arange(16))


# ---- (b) photon conservation: emitted + injected = absorbed + escaped ----------------------------
@pytest.mark.parametrize("periodic_box", [False, True])
def test_conservation(periodic_box):
    p = configs.voronoi_small(300, periodic_box=periodic_box, n_dir=12, n_groups=2, seed=3,
                              bc_inflow=not periodic_box)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     tol_pbc=1e-15, max_it_pbc=2000)
    st = r["stats"]
    src = st["emitted"] + st["injected"]
    assert abs(src - st["absorbed"] - st["escaped"]) <= 1e-12 * src
    assert abs(st["defect"]) <= 1e-12
    if periodic_box:
        assert st["escaped"] == 0.0 and st["it_pbc"] > 1


def test_conservation_with_scattering():
    p = configs.voronoi_small(250, n_dir=8, n_groups=1, seed=5, scatter_albedo=0.5)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                     tol_scat=1e-15, max_it_scat=3000)
    st = r["stats"]
    assert abs(st["defect"]) <= 1e-12
    assert st["it_scat"] > 2


def test_pure_streaming_escapes_everything():
    p = configs.voronoi_small(200, n_dir=10, seed=7)
    r = oracle.solve(p.mesh, p.omega, p.weight, np.zeros_like(p.kappa_abs), p.emissivity)
    st = r["stats"]
    assert st["absorbed"] == 0.0
    assert abs(st["escaped"] - st["emitted"]) <= 1e-13 * st["emitted"]


# ---- (c) Appendix A: sorting by Omega.x of the generators is a topological order ---------------
@pytest.mark.parametrize("periodic_box", [False, True])
def test_voronoi_invariant(periodic_box):
    rng = np.random.default_rng(11)
    m = voronoi_mesh(rng.random((500, 3)), periodic=periodic_box, threads=1)
    om, _ = fibonacci_directions(24, seed=2)
    rc, lev, depth = oracle.levels(m, om)
    assert rc == 0
    inner = m.flags == 0
    c0, c1 = m.face_cells[inner, 0], m.face_cells[inner, 1]
    for d in range(om.shape[0]):
        x = m.points @ om[d]
        up_is_c0 = lev[d, c1] > lev[d, c0]
        up = np.where(up_is_c0, c0, c1)
        down = np.where(up_is_c0, c1, c0)
        # every dependency runs from lower to higher Omega.x of the generators ...
        assert np.all(x[down] > x[up])
        # ... so sorting the cells by Omega.x gives a valid order: each cell after its upwind cells
        order = np.argsort(x, kind="stable")
        pos = np.empty_like(order)
        pos[order] = np.arange(order.size)
        assert np.all(pos[down] > pos[up])
        assert np.all(lev[d, c0] != lev[d, c1])


# ---- levels: brute-force longest paths on the dependency graph ---------------------------------
def _longest_paths(m, om):
    t = (m.normal[:, 0] * om[0] + m.normal[:, 1] * om[1]) + m.normal[:, 2] * om[2]
    succ = [[] for _ in range(m.n_cells)]
    pred = [[] for _ in range(m.n_cells)]
    for f in range(m.n_faces):
        if m.flags[f] & (FACE_BOUNDARY | FACE_PERIODIC) or t[f] == 0.0:
            continue
        a, b = int(m.face_cells[f, 0]), int(m.face_cells[f, 1])
        if t[f] < 0:
            a, b = b, a
        succ[a].append(b)
        pred[b].append(a)
    memo = {}

    def depth_to(c):  # longest path ending at c (recursion over predecessors)
        if c in memo:
            return memo[c]
        v = 0 if not pred[c] else 1 + max(depth_to(u) for u in pred[c])
        memo[c] = v
        return v

    import sys
    sys.setrecursionlimit(100000)
    return np.array([depth_to(c) for c in range(m.n_cells)])


@pytest.mark.parametrize("kind", ["voronoi", "lattice", "periodic"])
def test_levels_brute_force(kind):
    if kind == "lattice":
        m = lattice_mesh(7)
    else:
        rng = np.random.default_rng(4)
        m = voronoi_mesh(rng.random((400, 3)), periodic=kind == "periodic", threads=1)
    om, _ = fibonacci_directions(6, seed=9)
    rc, lev, depth = oracle.levels(m, om)
    assert rc == 0
    for d in range(om.shape[0]):
        bf = _longest_paths(m, om[d])
        assert np.array_equal(bf, lev[d])
        assert depth[d] == bf.max() + 1


def test_lattice_depth_axis_direction():
    m = lattice_mesh(9)
    rc, lev, depth = oracle.levels(m, np.array([[0.0, 0.0, 1.0]]))
    # Omega = +z: x and y faces are exact ties, the graph is 81 independent columns of 9
    assert rc == 0 and depth[0] == 9
    assert np.array_equal(lev[0], np.repeat(np.arange(9), 81))


def test_cycle_detected():
    # a ring of cells whose closing face is marked interior instead of periodic is cyclic
    m = column_mesh(6, periodic_x=True)
    m.flags = m.flags.copy()
    m.flags[m.flags == FACE_PERIODIC] = 0
    rc, _, _ = oracle.levels(m, np.array([[1.0, 0.0, 0.0]]))
    assert rc == oracle.ERR_CYCLE


# ---- (d) dense LU solves of L_Omega I = S ---------------------------------------------------------
@pytest.mark.parametrize("G", [1, 3])
def test_dense_plain(G):
    p = configs.voronoi_small(350, n_dir=6, n_groups=G, seed=21, bc_inflow=True)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     want_intensity=True)
    for d in range(p.n_dir):
        Id = dense.solve_direction(p.mesh, p.omega[d], p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow)
        assert rel(r["I"][d], Id) <= 1e-12


def test_dense_scattering_fixed_point():
    p = configs.voronoi_small(150, n_dir=6, n_groups=2, seed=23, scatter_albedo=0.6)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                     tol_scat=1e-15, max_it_scat=5000)
    _, Jd, Gd = dense.solve_coupled(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, p.kappa_scat)
    assert rel(r["J"], Jd) <= 1e-12
    assert rel(r["Gamma"], Gd) <= 1e-12


def test_dense_periodic_fixed_point():
    p = configs.voronoi_small(200, periodic_box=True, n_dir=6, n_groups=1, seed=25)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, tol_pbc=1e-15, max_it_pbc=5000)
    _, Jd, _ = dense.solve_coupled(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity)
    assert rel(r["J"], Jd) <= 1e-12


@pytest.mark.parametrize("fused", [False, True])
def test_dense_periodic_scattering_fixed_point(fused):
    # both couplings at once: the nested loops and the fused loop (one source-iteration sweep per
    # periodic iteration, Sec. 2.7) reach the same fixed point, the dense solve of the whole system
    p = configs.voronoi_small(200, periodic_box=True, n_dir=6, n_groups=2, seed=29, scatter_albedo=0.5)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                     tol_scat=1e-15, max_it_scat=3000, tol_pbc=1e-15, max_it_pbc=5000, fused=fused)
    assert r["rc"] == 0
    _, Jd, Gd = dense.solve_coupled(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, p.kappa_scat)
    assert rel(r["J"], Jd) <= 1e-12
    assert rel(r["Gamma"], Gd) <= 1e-12
    st = r["stats"]
    if fused:
        # one sweep per periodic iteration
        assert st["it_scat"] == st["it_pbc"]
    else:
        assert st["it_scat"] > st["it_pbc"]


def test_fused_loop_needs_both_couplings():
    # with only one coupling present the fused option changes nothing, sweep for sweep
    for box, alb in ((True, 0.0), (False, 0.5)):
        p = configs.voronoi_small(150, periodic_box=box, n_dir=6, n_groups=1, seed=31, scatter_albedo=alb)
        ks = p.kappa_scat if alb else None
        a = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, fused=False)
        b = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, fused=True)
        assert np.array_equal(a["J"], b["J"]) and a["stats"] == b["stats"]


def test_uniform_periodic_fixed_point():
    # eps_c = C kappa_a,c V_c with closed cells: I = C/(4pi) in every direction solves the balance
    p = configs.voronoi_small(300, periodic_box=True, n_dir=8, seed=27)
    C = 2.0
    eps = C * p.kappa_abs * p.mesh.volume[:, None]
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, eps, tol_pbc=1e-15, max_it_pbc=5000,
                     want_intensity=True)
    assert np.max(np.abs(r["I"] - C / (4 * math.pi))) <= 1e-12 * C
    # with scattering the same state is the fixed point of both iterations
    r2 = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, eps, kappa_scat=0.7 * p.kappa_abs, tol_scat=1e-15,
                      max_it_scat=3000, tol_pbc=1e-14, max_it_pbc=3000)
    assert np.max(np.abs(r2["J"] - C / (4 * math.pi))) <= 1e-11 * C


@pytest.mark.parametrize("law,dc_n", [("balance", 0), ("exp", 0), ("balance", 3), ("exp", 3)])
def test_linearity_in_sources(law, dc_n):
    # every law and scheme is a linear system in the sources
    p = configs.voronoi_small(250, n_dir=8, n_groups=2, seed=29, scatter_albedo=0.3)
    rng = np.random.default_rng(1)
    e1 = rng.random(p.emissivity.shape) * (rng.random(p.emissivity.shape) < 0.1)
    e2 = rng.random(p.emissivity.shape) * (rng.random(p.emissivity.shape) < 0.1)
    kw = dict(kappa_scat=p.kappa_scat, tol_scat=1e-15, max_it_scat=4000, law=law, dc_n=dc_n)
    J1 = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, e1, **kw)["J"]
    J2 = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, e2, **kw)["J"]
    J12 = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, e1 + e2, **kw)["J"]
    assert rel(J12, J1 + J2) <= 1e-13


def test_plain32_lattice_solution_is_symmetric_under_the_source():
    # unit source at (16,16,16) in a 32^3 lattice: conservation and total photon budget
    p = configs.plain32()
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, threads=4)
    st = r["stats"]
    assert st["emitted"] == pytest.approx(1.0, rel=1e-15)
    assert abs(st["defect"]) <= 1e-12
    assert r["J"][p.info["source_cell"], 0] == r["J"].max()


# ---- adjoint: reciprocity, dense transposed solve, finite differences -----------------------------
def test_adjoint_reciprocity():
    # BALANCE law: L_{-Omega} = L_Omega^T, so dJ/deps (adjoint with directions Omega and dL/dJ = r)
    # equals the forward mean intensity for directions -Omega with emissivity r
    p = configs.voronoi_small(300, n_dir=10, n_groups=2, seed=31)
    rng = np.random.default_rng(2)
    r_ = rng.random(p.emissivity.shape)
    rc, gk, ge = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dl_dJ=r_)
    assert rc == 0
    Jrev = oracle.solve(p.mesh, -p.omega, p.weight, p.kappa_abs, r_)["J"]
    assert rel(ge, Jrev) <= 1e-12


def test_adjoint_dense_transpose():
    p = configs.voronoi_small(200, n_dir=5, n_groups=1, seed=33)
    rng = np.random.default_rng(3)
    dg = rng.normal(size=p.kappa_abs.shape)
    rc, gk, ge = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dl_dGamma=dg)
    ge_d = np.zeros_like(ge)
    gk_d = np.zeros_like(gk)
    V = p.mesh.volume[:, None]
    for d in range(p.n_dir):
        I = dense.solve_direction(p.mesh, p.omega[d], p.kappa_abs, p.emissivity)
        g = p.weight[d] * dg * p.kappa_abs * V
        lam = dense.adjoint_direction(p.mesh, p.omega[d], p.kappa_abs, g)
        ge_d += lam / (4 * math.pi)
        gk_d += V * I * (p.weight[d] * dg - lam)
    assert rel(ge, ge_d) <= 1e-11
    assert rel(gk, gk_d) <= 1e-11


def test_adjoint_finite_differences():
    # the 2^12-cell differentiation sub-mesh
    p = configs.voronoi_small(4096, n_dir=8, n_groups=2, seed=35)
    rng = np.random.default_rng(4)
    T = rng.random(p.kappa_abs.shape) * 1e-3

    def loss(ka, em):
        r = oracle.solve(p.mesh, p.omega, p.weight, ka, em)
        # exact summation: the loss difference of two nearby inputs is not drowned by rounding of the sum
        return math.fsum(((r["Gamma"] - T) ** 2).ravel()), r["Gamma"]

    L0, G0 = loss(p.kappa_abs, p.emissivity)
    rc, gk, ge = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dl_dGamma=2 * (G0 - T))
    assert rc == 0
    # central differences, step 1e-4 relative: truncation ~1e-8, rounding ~1e-15 / step
    big = np.argsort(np.abs(gk[:, 0]))[-40:]
    for c in rng.choice(big, 6, replace=False):
        for g in range(2):
            h = 1e-4 * p.kappa_abs[c, g]
            kp, km = p.kappa_abs.copy(), p.kappa_abs.copy()
            kp[c, g] += h
            km[c, g] -= h
            fd = (loss(kp, p.emissivity)[0] - loss(km, p.emissivity)[0]) / (2 * h)
            assert gk[c, g] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gk).max())
            he = 1e-4 * max(p.emissivity[c, g], 1.0)
            ep, emn = p.emissivity.copy(), p.emissivity.copy()
            ep[c, g] += he
            emn[c, g] -= he
            fde = (loss(p.kappa_abs, ep)[0] - loss(p.kappa_abs, emn)[0]) / (2 * he)
            assert ge[c, g] == pytest.approx(fde, rel=1e-6, abs=1e-7 * np.abs(ge).max())


def test_invalid_inputs_rejected():
    p = configs.voronoi_small(50, n_dir=4, seed=1)
    m = p.mesh
    bad = m.face_cells.copy()
    bad[0, 0] = m.n_cells + 5
    from synth.mesh import Mesh
    mb = Mesh(volume=m.volume, face_cells=bad, area=m.area, normal=m.normal, flags=m.flags)
    assert oracle.solve(mb, p.omega, p.weight, p.kappa_abs, p.emissivity)["rc"] == oracle.ERR_ARG


def test_oracle_matches_stored_plain32_golden():
    # tests/golden/oracle_plain32.json was written by tests/golden/make_oracle_golden.py (oracle only);
    # its depths are also the lattice closed form 3(n-1)+1 for directions with no zero component, and its
    # absorbed plus escaped rate is the unit source (vacuum conservation)
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_plain32.json")) as f:
        g = json.load(f)
    p = configs.plain32()
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, threads=4)
    assert np.allclose(r["J"][g["cells"], 0], g["J"], rtol=1e-13, atol=0)
    assert np.allclose(r["Gamma"][g["cells"], 0], g["Gamma"], rtol=1e-13, atol=0)
    assert g["Gamma_total"] + g["escaped"] == pytest.approx(1.0, abs=1e-12)
    assert np.all(np.abs(p.omega) > 0)
    assert g["depths"] == [3 * 31 + 1] * p.n_dir
    rc, _, depth = oracle.levels(p.mesh, p.omega)
    assert rc == 0 and list(depth) == g["depths"]


# ---- (f) the adjoint through the source iteration (scattering) ------------------------------------
def _scat_problem(n=300, seed=37):
    return configs.voronoi_small(n, n_dir=8, n_groups=2, seed=seed, scatter_albedo=0.5, n_src=6)


def test_adjoint_scattering_dense_transpose():
    # lambda of the transposed source iteration is the solution of A^T lambda = dL/dI for the whole
    # coupled system (every direction and the scattering coupling in one dense matrix)
    p = _scat_problem(200, 39)
    rng = np.random.default_rng(5)
    dg = rng.normal(size=p.kappa_abs.shape)
    dj = rng.normal(size=p.kappa_abs.shape)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                            dl_dJ=dj, dl_dGamma=dg, tol_scat=1e-15, max_it_scat=5000)
    assert r["rc"] == 0 and r["it_adjoint"] > 1
    V = p.mesh.volume[:, None]
    gsrc = p.weight[:, None, None] * (dg * p.kappa_abs * V + dj / (4 * math.pi))[None]
    lam = dense.adjoint_coupled(p.mesh, p.omega, p.weight, p.kappa_abs, p.kappa_scat, gsrc)
    assert rel(r["grad_emissivity"], lam.sum(axis=0) / (4 * math.pi)) <= 1e-11


def test_adjoint_scattering_finite_differences():
    p = _scat_problem()
    rng = np.random.default_rng(6)
    T = rng.random(p.kappa_abs.shape) * np.median(p.emissivity[p.emissivity > 0])
    rJ = rng.normal(size=p.kappa_abs.shape)
    kw = dict(tol_scat=1e-15, max_it_scat=5000)

    def loss(ka, em, ks):
        r = oracle.solve(p.mesh, p.omega, p.weight, ka, em, kappa_scat=ks, **kw)
        assert r["rc"] == 0
        return math.fsum(((r["Gamma"] - T) ** 2).ravel()) + math.fsum((rJ * r["J"]).ravel()), r["Gamma"]

    _, G0 = loss(p.kappa_abs, p.emissivity, p.kappa_scat)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                            dl_dJ=rJ, dl_dGamma=2 * (G0 - T), **kw)
    assert r["rc"] == 0
    grads = {"ka": r["grad_kappa_abs"], "em": r["grad_emissivity"], "ks": r["grad_kappa_scat"]}
    base = {"ka": p.kappa_abs, "em": p.emissivity, "ks": p.kappa_scat}
    for name, gr in grads.items():
        big = np.argsort(np.abs(gr).ravel())[-30:]
        for flat in rng.choice(big, 4, replace=False):
            c, g = divmod(int(flat), p.n_groups)
            h = 1e-4 * max(base[name][c, g], 1e-3 * base[name].max())
            args_p = {k: v.copy() for k, v in base.items()}
            args_m = {k: v.copy() for k, v in base.items()}
            args_p[name][c, g] += h
            args_m[name][c, g] -= h
            fd = (loss(args_p["ka"], args_p["em"], args_p["ks"])[0]
                  - loss(args_m["ka"], args_m["em"], args_m["ks"])[0]) / (2 * h)
            assert gr[c, g] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(gr).max()), (name, c, g)


def test_adjoint_without_scattering_is_one_transposed_sweep():
    p = configs.voronoi_small(300, n_dir=8, n_groups=2, seed=41)
    rng = np.random.default_rng(7)
    dg = rng.normal(size=p.kappa_abs.shape)
    rc, gk, ge = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dl_dGamma=dg)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity,
                            kappa_scat=np.zeros_like(p.kappa_abs), dl_dGamma=dg)
    assert r["it_forward"] == r["it_adjoint"] == 1
    assert np.array_equal(r["grad_kappa_abs"], gk) and np.array_equal(r["grad_emissivity"], ge)


# ---- (g) the adjoint through the periodic iteration ---------------------------------------------
@pytest.mark.parametrize("albedo", [0.0, 0.5])
def test_adjoint_periodic_dense_transpose(albedo):
    # the transposed iteration reads the partner's lambda across periodic outflow sides: its fixed
    # point is the transposed solve of the whole system with the periodic coupling in the matrix
    p = configs.voronoi_small(200, periodic_box=True, n_dir=6, n_groups=2, seed=43, scatter_albedo=albedo)
    ks = p.kappa_scat if albedo else np.zeros_like(p.kappa_abs)
    rng = np.random.default_rng(8)
    dg = rng.normal(size=p.kappa_abs.shape)
    dj = rng.normal(size=p.kappa_abs.shape)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, dl_dJ=dj,
                            dl_dGamma=dg, tol_scat=1e-15, max_it_scat=5000, tol_pbc=1e-15, max_it_pbc=5000)
    assert r["rc"] == 0 and r["it_adjoint"] > 1
    V = p.mesh.volume[:, None]
    gsrc = p.weight[:, None, None] * (dg * p.kappa_abs * V + dj / (4 * math.pi))[None]
    lam = dense.adjoint_coupled(p.mesh, p.omega, p.weight, p.kappa_abs, ks, gsrc)
    assert rel(r["grad_emissivity"], lam.sum(axis=0) / (4 * math.pi)) <= 1e-11


@pytest.mark.parametrize("albedo", [0.0, 0.5])
def test_adjoint_periodic_finite_differences(albedo):
    p = configs.voronoi_small(300, periodic_box=True, n_dir=8, n_groups=1, seed=45, scatter_albedo=albedo,
                              n_src=6)
    ks = p.kappa_scat if albedo else np.zeros_like(p.kappa_abs)
    rng = np.random.default_rng(9)
    T = rng.random(p.kappa_abs.shape) * np.median(p.emissivity[p.emissivity > 0])
    kw = dict(tol_scat=1e-15, max_it_scat=5000, tol_pbc=1e-15, max_it_pbc=5000)

    def loss(ka, em, k_s):
        # the fused loops reach the nested loops' fixed point in far fewer sweeps
        r = oracle.solve(p.mesh, p.omega, p.weight, ka, em, kappa_scat=k_s, fused=bool(albedo), threads=4, **kw)
        assert r["rc"] == 0
        return math.fsum(((r["Gamma"] - T) ** 2).ravel()), r["Gamma"]

    _, G0 = loss(p.kappa_abs, p.emissivity, ks)
    r = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks,
                            dl_dGamma=2 * (G0 - T), **kw)
    assert r["rc"] == 0
    grads = {"ka": r["grad_kappa_abs"], "em": r["grad_emissivity"]}
    base = {"ka": p.kappa_abs, "em": p.emissivity, "ks": ks}
    if albedo:
        grads["ks"] = r["grad_kappa_scat"]
    for name, gr in grads.items():
        big = np.argsort(np.abs(gr).ravel())[-30:]
        for c in rng.choice(big, 4, replace=False):
            h = 1e-4 * max(base[name][c, 0], 1e-3 * base[name].max())
            a_p = {k: v.copy() for k, v in base.items()}
            a_m = {k: v.copy() for k, v in base.items()}
            a_p[name][c, 0] += h
            a_m[name][c, 0] -= h
            fd = (loss(a_p["ka"], a_p["em"], a_p["ks"])[0] - loss(a_m["ka"], a_m["em"], a_m["ks"])[0]) / (2 * h)
            assert gr[c, 0] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(gr).max()), (name, c)


# ---- (h) the EXP law: exact attenuation through each cell's mean chord ---------------------------
def test_exp_column_is_the_exact_transport_solution():
    # along a column of cubes the mean chord V/P is the cell length h, so the EXP update is exact:
    # the outgoing intensity of cell k is exp(-kappa (k+1) h) and the cell mean is the chord average
    # of exp(-kappa x) over the cell, (1/h) int_kh^(k+1)h exp(-kappa x) dx
    n, h, kap = 96, 1.0 / 64, 2.5
    p = configs.column(n, kappa=kap, h=h)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     want_intensity=True, law="exp")
    assert r["rc"] == oracle.OK
    k = np.arange(n)
    assert rel(r["I"][0, :, 0], np.exp(-kap * h * (k + 1.0))) <= 1e-14
    mean = (np.exp(-kap * h * k) - np.exp(-kap * h * (k + 1.0))) / (kap * h)
    # one direction of weight 4pi: J is the cell mean itself
    assert rel(r["J"][:, 0], mean) <= 1e-14
    st = r["stats"]
    assert abs(st["defect"]) <= 1e-14


def test_exp_column_with_sources():
    # the cell's own emission leaves unattenuated: I_k = r I_(k-1) + q / A with r = exp(-kappa h)
    n, h, kap, s = 80, 1.0 / 32, 1.7, 0.3
    p = configs.column(n, kappa=kap, h=h, source=s)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, bc_inflow=p.boundary_inflow,
                     want_intensity=True, law="exp")
    A, rr = h * h, math.exp(-kap * h)
    b = (s / (4 * math.pi)) / A
    k = np.arange(n) + 1.0
    assert rel(r["I"][0, :, 0], rr ** k + b * (1.0 - rr ** k) / (1.0 - rr)) <= 1e-13


@pytest.mark.parametrize("box,albedo", [(False, 0.0), (False, 0.6), (True, 0.0), (True, 0.5)])
def test_exp_dense_and_conservation(box, albedo):
    p = configs.voronoi_small(150, periodic_box=box, n_dir=6, n_groups=2, seed=47, scatter_albedo=albedo,
                              bc_inflow=not box)
    ks = p.kappa_scat if albedo else None
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks,
                     bc_inflow=p.boundary_inflow, tol_scat=1e-15, max_it_scat=5000, tol_pbc=1e-15, max_it_pbc=5000,
                     want_intensity=True, law="exp")
    assert r["rc"] == 0
    I, _, J, Gam = dense.solve_coupled_exp(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, ks,
                                           p.boundary_inflow)
    assert rel(r["I"], I) <= 1e-11
    assert rel(r["J"], J) <= 1e-11 and rel(r["Gamma"], Gam) <= 1e-11
    assert abs(r["stats"]["defect"]) <= 1e-12


def test_exp_and_balance_agree_when_thin_away_from_sources():
    # in an optically thin medium both laws stream the radiation unchanged, so the cells without a
    # source see the same J; a source cell's J differs by its own emission, which BALANCE counts in
    # the cell and EXP lets leave unattenuated
    p = configs.voronoi_small(200, n_dir=6, n_groups=1, seed=49)
    free = p.emissivity[:, 0] == 0.0
    assert free.any() and not free.all()
    a = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity)
    b = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, law="exp")
    assert rel(a["J"][free], b["J"][free]) > 1e-3
    thin = p.kappa_abs * 1e-7
    a = oracle.solve(p.mesh, p.omega, p.weight, thin, p.emissivity)
    b = oracle.solve(p.mesh, p.omega, p.weight, thin, p.emissivity, law="exp")
    assert rel(a["J"][free], b["J"][free]) <= 1e-5


# ---- (i) direction-conserving transport, scheme (b) of Sec. 2.6 ---------------------------------
def test_dc_equals_scheme_a_on_the_lattice_diagonal():
    # along a body diagonal every cube has three outflow faces with the same area and n . Omega:
    # both schemes split the outflow in equal thirds, and choose the same faces
    m = lattice_mesh(7)
    om = np.array([[s1, s2, s3] for s1 in (1, -1) for s2 in (1, -1) for s3 in (1, -1)], float) / math.sqrt(3.0)
    assert np.all(om[:, 0] ** 2 == om[:, 1] ** 2) and np.all(om[:, 1] ** 2 == om[:, 2] ** 2)
    w = np.full(len(om), 4 * math.pi / len(om))
    rng = np.random.default_rng(10)
    ka = rng.random((m.n_cells, 1)) * 5
    em = rng.random((m.n_cells, 1))
    a = oracle.solve(m, om, w, ka, em, want_intensity=True)
    b = oracle.solve(m, om, w, ka, em, want_intensity=True, dc_n=3)
    assert rel(a["I"], b["I"]) <= 1e-14
    assert np.array_equal(oracle.levels(m, om)[1], oracle.levels(m, om, dc_n=3)[1])


@pytest.mark.parametrize("n_dc", [1, 3])
@pytest.mark.parametrize("box,albedo", [(False, 0.0), (False, 0.5), (True, 0.0), (True, 0.5)])
def test_dc_dense_and_conservation(n_dc, box, albedo):
    p = configs.voronoi_small(150, periodic_box=box, n_dir=6, n_groups=2, seed=51, scatter_albedo=albedo,
                              bc_inflow=not box)
    ks = p.kappa_scat if albedo else None
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks,
                     bc_inflow=p.boundary_inflow, tol_scat=1e-15, max_it_scat=5000, tol_pbc=1e-15, max_it_pbc=5000,
                     want_intensity=True, dc_n=n_dc)
    assert r["rc"] == 0
    I, J, Gam = dense.solve_coupled_dc(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, n_dc, ks,
                                       p.boundary_inflow)
    assert rel(r["I"], I) <= 1e-11
    assert rel(r["J"], J) <= 1e-11 and rel(r["Gamma"], Gam) <= 1e-11
    assert abs(r["stats"]["defect"]) <= 1e-12


def test_dc_thins_the_dependency_graph():
    # Sec. 2.6: direction-conserving transport to 3 neighbours cuts the downwind dependencies per cell
    # from about 15.54 / 2 to 3; its wavefront levels are the longest paths of the thinner graph, so
    # no cell sits deeper than under scheme (a)
    p = configs.voronoi_small(400, n_dir=4, n_groups=1, seed=53)
    m = p.mesh
    na = nd = 0
    rc_a, lev_a, _ = oracle.levels(m, p.omega)
    rc_b, lev_b, _ = oracle.levels(m, p.omega, dc_n=3)
    assert rc_a == rc_b == 0
    for d in range(p.n_dir):
        _, _, deps = dense.dc_operator(m, p.omega[d], p.kappa_abs, 3)
        _, _, deps_a = dense.dc_operator(m, p.omega[d], p.kappa_abs, 10 ** 6)
        nd += sum(len(v) for v in deps.values())
        na += sum(len(v) for v in deps_a.values())
        # brute-force longest paths of the scheme (b) graph
        lev = np.zeros(m.n_cells, np.int64)
        for _ in range(m.n_cells):
            changed = False
            for u, vs in deps.items():
                for v in vs:
                    if lev[v] < lev[u] + 1:
                        lev[v] = lev[u] + 1
                        changed = True
            if not changed:
                break
        assert np.array_equal(lev_b[d], lev)
        assert np.all(lev_b[d] <= lev_a[d])
    assert nd / (p.n_dir * m.n_cells) <= 3.0 < na / (p.n_dir * m.n_cells)


def test_dc_downwind_counts_match_the_paper():
    # in a periodic Voronoi box (no boundary) each cell has 15.54 neighbours on average, half of them
    # downwind under scheme (a); scheme (b) hands flux to exactly 3 of them (Sec. 2.6,
    # tests/golden/paper_values.json)
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        gold = json.load(f)
    p = configs.voronoi_small(2000, periodic_box=True, n_dir=4, n_groups=1, seed=53)
    m = p.mesh
    assert (m.face_cells[:, 1] >= 0).all()
    down_a = down_b = 0
    for d in range(p.n_dir):
        L, _, _ = dense.dc_operator(m, p.omega[d], p.kappa_abs, 3)
        La, _, _ = dense.dc_operator(m, p.omega[d], p.kappa_abs, 10 ** 6)
        off = ~np.eye(m.n_cells, dtype=bool)
        down_b += int(((L != 0) & off).sum())  # one entry per (chosen face) downwind pair
        down_a += int(((La != 0) & off).sum())
    per_b = down_b / (p.n_dir * m.n_cells)
    per_a = down_a / (p.n_dir * m.n_cells)
    g = gold["scheme_a_downwind_per_cell"]
    assert abs(per_a - g["value"]) <= g["abs_tol"]
    assert abs(per_b - gold["dc_downwind_per_cell"]["value"]) <= 0.01


@pytest.mark.parametrize("box,albedo", [(False, 0.5), (True, 0.5)])
def test_dc_with_the_exp_law(box, albedo):
    # the two options combine: scheme (b) decides where the outflow goes, the EXP law how much of
    # the inflow crosses the cell
    p = configs.voronoi_small(150, periodic_box=box, n_dir=6, n_groups=1, seed=51, scatter_albedo=albedo,
                              bc_inflow=not box)
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=p.kappa_scat,
                     bc_inflow=p.boundary_inflow, tol_scat=1e-15, max_it_scat=5000, tol_pbc=1e-15, max_it_pbc=5000,
                     want_intensity=True, law="exp", dc_n=3)
    assert r["rc"] == 0
    I, _, J, Gam = dense.solve_coupled_exp(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, p.kappa_scat,
                                           p.boundary_inflow, dc_n=3)
    assert rel(r["I"], I) <= 1e-11 and rel(r["J"], J) <= 1e-11
    assert abs(r["stats"]["defect"]) <= 1e-12


@pytest.mark.parametrize("seed,box", [(s, False) for s in range(61, 73)] + [(s, True) for s in range(61, 67)])
def test_every_option_against_its_dense_solve(seed, box):
    # several small meshes, every combination of law, transport scheme and scattering, against the
    # dense solve of the same system; conservation throughout
    p = configs.voronoi_small(150 if box else 90, periodic_box=box, n_dir=4, n_groups=1, seed=seed,
                              scatter_albedo=0.4, bc_inflow=not box)
    kw = dict(bc_inflow=p.boundary_inflow, tol_scat=1e-15, max_it_scat=5000, tol_pbc=1e-15, max_it_pbc=5000,
              want_intensity=True)
    for law in ("balance", "exp"):
        for dc_n in (0, 2, 3):
            for ks in (None, p.kappa_scat):
                r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=ks, law=law,
                                 dc_n=dc_n, **kw)
                assert r["rc"] == 0
                if law == "exp":
                    I = dense.solve_coupled_exp(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, ks,
                                                p.boundary_inflow, dc_n=dc_n)[0]
                elif dc_n:
                    I = dense.solve_coupled_dc(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dc_n, ks,
                                               p.boundary_inflow)[0]
                else:
                    I = dense.solve_coupled(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, ks,
                                            p.boundary_inflow)[0]
                assert rel(r["I"], I) <= 1e-11, (law, dc_n, ks is not None)
                assert abs(r["stats"]["defect"]) <= 1e-12



# ---- remap coefficients of a rotated direction set (Sec. 2.6, the rotation paragraph) ---------------------
def test_remap_identity_and_row_sums():
    om, _ = fibonacci_directions(24, seed=4)
    assert np.array_equal(oracle.remap_coeffs(om, om), np.eye(24))
    c = oracle.remap_coeffs(om, oracle.rotate(om, oracle.rotation(0.7, 2.1)))
    assert (c >= 0).all()
    assert np.max(np.abs(c.sum(1) - 1.0)) <= 1e-14
    assert np.count_nonzero(c) < 24 * 10  # a rotated bin overlaps only a few old bins


def test_remap_two_antipodal_directions():
    # the bins of +z and -z are the hemispheres; a quarter turn about x makes the new bins the hemispheres
    # of -y and +y, each of which shares exactly half of its solid angle with each old bin
    om = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    R = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])
    c = oracle.remap_coeffs(om, oracle.rotate(om, R))
    assert np.max(np.abs(c - 0.5)) <= 1e-3


def test_remap_of_a_symmetry_is_a_permutation():
    # a quarter turn about z maps the six axis directions onto themselves: the bins coincide
    om = np.concatenate([np.eye(3), -np.eye(3)])
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    new = oracle.rotate(om, R)
    perm = np.array([int(np.argmax(om @ v)) for v in new])
    c = oracle.remap_coeffs(om, new)
    assert np.array_equal(c, np.eye(6)[perm])


def test_remap_against_monte_carlo():
    # brute force with independent code: random points on the sphere, each in the bin of its nearest
    # direction of either set
    om, _ = fibonacci_directions(16, seed=2)
    new = oracle.rotate(om, oracle.rotation(1.1, 4.0))
    c = oracle.remap_coeffs(om, new, n_quad=1 << 18)
    rng = np.random.default_rng(3)
    p = rng.normal(size=(1_000_000, 3))
    p /= np.linalg.norm(p, axis=1)[:, None]
    i = np.argmax(p @ new.T, axis=1)
    j = np.argmax(p @ om.T, axis=1)
    cnt = np.zeros((16, 16))
    np.add.at(cnt, (i, j), 1.0)
    mc = cnt / cnt.sum(1, keepdims=True)
    assert np.max(np.abs(c - mc)) <= 6e-3
