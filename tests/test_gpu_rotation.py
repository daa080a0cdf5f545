"""GPU parity of the rotation of the direction set with the remap of the intensities (Sec. 2.6, the
rotation paragraph; sweep_rotate_directions) against the FP64 oracle (oracle.remap_coeffs, and
oracle.solve started from the remapped intensities)."""
import numpy as np
import pytest

import oracle
from synth import configs

pytestmark = pytest.mark.gpu


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def fp32_err(x, ref):
    m = ref >= 1e-30 * ref.max()
    return float(np.max(np.abs(x[m] - ref[m]) / ref[m]))


def load(ctx, p, scale=1.0):
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ctx.set_material(p.kappa_abs, p.emissivity * scale, kappa_scat=p.kappa_scat)


def intensities(ctx, n_dir):
    return np.stack([ctx.intensity(d) for d in range(n_dir)])


@pytest.mark.parametrize("precision", [64, 32])
def test_remap_matches_the_oracle(ctx, precision):
    p = configs.voronoi_small(3000, periodic_box=True, n_dir=16, n_groups=2, seed=110, n_src=8)
    load(ctx, p)
    ctx.solve(precision=precision, tol_pbc=0.0, max_it_pbc=3)
    I0 = intensities(ctx, p.n_dir)
    R = oracle.rotation(0.9, 2.3)
    ctx.rotate_directions(R)
    c = oracle.remap_coeffs(p.omega, oracle.rotate(p.omega, R))
    expect = np.einsum("ij,jng->ing", c, I0)
    got = intensities(ctx, p.n_dir)
    if precision == 64:
        assert rel_max(got, expect) <= 1e-13
    else:  # FP32 values remapped in FP64 and rounded once
        m = expect > 0
        assert np.max(np.abs(got[m] - expect[m]) / expect[m]) <= 1.2e-7
        assert np.array_equal(got[~m], expect[~m])


def test_identity_rotation_changes_nothing(ctx):
    p = configs.voronoi_small(2000, periodic_box=True, n_dir=8, seed=111, n_src=6)
    load(ctx, p)
    J0, _, st0, _ = ctx.solve(precision=64, tol_pbc=0.0, max_it_pbc=2)
    I0 = intensities(ctx, p.n_dir)
    ctx.rotate_directions(np.eye(3))
    assert np.array_equal(intensities(ctx, p.n_dir), I0)
    J1, _, st1, _ = ctx.solve(precision=64, tol_pbc=0.0, max_it_pbc=2)
    assert np.array_equal(J1, J0) and st1["depth_max"] == st0["depth_max"]


@pytest.mark.parametrize("precision", [64, 32])
def test_warm_started_rotated_solve_matches_the_oracle(ctx, precision):
    # a converged solve, a rotation with the remap, then three periodic iterations started from the remapped
    # intensities; the oracle does the same from its own converged intensities and the same coefficients
    p = configs.voronoi_small(3000, periodic_box=True, n_dir=12, n_groups=1, seed=112, n_src=8)
    load(ctx, p)
    conv = dict(tol_pbc=1e-12, max_it_pbc=1000)
    ctx.solve(precision=precision, **conv)
    r0 = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, want_intensity=True, threads=8, **conv)
    R = oracle.rotation(2.0, 0.4)
    ctx.rotate_directions(R)
    om2 = oracle.rotate(p.omega, R)
    prev = np.einsum("ij,jng->ing", oracle.remap_coeffs(p.omega, om2), r0["I"])
    it = dict(tol_pbc=0.0, max_it_pbc=3)
    J, Gm, st, s = ctx.solve(precision=precision, warm_start=1, **it)
    r = oracle.solve(p.mesh, om2, p.weight, p.kappa_abs, p.emissivity, prev_init=prev, threads=8, **it)
    if precision == 64:
        assert rel_max(J, r["J"]) <= 1e-10 and rel_max(Gm, r["Gamma"]) <= 1e-10
    else:
        assert fp32_err(J, r["J"]) <= 1e-5


def test_rotated_substeps(ctx):
    # N_rot substeps with the sources divided by N_rot and a random rotation (theta in [0, pi], phi in
    # [0, 2 pi]) after each: every substep conserves photons, the remapped warm start reaches the same
    # fixed point as a cold start in fewer periodic iterations, and the substeps' absorbed rates add up
    n_rot = 4
    p = configs.voronoi_small(6000, periodic_box=True, n_dir=24, seed=113, n_src=10)
    load(ctx, p, scale=1.0 / n_rot)
    it = dict(tol_pbc=1e-8, max_it_pbc=500)
    _, G0, st, _ = ctx.solve(precision=32, **it)
    total = G0.copy()
    rng = np.random.default_rng(7)
    warm, cold = [], []
    for _ in range(n_rot - 1):
        ctx.rotate_directions(oracle.rotation(rng.uniform(0.0, np.pi), rng.uniform(0.0, 2 * np.pi)))
        J, G, st, s = ctx.solve(precision=32, warm_start=1, **it)
        assert s == 0 and abs(st["defect"]) <= 1e-6
        warm.append(st["it_pbc"])
        J2, _, st2, s2 = ctx.solve(precision=32, warm_start=0, **it)
        assert s2 == 0 and fp32_err(J, J2) <= 1e-5
        cold.append(st2["it_pbc"])
        total += G
    assert sum(warm) < sum(cold)
    assert total.sum() == pytest.approx(p.emissivity.sum(), rel=1e-5)  # a closed box absorbs what it emits
