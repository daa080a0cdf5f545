"""Pins of the synthetic input generators (meshes, directions, fields)."""
import json
import math
import os

import numpy as np
import pytest

from synth import configs
from synth import fields as F
from synth.mesh import FACE_BOUNDARY, FACE_PERIODIC, closure_defect, column_mesh, concat_meshes, lattice_mesh, \
    voronoi_mesh


@pytest.mark.parametrize("periodic", [False, True])
def test_voronoi_closed_cells_fill_the_box(periodic):
    rng = np.random.default_rng(0)
    m = voronoi_mesh(rng.random((3000, 3)), periodic=periodic, threads=2)
    assert m.volume.sum() == pytest.approx(1.0, abs=1e-12)
    scale = m.volume ** (2.0 / 3.0)
    assert np.all(closure_defect(m) <= 1e-10 * scale)
    assert np.all(m.volume > 0) and np.all(m.area >= 0)
    assert np.allclose(np.linalg.norm(m.normal, axis=1), 1.0, atol=1e-14)
    assert m.extra["asymmetric_dropped"] == 0
    if periodic:
        assert not np.any(m.flags & FACE_BOUNDARY) and np.any(m.flags & FACE_PERIODIC)
    else:
        assert not np.any(m.flags & FACE_PERIODIC)
        assert np.all(m.face_cells[m.flags == FACE_BOUNDARY, 1] == -1)


def test_voronoi_normals_follow_generators():
    # Appendix A, Eq. normalDefinition: n = (p' - p) / |p' - p| for interior faces
    rng = np.random.default_rng(1)
    m = voronoi_mesh(rng.random((500, 3)), threads=1)
    inner = m.flags == 0
    d = m.points[m.face_cells[inner, 1]] - m.points[m.face_cells[inner, 0]]
    assert np.allclose(m.normal[inner], d / np.linalg.norm(d, axis=1)[:, None], atol=1e-15)


def test_poisson_voronoi_mean_neighbours_matches_paper():
    # Sec. 2.6 prints the average neighbour count of a 3-D Voronoi grid (tests/golden/paper_values.json);
    # the Poisson-Voronoi expectation is 2 + 48 pi^2 / 35 = 15.535
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        ref = json.load(f)["mean_voronoi_neighbours"]
    rng = np.random.default_rng(2)
    m = voronoi_mesh(rng.random((40000, 3)), periodic=True, threads=4)
    mean = m.neighbour_counts().mean()
    assert mean == pytest.approx(2 + 48 * math.pi ** 2 / 35, abs=0.03)
    assert mean == pytest.approx(ref["value"], abs=ref["abs_tol"])


def test_lattice_and_column_meshes():
    m = lattice_mesh(4)
    assert m.n_cells == 64 and m.volume.sum() == pytest.approx(1.0)
    assert np.all(closure_defect(m) < 1e-15)
    assert np.count_nonzero(m.flags == FACE_BOUNDARY) == 6 * 16
    mp = lattice_mesh(4, periodic=True)
    assert np.count_nonzero(mp.flags == FACE_PERIODIC) == 3 * 16
    assert np.all(closure_defect(mp) < 1e-15)
    c = column_mesh(10)
    assert c.n_cells == 10 and np.all(closure_defect(c) < 1e-15)


def test_concat_meshes_keeps_faces_inside_each_mesh():
    rng = np.random.default_rng(3)
    a = voronoi_mesh(rng.random((100, 3)), threads=1)
    b = voronoi_mesh(rng.random((150, 3)), threads=1)
    m = concat_meshes([a, b])
    assert m.n_cells == 250 and list(m.mesh_cell_offset) == [0, 100, 250]
    inner = m.face_cells[:, 1] >= 0
    side = lambda c: np.searchsorted(m.mesh_cell_offset, c, side="right") - 1
    assert np.all(side(m.face_cells[inner, 0]) == side(m.face_cells[inner, 1]))


def test_fibonacci_directions():
    om, w = F.fibonacci_directions(128, seed=4)
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-15)
    assert w.sum() == pytest.approx(4 * math.pi, rel=1e-14)
    assert np.linalg.norm(om.mean(0)) < 1e-2  # nearly isotropic
    om2, _ = F.fibonacci_directions(128, seed=4)
    assert np.array_equal(om, om2)


def test_lognormal_field_statistics():
    f = F.lognormal_field(64, -3.0, 1.0, seed=5)
    assert np.log(f).std() == pytest.approx(1.0, rel=1e-12)
    assert f.mean() == pytest.approx(1.0, rel=0.2)


def test_hilbert_order_is_a_local_permutation():
    rng = np.random.default_rng(6)
    p = rng.random((4096, 3))
    o = F.hilbert_order(p)
    assert np.array_equal(np.sort(o), np.arange(4096))
    step = np.linalg.norm(np.diff(p[o], axis=0), axis=1).mean()
    assert step < 0.5 * np.linalg.norm(np.diff(p, axis=0), axis=1).mean()


def test_batched_sizes_sum():
    s = configs._sizes_loguniform(64, 1 << 22, 1 << 12, 1 << 17, seed=1)
    assert s.sum() == 1 << 22 and s.min() >= 1 << 12 and s.max() <= 1 << 17


def test_small_problem_recipe():
    p = configs.voronoi_small(200, n_dir=8, n_groups=2, seed=1, bc_inflow=True)
    tau = p.kappa_abs * np.cbrt(p.mesh.volume)[:, None]
    assert tau.min() >= 0.01 * (1 - 1e-12) and tau.max() <= 10.0 * (1 + 1e-12)
    assert p.boundary_inflow.shape == (int(np.count_nonzero(p.mesh.flags & 1)), 2)
