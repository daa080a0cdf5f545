"""The allocation-free levelisation entry point (sweep_levels_noalloc), for callers that cannot
allocate device memory where they need a sweep order (a fixed memory budget, an arena that hands
out no new blocks, memory nearly exhausted by another component). It must agree exactly with
sweep_levels, call after call, since every call reuses the same static working memory.
This file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from synth import configs
from synth.fields import fibonacci_directions
from synth.mesh import column_mesh, lattice_mesh

pytestmark = pytest.mark.gpu

MAX_CELLS = 65536


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _noalloc_levels(lib, torch, m, om, stream):
    fc = _dev(torch, m.face_cells, np.int32)
    nr = _dev(torch, m.normal, np.float64)
    fl = _dev(torch, m.flags, np.uint8)
    lev = torch.full((m.n_cells,), -7, dtype=torch.int32, device="cuda")
    depth = ctypes.c_int32(0)
    omh = np.ascontiguousarray(om, dtype=np.float64)
    st = lib.sweep_levels_noalloc(0, ctypes.c_void_p(stream), m.n_cells, m.n_faces, fc.data_ptr(), nr.data_ptr(),
                                  fl.data_ptr(), omh.ctypes.data, lev.data_ptr(), ctypes.byref(depth))
    return st, lev.cpu().numpy(), depth.value


@pytest.mark.parametrize("kind", ["voronoi", "periodic", "lattice"])
def test_noalloc_levels_match_sweep_levels(ctx, kind):
    torch = pytest.importorskip("torch")
    if kind == "lattice":
        m = lattice_mesh(20)  # axis-aligned faces: exact ties
        om = np.concatenate([fibonacci_directions(3, seed=4)[0], np.eye(3)[:1]])
    else:
        p = configs.voronoi_small(20000, periodic_box=kind == "periodic", n_dir=4, seed=77)
        m, om = p.mesh, p.omega
    w = np.full(om.shape[0], 4 * math.pi / om.shape[0])
    ctx.set_mesh(m)
    ctx.set_directions(om, w)
    stream = torch.cuda.current_stream().cuda_stream
    for d in range(om.shape[0]):
        ref, ref_depth = ctx.levels(d)
        for _ in range(2):  # two calls in a row share the static working memory
            st, lev, depth = _noalloc_levels(ctx.lib, torch, m, om[d], stream)
            assert st == 0
            assert np.array_equal(lev, ref)
            assert depth == ref_depth


def test_noalloc_rejects_meshes_over_the_limit(gpu_lib):
    depth = ctypes.c_int32(0)
    om = np.array([1.0, 0.0, 0.0])
    # sizes are checked before any GPU work; the pointers are never touched
    st = gpu_lib.sweep_levels_noalloc(0, None, MAX_CELLS + 1, 10, 8, 8, 8, om.ctypes.data, 8, ctypes.byref(depth))
    assert st == 1


def test_noalloc_reports_a_cycle(gpu_lib):
    # a column whose last cell is joined back to its first by an interior face: along +x every cell
    # waits on the one before it, so no cell is ever ready; the count of cells never reached reports it
    torch = pytest.importorskip("torch")
    m = column_mesh(8, periodic_x=True)
    m.flags = m.flags & ~np.uint8(2)  # the wrap-around face becomes an ordinary interior face
    st, lev, depth = _noalloc_levels(gpu_lib, torch, m, np.array([1.0, 0.0, 0.0]), 0)
    assert st == 2


def test_noalloc_rejects_an_out_of_range_cell_index(gpu_lib):
    # an interior face naming cell n_cells + 1: the device-side check refuses it before any counter is
    # touched, and the next call on good input is unaffected
    torch = pytest.importorskip("torch")
    p = configs.voronoi_small(2000, n_dir=1, seed=78)
    m = p.mesh
    bad = m.face_cells.copy()
    inner = np.flatnonzero(m.face_cells[:, 1] >= 0)
    bad[inner[len(inner) // 2], 1] = m.n_cells + 1
    good_fc = m.face_cells
    m.face_cells = bad
    st, _, _ = _noalloc_levels(gpu_lib, torch, m, p.omega[0], 0)
    assert st == 1
    m.face_cells = good_fc
    st, lev, depth = _noalloc_levels(gpu_lib, torch, m, p.omega[0], 0)
    assert st == 0 and depth > 0 and lev.min() == 0
