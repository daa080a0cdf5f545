"""Error paths through the C ABI: host-side rejection, cyclic graphs, bounded device waits.
No test here faults or hangs the GPU: the stalled wait gives up after a short poll budget."""
import math

import numpy as np
import pytest

from paper_2207_12848_gb300 import SweepError
from synth import configs
from synth.fields import fibonacci_directions
from synth.mesh import FACE_PERIODIC, Mesh, column_mesh

pytestmark = pytest.mark.gpu


def test_invalid_arguments_rejected(ctx):
    p = configs.voronoi_small(300, n_dir=4, seed=1)
    m = p.mesh
    with pytest.raises(SweepError) as e:
        ctx.set_material(p.kappa_abs, p.emissivity)  # no mesh yet
    assert e.value.status == 1
    bad = m.face_cells.copy()
    bad[3, 1] = m.n_cells + 1
    with pytest.raises(SweepError) as e:
        ctx.set_mesh(Mesh(volume=m.volume, face_cells=bad, area=m.area, normal=m.normal, flags=m.flags))
    assert e.value.status == 1
    nrm = m.normal.copy()
    nrm[0] *= 1.01
    with pytest.raises(SweepError):
        ctx.set_mesh(Mesh(volume=m.volume, face_cells=m.face_cells, area=m.area, normal=nrm, flags=m.flags))
    ctx.set_mesh(m)
    with pytest.raises(SweepError):
        ctx.set_directions(p.omega, p.weight * 1.001)  # weights must sum to 4 pi
    with pytest.raises(SweepError):
        ctx.set_directions(np.zeros((0, 3)), np.zeros(0))
    ctx.set_directions(p.omega, p.weight)
    ka = p.kappa_abs.copy()
    ka[5, 0] = -1.0
    with pytest.raises(SweepError):
        ctx.set_material(ka, p.emissivity)
    ka[5, 0] = np.nan
    with pytest.raises(SweepError):
        ctx.set_material(ka, p.emissivity)
    # the context is still usable after rejected calls
    ctx.set_material(p.kappa_abs, p.emissivity)
    J, G, st, s = ctx.solve(precision=64)
    assert s == 0 and J.max() > 0


def test_cycle_is_reported(ctx):
    m = column_mesh(8, periodic_x=True)
    m.flags = m.flags.copy()
    m.flags[m.flags == FACE_PERIODIC] = 0  # the ring closes through an interior face
    ctx.set_mesh(m)
    ctx.set_directions(np.array([[1.0, 0.0, 0.0]]), np.array([4 * math.pi]))
    ctx.set_material(np.ones((8, 1)), np.ones((8, 1)))
    with pytest.raises(SweepError) as e:
        ctx.solve()
    assert e.value.status == 2


@pytest.mark.parametrize("schedule", ["level", "dataflow"])
def test_stalled_wait_times_out_and_context_recovers(ctx, schedule):
    p = configs.voronoi_small(2000, n_dir=8, seed=3)
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ctx.set_material(p.kappa_abs, p.emissivity)
    with pytest.raises(SweepError) as e:
        ctx.solve(schedule=schedule, debug_stall=1, spin_budget=20000)
    assert e.value.status == 4
    J, G, st, s = ctx.solve(schedule=schedule, precision=64)
    assert s == 0 and abs(st["defect"]) < 1e-12


def test_not_converged_still_writes_outputs(ctx):
    p = configs.voronoi_small(2000, periodic_box=True, n_dir=8, seed=5)
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ctx.set_material(p.kappa_abs, p.emissivity)
    J, G, st, s = ctx.solve(tol_pbc=1e-30, max_it_pbc=2)
    assert s == 3 and st["it_pbc"] == 2 and J.max() > 0
