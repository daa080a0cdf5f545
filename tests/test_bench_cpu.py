"""Host logic of bench.py that needs no GPU: the algorithmic bytes per update of the roofline, and the
rule that a recorded DRAM-traffic figure is only used while the kernel sources it was measured on are
unchanged."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth import configs  # noqa: E402
from synth.mesh import lattice_mesh  # noqa: E402


@pytest.mark.parametrize("periodic,G", [(True, 1), (True, 4), (False, 2)])
def test_bytes_per_update_on_a_lattice(periodic, G):
    # an n^3 lattice has 6 face sides per cell either way: periodic faces have two sides, and with
    # vacuum walls each of the 6n^2 boundary faces has one side and the interior faces two
    n = 6
    m = lattice_mesh(n, periodic=periodic)
    p = configs.Problem("lattice", m, np.zeros((1, 3)), np.ones(1), np.ones((m.n_cells, G)),
                        np.zeros((m.n_cells, G)))
    bpu, fbar = bench.bytes_per_update(p)
    sides = 6 * n ** 3
    assert fbar == pytest.approx(sides / n ** 3)
    assert bpu == pytest.approx((8.0 + 16.0 * fbar) / G + 12.0)
    assert bench.bytes_per_update(p, "exp")[0] == pytest.approx(bpu + 4.0)  # the cell-mean write


def test_traffic_figure_follows_the_kernel_sources(tmp_path, monkeypatch):
    summary = tmp_path / "traffic.txt"
    summary.write_text("kernel_sha: %s\ntraffic_bytes_per_launch: 12345\n" % bench.kernel_sha())
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench.profiled_traffic("periodic") == 12345.0
    assert bench.profiled_traffic("batched") is None  # measured on the periodic box only
    summary.write_text("kernel_sha: 0000000000000000\ntraffic_bytes_per_launch: 12345\n")
    assert bench.profiled_traffic("periodic") is None  # sources changed since the capture


def test_single_rank_aggregate():
    d = bench.Dist()
    assert d.world == 1
    v, t = bench.aggregate(d, 2.0, 10.0)
    assert (v, t) == (5.0, 2.0)


def test_step_text_names_the_loops():
    m = lattice_mesh(4, periodic=True)
    one = np.ones((m.n_cells, 1))
    p = configs.Problem("box", m, np.zeros((1, 3)), np.ones(1), one, 0 * one, kappa_scat=one)
    assert "inside periodic iteration" in bench.step_text(p, 0)
    assert "fused" in bench.step_text(p, 1)
    q = configs.Problem("box", lattice_mesh(4), np.zeros((1, 3)), np.ones(1), one, 0 * one)
    assert bench.step_text(q, 1).endswith("one sweep")


def test_roofline_over_sweeps_of_different_widths():
    # the adjoint's roofline: per sweep every task reads its row once, per update 12 bytes; with sweeps
    # of one width it is the per-launch roofline, and a transposed sweep over 2G groups adds only the
    # per-update bytes of its extra groups
    n = 6
    m = lattice_mesh(n, periodic=True)
    G, D = 2, 3
    p = configs.Problem("lattice", m, np.zeros((D, 3)), np.ones(D), np.ones((m.n_cells, G)),
                        np.zeros((m.n_cells, G)))
    peaks = {"hbm_gbs": 1000.0, "source": "test"}
    one = bench._roof(p, 2.0, peaks, "k")
    upd = m.n_cells * D * G
    same = bench._roof_sweeps(p, 6.0, 3, 3.0 * upd, peaks, "k")
    assert same["achieved"] == pytest.approx(one["achieved"])
    assert same["bytes_per_update"] == pytest.approx(one["bytes_per_update"])
    assert same["avg_launch_ms"] == pytest.approx(2.0)
    mixed = bench._roof_sweeps(p, 4.0, 2, 3.0 * upd, peaks, "k")  # one sweep over G, one over 2G
    row = m.n_cells * D * (8.0 + 16.0 * 6.0)
    assert mixed["achieved"] * 1e9 * 4.0e-3 == pytest.approx(2 * row + 12.0 * 3.0 * upd)
    assert mixed["frac"] == pytest.approx(mixed["achieved"] / 1000.0)
