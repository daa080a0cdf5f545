"""Synthetic Voronoi meshes: the seeded input generator shared by the oracle
tests, the GPU tests and the benchmark.

A mesh is given the way the transport method receives it (paper Sec. 2.5 and
Appendix A): cell volumes, faces stored once as a neighbour pair (c0, c1) with
an area and a unit normal pointing from c0 towards c1, and per-face flags for
box-boundary faces (c1 = -1) and periodic faces (c1 is the partner cell across
the box). Nothing here evaluates the transport method itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

FACE_BOUNDARY = 1
FACE_PERIODIC = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LIB_LOCK = threading.Lock()


def build_lib(force: bool = False) -> str:
    """Compile the Voronoi clipper (plain C, host only)."""
    src = os.path.join(_HERE, "voronoi.c")
    out = os.path.join(_HERE, "_voronoi.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_lib())
            P = ctypes.c_void_p
            lib.vor_build.restype = ctypes.c_int
            lib.vor_build.argtypes = [P, ctypes.c_int64, ctypes.c_int, P, P, P, ctypes.c_double, P, ctypes.c_int32,
                                      ctypes.c_int64, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P, P, P, P]
            _LIB = lib
    return _LIB


@dataclass
class Mesh:
    """Cells, faces and (optionally) the generating points of one or more meshes."""

    volume: np.ndarray            # [N] float64
    face_cells: np.ndarray        # [F,2] int32; [:,1] = -1 on boundary faces
    area: np.ndarray              # [F] float64
    normal: np.ndarray            # [F,3] float64, unit, c0 -> c1 (outward for boundary faces)
    flags: np.ndarray             # [F] uint8 (FACE_BOUNDARY | FACE_PERIODIC)
    points: np.ndarray | None = None   # [N,3] generators, when known
    mesh_cell_offset: np.ndarray = field(default=None)  # [M+1] int64
    box: float = 1.0
    periodic: bool = False
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        if self.mesh_cell_offset is None:
            self.mesh_cell_offset = np.array([0, self.n_cells], dtype=np.int64)

    @property
    def n_cells(self) -> int:
        return int(self.volume.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.area.shape[0])

    @property
    def n_meshes(self) -> int:
        return int(self.mesh_cell_offset.shape[0] - 1)

    def boundary_face_ids(self) -> np.ndarray:
        return np.nonzero(self.flags & FACE_BOUNDARY)[0]

    def neighbour_counts(self) -> np.ndarray:
        """Faces per cell (a periodic self-face counts twice, once per side)."""
        cnt = np.bincount(self.face_cells[:, 0], minlength=self.n_cells)
        inner = self.face_cells[:, 1] >= 0
        cnt = cnt + np.bincount(self.face_cells[inner, 1], minlength=self.n_cells)
        return cnt


# ----------------------------------------------------------------------------------------------
# Analytic meshes
# ----------------------------------------------------------------------------------------------
def lattice_mesh(n: int, periodic: bool = False, box: float = 1.0) -> Mesh:
    """Voronoi mesh of an n^3 cubic lattice of generators: cube cells of side h = box/n.

    Cell (i, j, k) has index i + n*(j + n*k) and its generator at the cell centre.
    Only the six cube faces are kept (diagonal contacts have zero area).
    """
    h = box / n
    idx = np.arange(n ** 3, dtype=np.int64).reshape(n, n, n)  # [k, j, i]
    faces, normals, flags = [], [], []
    for ax in range(3):  # ax 0 = x (i), 1 = y (j), 2 = z (k)
        npax = 2 - ax  # numpy axis for this coordinate
        lo = np.take(idx, np.arange(n - 1), axis=npax).ravel()
        hi = np.take(idx, np.arange(1, n), axis=npax).ravel()
        e = np.zeros(3)
        e[ax] = 1.0
        faces.append(np.stack([lo, hi], 1))
        normals.append(np.tile(e, (lo.size, 1)))
        flags.append(np.zeros(lo.size, np.uint8))
        first = np.take(idx, [0], axis=npax).ravel()
        last = np.take(idx, [n - 1], axis=npax).ravel()
        if periodic:
            faces.append(np.stack([last, first], 1))
            normals.append(np.tile(e, (last.size, 1)))
            flags.append(np.full(last.size, FACE_PERIODIC, np.uint8))
        else:
            faces.append(np.stack([first, np.full_like(first, -1)], 1))
            normals.append(np.tile(-e, (first.size, 1)))
            flags.append(np.full(first.size, FACE_BOUNDARY, np.uint8))
            faces.append(np.stack([last, np.full_like(last, -1)], 1))
            normals.append(np.tile(e, (last.size, 1)))
            flags.append(np.full(last.size, FACE_BOUNDARY, np.uint8))
    fc = np.concatenate(faces).astype(np.int32)
    nr = np.concatenate(normals)
    fl = np.concatenate(flags)
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pts = (np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1) + 0.5) * h
    return Mesh(volume=np.full(n ** 3, h ** 3), face_cells=fc, area=np.full(fc.shape[0], h * h), normal=nr,
                flags=fl, points=pts, box=box, periodic=periodic, extra={"kind": "lattice", "n": n, "h": h})


def column_mesh(n: int, h: float = 1.0 / 256, periodic_x: bool = False) -> Mesh:
    """n cube cells of side h in a row along +x; every other face is a box-boundary face.

    Boundary faces are ordered: the -x end face first (index 0 among boundary faces),
    then the +x end face (absent with periodic_x), then the four side faces of each cell.
    """
    faces, normals, flags = [], [], []
    ex = np.array([1.0, 0, 0])
    if periodic_x:
        faces.append([n - 1, 0]); normals.append(ex); flags.append(FACE_PERIODIC)
    else:
        faces.append([0, -1]); normals.append(-ex); flags.append(FACE_BOUNDARY)
        faces.append([n - 1, -1]); normals.append(ex); flags.append(FACE_BOUNDARY)
    for c in range(n):
        for nv in ([0, 1.0, 0], [0, -1.0, 0], [0, 0, 1.0], [0, 0, -1.0]):
            faces.append([c, -1]); normals.append(np.array(nv)); flags.append(FACE_BOUNDARY)
    for c in range(n - 1):
        faces.append([c, c + 1]); normals.append(ex); flags.append(0)
    fc = np.array(faces, np.int32)
    pts = np.stack([(np.arange(n) + 0.5) * h, np.full(n, 0.5 * h), np.full(n, 0.5 * h)], 1)
    return Mesh(volume=np.full(n, h ** 3), face_cells=fc, area=np.full(len(faces), h * h),
                normal=np.array(normals, float), flags=np.array(flags, np.uint8), points=pts, box=n * h,
                periodic=periodic_x, extra={"kind": "column", "n": n, "h": h})


def star_mesh(n_arms: int, seed: int) -> Mesh:
    """One hub cell joined to n_arms cells by faces whose normals cover the sphere; every arm cell has a
    box-boundary face on its far side. Not a tessellation (the cells are not closed), but every step of
    the sweep is defined on it, and the oracle runs the same algorithm."""
    from synth.fields import fibonacci_directions
    nrm, _ = fibonacci_directions(n_arms, seed=seed)
    rng = np.random.default_rng(seed)
    fc = np.zeros((2 * n_arms, 2), np.int32)
    fc[:n_arms, 0] = 0
    fc[:n_arms, 1] = np.arange(1, n_arms + 1)
    fc[n_arms:, 0] = np.arange(1, n_arms + 1)
    fc[n_arms:, 1] = -1
    normal = np.concatenate([nrm, nrm])
    area = rng.uniform(0.5, 1.5, 2 * n_arms) * 0.01
    flags = np.zeros(2 * n_arms, np.uint8)
    flags[n_arms:] = FACE_BOUNDARY
    vol = np.full(n_arms + 1, 1e-3)
    vol[0] = 1e-2
    return Mesh(volume=vol, face_cells=fc, area=area, normal=normal, flags=flags)


# ----------------------------------------------------------------------------------------------
# Voronoi meshes from generator points
# ----------------------------------------------------------------------------------------------
def _ghosts(points: np.ndarray, margin: float):
    """Generators plus their periodic images within `margin` of the unit box."""
    n = points.shape[0]
    ext = [points]
    orig = [np.arange(n, dtype=np.int32)]
    code = [np.full(n, 13, np.int8)]
    for sz in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sx in (-1, 0, 1):
                if sx == sy == sz == 0:
                    continue
                s = np.array([sx, sy, sz], float)
                m = np.ones(n, bool)
                for a in range(3):
                    if s[a] > 0:
                        m &= points[:, a] < margin
                    elif s[a] < 0:
                        m &= points[:, a] >= 1.0 - margin
                ids = np.nonzero(m)[0]
                ext.append(points[ids] + s)
                orig.append(ids.astype(np.int32))
                code.append(np.full(ids.size, (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1), np.int8))
    return np.ascontiguousarray(np.concatenate(ext)), np.concatenate(orig), np.concatenate(code)


def _shift_of_code(code: np.ndarray) -> np.ndarray:
    c = code.astype(np.int64)
    return np.stack([c % 3 - 1, (c // 3) % 3 - 1, c // 9 - 1], 1).astype(float)


def voronoi_mesh(points: np.ndarray, periodic: bool = False, threads: int | None = None, k0: int = 48) -> Mesh:
    """Voronoi tessellation of generators in the unit box (vacuum walls or periodic)."""
    from scipy.spatial import cKDTree

    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    threads = threads or max(1, os.cpu_count() or 1)
    lib = _lib()
    if periodic:
        margin = min(0.5, max(0.05, 8.0 * n ** (-1.0 / 3.0)))
    else:
        margin = 0.0
    volume = np.zeros(n)
    nfaces = np.zeros(n, np.int32)
    status = np.full(n, -1, np.int32)
    todo = np.arange(n, dtype=np.int64)
    k = k0
    records = []
    for _attempt in range(8):
        if todo.size == 0:
            break
        if periodic:
            ext, orig, code = _ghosts(pts, margin)
        else:
            ext, orig, code = pts, np.arange(n, dtype=np.int32), np.full(n, 13, np.int8)
        tree = cKDTree(ext)
        kk = min(k, ext.shape[0])
        _, cand = tree.query(pts[todo], k=kk, workers=threads)
        cand = np.ascontiguousarray(np.asarray(cand).reshape(todo.size, kk).astype(np.int32))
        # cells are processed in chunks; each chunk writes into its own record buffers
        chunk = max(256, (todo.size + 4 * threads - 1) // (4 * threads))
        sub_pts = np.ascontiguousarray(pts[todo])
        sub_vol = np.zeros(todo.size)
        sub_nf = np.zeros(todo.size, np.int32)
        sub_st = np.zeros(todo.size, np.int32)

        def run(b):
            e = min(todo.size, b + chunk)
            cap = (e - b) * 64
            while True:
                oc = np.empty(cap, np.int32); on = np.empty(cap, np.int32)
                ocode = np.empty(cap, np.int8); oa = np.empty(cap)
                nw = ctypes.c_int64(0)
                rc = lib.vor_build(sub_pts.ctypes.data, todo.size, int(periodic), ext.ctypes.data,
                                   orig.ctypes.data, code.ctypes.data, margin, cand.ctypes.data, kk, b, e,
                                   sub_vol.ctypes.data, sub_nf.ctypes.data, sub_st.ctypes.data, cap,
                                   oc.ctypes.data, on.ctypes.data, ocode.ctypes.data, oa.ctypes.data,
                                   ctypes.byref(nw))
                if rc == 0:
                    w = nw.value
                    return oc[:w], on[:w], ocode[:w], oa[:w]
                if rc != 1:
                    raise MemoryError("voronoi clipper failed")
                cap *= 2

        # vor_build indexes generators by position in sub_pts; the candidate rows follow todo order
        with ThreadPoolExecutor(threads) as ex:
            outs = list(ex.map(run, range(0, todo.size, chunk)))
        oc = np.concatenate([o[0] for o in outs]).astype(np.int64)
        on = np.concatenate([o[1] for o in outs])
        ocode = np.concatenate([o[2] for o in outs])
        oa = np.concatenate([o[3] for o in outs])
        cell_global = todo[oc]
        # faces towards the generator's own periodic images come back with nbr = -2
        on = np.where(on == -2, cell_global.astype(np.int32), on)
        ok = sub_st == 0
        if np.any(sub_st == 4):
            raise RuntimeError("voronoi clipper: cell too complex")
        keep = ok[oc]
        records.append((cell_global[keep], on[keep], ocode[keep], oa[keep]))
        volume[todo[ok]] = sub_vol[ok]
        nfaces[todo[ok]] = sub_nf[ok]
        status[todo] = sub_st
        if np.any(sub_st == 3):
            margin = min(1.0, 2.0 * margin)  # up to a full periodic image of the box in every shell
        todo = todo[~ok]
        k *= 3
    if todo.size:
        raise RuntimeError("voronoi: %d cells did not close" % todo.size)
    cell = np.concatenate([r[0] for r in records])
    nbr = np.concatenate([r[1] for r in records]).astype(np.int64)
    code = np.concatenate([r[2] for r in records]).astype(np.int64)
    area = np.concatenate([r[3] for r in records])
    return _assemble(pts, volume, cell, nbr, code, area, periodic)


def _assemble(pts, volume, cell, nbr, code, area, periodic) -> Mesh:
    n = pts.shape[0]
    wall = nbr < 0
    # interior/periodic records: keep the canonical side, require its mirror record to exist
    inner = ~wall
    ci, nj, cd, ar = cell[inner], nbr[inner], code[inner], area[inner]
    key = (ci * n + nj) * 27 + cd
    rkey = (nj * n + ci) * 27 + (26 - cd)
    canon = (ci < nj) | ((ci == nj) & (cd < 13))
    skey = np.sort(key)
    pos = np.searchsorted(skey, rkey)
    pos = np.minimum(pos, skey.size - 1)
    has_mirror = skey[pos] == rkey
    sel = canon & has_mirror
    dropped = int(np.count_nonzero(~has_mirror))
    c0, c1, cc, aa = ci[sel], nj[sel], cd[sel], ar[sel]
    d = pts[c1] + _shift_of_code(cc) - pts[c0]
    nrm = d / np.linalg.norm(d, axis=1)[:, None]
    fl = np.where(cc != 13, FACE_PERIODIC, 0).astype(np.uint8)
    # box walls (vacuum): wall id 2*axis + side
    wc, wcode, wa = cell[wall], code[wall], area[wall]
    wn = np.zeros((wc.size, 3))
    wn[np.arange(wc.size), wcode // 2] = np.where(wcode % 2 == 1, 1.0, -1.0)
    face_cells = np.concatenate([np.stack([c0, c1], 1), np.stack([wc, np.full_like(wc, -1)], 1)]).astype(np.int32)
    normal = np.concatenate([nrm, wn])
    areas = np.concatenate([aa, wa])
    flags = np.concatenate([fl, np.full(wc.size, FACE_BOUNDARY, np.uint8)])
    order = np.lexsort((face_cells[:, 1], face_cells[:, 0]))
    return Mesh(volume=volume, face_cells=face_cells[order], area=areas[order], normal=normal[order],
                flags=flags[order], points=pts, periodic=periodic,
                extra={"kind": "voronoi", "asymmetric_dropped": dropped})


def concat_meshes(meshes: list[Mesh]) -> Mesh:
    """Join independent meshes into one cell index space (faces never cross meshes)."""
    off = np.zeros(len(meshes) + 1, np.int64)
    for i, m in enumerate(meshes):
        off[i + 1] = off[i] + m.n_cells
    fcs = []
    for i, m in enumerate(meshes):
        fc = m.face_cells.astype(np.int64).copy()
        fc[:, 0] += off[i]
        inner = fc[:, 1] >= 0
        fc[inner, 1] += off[i]
        fcs.append(fc)
    pts = None
    if all(m.points is not None for m in meshes):
        pts = np.concatenate([m.points for m in meshes])
    return Mesh(volume=np.concatenate([m.volume for m in meshes]),
                face_cells=np.concatenate(fcs).astype(np.int32),
                area=np.concatenate([m.area for m in meshes]),
                normal=np.concatenate([m.normal for m in meshes]),
                flags=np.concatenate([m.flags for m in meshes]), points=pts, mesh_cell_offset=off,
                periodic=any(m.periodic for m in meshes), extra={"kind": "batch"})


def closure_defect(mesh: Mesh) -> np.ndarray:
    """|sum_f A_f n_f| per cell (outward orientation), zero for closed cells."""
    s = np.zeros((mesh.n_cells, 3))
    an = mesh.area[:, None] * mesh.normal
    np.add.at(s, mesh.face_cells[:, 0], an)
    inner = mesh.face_cells[:, 1] >= 0
    np.add.at(s, mesh.face_cells[inner, 1], -an[inner])
    return np.linalg.norm(s, axis=1)
