"""ctypes binding of libsweep.so (include/sweep.h). Argument marshalling only: every step of
the transport sweep runs in the CUDA library; there is no Python or CPU fallback."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsweep.so")

SWEEP_OK = 0
SWEEP_ERR_INVALID_ARG = 1
SWEEP_ERR_CYCLE = 2
SWEEP_NOT_CONVERGED = 3
SWEEP_ERR_TIMEOUT = 4
SWEEP_ERR_OOM = 5
SWEEP_ERR_CUDA = 6
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CYCLE", 3: "NOT_CONVERGED", 4: "TIMEOUT", 5: "OOM", 6: "CUDA"}

SWEEP_FACE_BOUNDARY = 1
SWEEP_FACE_PERIODIC = 2
SWEEP_SCHED_AUTO, SWEEP_SCHED_LEVEL, SWEEP_SCHED_DATAFLOW, SWEEP_SCHED_PLAIN = 0, 1, 2, 3
SCHEDULES = {"auto": 0, "level": 1, "dataflow": 2, "plain": 3}
LAWS = {"balance": 0, "exp": 1}
# forms of the batched sweep kernel (sweep_stats.kernel_used)
KERNELS = {0: "none", 1: "k_plain", 2: "k_sweep", 3: "k_sweep_rec", 4: "k_sweep_op", 5: "k_sweep_op1", 6: "k_sweep_op2",
           7: "k_sweep_pk"}
OP_FORMATS = {"auto": 0, "lines": 1, "packets": 2}

# every entry point include/sweep.h declares
EXPORTS = ("sweep_default_opts", "sweep_create", "sweep_destroy", "sweep_set_mesh", "sweep_set_directions",
           "sweep_set_material", "sweep_set_material_dev", "sweep_solve", "sweep_solve_dev", "sweep_levels",
           "sweep_intensity", "sweep_adjoint", "sweep_adjoint_dev", "sweep_status_string", "sweep_last_error",
           "sweep_levels_noalloc", "sweep_rotate_directions")


class sweep_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("law", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("max_it_scat", ctypes.c_int32), ("tol_scat", ctypes.c_double), ("max_it_pbc", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("tol_pbc", ctypes.c_double), ("dir_batch", ctypes.c_int32),
                ("relevel", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("spin_budget", ctypes.c_int64), ("debug_stall", ctypes.c_int32),
                ("lanes_per_task", ctypes.c_int32), ("geometry_only", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("fused_loops", ctypes.c_int32),
                ("op_format", ctypes.c_int32), ("packets_per_step", ctypes.c_int32), ("transport", ctypes.c_int32)]


class sweep_stats(ctypes.Structure):
    _fields_ = [("it_scat", ctypes.c_int32), ("it_pbc", ctypes.c_int32), ("n_sweeps", ctypes.c_int32),
                ("depth_max", ctypes.c_int32), ("depth_mean", ctypes.c_double), ("res_scat", ctypes.c_double),
                ("res_pbc", ctypes.c_double), ("res_pbc_mean", ctypes.c_double), ("emitted", ctypes.c_double),
                ("injected", ctypes.c_double), ("absorbed", ctypes.c_double), ("escaped", ctypes.c_double),
                ("defect", ctypes.c_double), ("t_ms", ctypes.c_double * 8), ("updates", ctypes.c_double),
                ("updates_per_s", ctypes.c_double), ("sweep_launches", ctypes.c_int32),
                ("schedule_used", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("lanes_used", ctypes.c_int32), ("threads_used", ctypes.c_int32),
                ("blocks_per_sm_used", ctypes.c_int32), ("kernel_used", ctypes.c_int32),
                ("graph_used", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "t_ms"}
        t = list(self.t_ms)
        d.update(t_classify_ms=t[0], t_levelise_ms=t[1], t_sweep_ms=t[2], t_update_ms=t[3], t_total_ms=t[4],
                 t_assemble_ms=t[5], t_transposed_ms=t[6])
        return d


_LIB = None


def load(path: str | None = None):
    """Load libsweep.so; raises if it has not been built (no fallback exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libsweep.so is missing (%s): build it with paper_2207_12848_gb300.build.build()" % p)
    lib = ctypes.CDLL(p)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    S = ctypes.c_int
    OP, SP = ctypes.POINTER(sweep_opts), ctypes.POINTER(sweep_stats)
    sig = {
        "sweep_default_opts": (None, [OP]),
        "sweep_create": (S, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, P]),
        "sweep_destroy": (S, [P]),
        "sweep_set_mesh": (S, [P, I64, P, I64, P, P, P, P, I32, P]),
        "sweep_set_directions": (S, [P, I32, P, P]),
        "sweep_set_material": (S, [P, I32, P, P, P, P]),
        "sweep_set_material_dev": (S, [P, I32, P, P, P, P]),
        "sweep_solve": (S, [P, OP, P, P, SP]),
        "sweep_solve_dev": (S, [P, OP, P, P, SP]),
        "sweep_levels": (S, [P, I32, P, ctypes.POINTER(I32)]),
        "sweep_intensity": (S, [P, I32, P]),
        "sweep_adjoint": (S, [P, OP, P, P, P, P, P, SP]),
        "sweep_adjoint_dev": (S, [P, OP, P, P, P, P, P, SP]),
        "sweep_status_string": (ctypes.c_char_p, [S]),
        "sweep_last_error": (ctypes.c_char_p, [P]),
        "sweep_levels_noalloc": (S, [ctypes.c_int, P, I64, I64, P, P, P, P, P, ctypes.POINTER(I32)]),
        "sweep_rotate_directions": (S, [P, P, I64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class SweepError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def default_opts(**kw) -> sweep_opts:
    o = sweep_opts()
    load().sweep_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "schedule" and isinstance(v, str):
            v = SCHEDULES[v]
        if k == "law" and isinstance(v, str):
            v = LAWS[v]
        if k == "op_format" and isinstance(v, str):
            v = OP_FORMATS[v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _host(a, dtype):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return None if a is None else a.ctypes.data


def _dp(t):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


class Context:
    """One sweep_ctx: a GPU, a CUDA stream and the device copies of mesh, directions and material."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.sweep_create(ctypes.byref(h), device, ctypes.c_void_p(stream or 0))
        if st != SWEEP_OK:
            raise SweepError(st, "sweep_create failed")
        self.h = h
        self.device = device
        self.stream = stream or 0
        self.n_cells = 0
        self.n_dir = 0
        self.n_groups = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.sweep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st: int, ok=(SWEEP_OK,)):
        if st not in ok:
            raise SweepError(st, self.lib.sweep_last_error(self.h).decode())
        return st

    # ---- inputs ---------------------------------------------------------------------------
    def set_mesh(self, mesh=None, *, volume=None, face_cells=None, area=None, normal=None, flags=None,
                 mesh_cell_offset=None):
        if mesh is not None:
            volume, face_cells, area, normal, flags = mesh.volume, mesh.face_cells, mesh.area, mesh.normal, mesh.flags
            mesh_cell_offset = mesh.mesh_cell_offset
        vol = _host(volume, np.float64)
        fc = _host(face_cells, np.int32).reshape(-1, 2)
        ar = _host(area, np.float64)
        nr = _host(normal, np.float64).reshape(-1, 3)
        fl = _host(flags, np.uint8)
        off = _host(mesh_cell_offset, np.int64)
        nm = 0 if off is None else off.size - 1
        self._check(self.lib.sweep_set_mesh(self.h, vol.size, _hp(vol), fc.shape[0], _hp(fc), _hp(ar), _hp(nr),
                                            _hp(fl), nm, _hp(off)))
        self.n_cells = vol.size
        self.n_boundary = int(np.count_nonzero(fl & SWEEP_FACE_BOUNDARY))

    def set_directions(self, omega, weight):
        om = _host(omega, np.float64).reshape(-1, 3)
        w = _host(weight, np.float64)
        self._check(self.lib.sweep_set_directions(self.h, om.shape[0], _hp(om), _hp(w)))
        self.n_dir = om.shape[0]

    def set_material(self, kappa_abs, emissivity, kappa_scat=None, boundary_inflow=None):
        """Host arrays (numpy) or CUDA tensors (float64) of shape [n_cells, G]."""
        if hasattr(kappa_abs, "is_cuda") and kappa_abs.is_cuda:
            G = kappa_abs.reshape(self.n_cells, -1).shape[1]
            self._check(self.lib.sweep_set_material_dev(self.h, G, _dp(kappa_abs), _dp(kappa_scat), _dp(emissivity),
                                                        _dp(boundary_inflow)))
        else:
            ka = _host(kappa_abs, np.float64)
            ka = ka.reshape(ka.shape[0], -1) if ka.ndim > 1 else ka.reshape(-1, 1)
            G = ka.shape[1]
            em = _host(emissivity, np.float64).reshape(-1, G)
            ks = None if kappa_scat is None else _host(kappa_scat, np.float64).reshape(-1, G)
            bc = None if boundary_inflow is None else _host(boundary_inflow, np.float64)
            self._check(self.lib.sweep_set_material(self.h, G, _hp(ka), _hp(ks), _hp(em), _hp(bc)))
        self.n_groups = G

    # ---- solves ---------------------------------------------------------------------------
    def solve(self, opts: sweep_opts | None = None, allow_not_converged: bool = True, **kw):
        """Host outputs: (J[N,G], Gamma[N,G], stats dict, status)."""
        o = opts or default_opts(**kw)
        J = np.zeros((self.n_cells, self.n_groups))
        Gm = np.zeros((self.n_cells, self.n_groups))
        st = sweep_stats()
        ok = (SWEEP_OK, SWEEP_NOT_CONVERGED) if allow_not_converged else (SWEEP_OK,)
        s = self._check(self.lib.sweep_solve(self.h, ctypes.byref(o), _hp(J), _hp(Gm), ctypes.byref(st)), ok)
        return J, Gm, st.as_dict(), s

    def solve_dev(self, J_out, Gamma_out, opts: sweep_opts | None = None, **kw):
        """Device outputs into CUDA float64 tensors [N,G]; returns (stats dict, status)."""
        o = opts or default_opts(**kw)
        st = sweep_stats()
        s = self._check(self.lib.sweep_solve_dev(self.h, ctypes.byref(o), _dp(J_out), _dp(Gamma_out),
                                                 ctypes.byref(st)), (SWEEP_OK, SWEEP_NOT_CONVERGED))
        return st.as_dict(), s

    def rotate_directions(self, rotation, n_quad: int = 0):
        """Rotate the direction set by a 3x3 rotation and remap the last solve's intensities onto it."""
        R = _host(rotation, np.float64).reshape(3, 3)
        self._check(self.lib.sweep_rotate_directions(self.h, _hp(R), n_quad))

    def levels(self, direction: int):
        lev = np.zeros(self.n_cells, np.int32)
        depth = ctypes.c_int32(0)
        self._check(self.lib.sweep_levels(self.h, direction, _hp(lev), ctypes.byref(depth)))
        return lev, depth.value

    def intensity(self, direction: int):
        out = np.zeros((self.n_cells, self.n_groups))
        self._check(self.lib.sweep_intensity(self.h, direction, _hp(out)))
        return out

    def adjoint(self, dl_dJ=None, dl_dGamma=None, opts: sweep_opts | None = None, with_kappa_scat: bool = False,
                allow_not_converged: bool = False, **kw):
        """Host gradients (dL/dkappa_abs, dL/demissivity[, dL/dkappa_scat], stats dict) [N,G]."""
        o = opts or default_opts(**kw)
        N, G = self.n_cells, self.n_groups
        dj = None if dl_dJ is None else _host(dl_dJ, np.float64).reshape(N, G)
        dg = None if dl_dGamma is None else _host(dl_dGamma, np.float64).reshape(N, G)
        gk = np.zeros((N, G))
        ge = np.zeros((N, G))
        gs = np.zeros((N, G)) if with_kappa_scat else None
        st = sweep_stats()
        ok = (SWEEP_OK, SWEEP_NOT_CONVERGED) if allow_not_converged else (SWEEP_OK,)
        self._check(self.lib.sweep_adjoint(self.h, ctypes.byref(o), _hp(dj), _hp(dg), _hp(gk), _hp(ge), _hp(gs),
                                           ctypes.byref(st)), ok)
        return (gk, ge, gs, st.as_dict()) if with_kappa_scat else (gk, ge, st.as_dict())

    def adjoint_dev(self, grad_kappa_out, grad_emissivity_out, dl_dJ=None, dl_dGamma=None,
                    opts: sweep_opts | None = None, grad_kappa_scat_out=None, **kw):
        o = opts or default_opts(**kw)
        st = sweep_stats()
        self._check(self.lib.sweep_adjoint_dev(self.h, ctypes.byref(o), _dp(dl_dJ), _dp(dl_dGamma),
                                               _dp(grad_kappa_out), _dp(grad_emissivity_out),
                                               _dp(grad_kappa_scat_out), ctypes.byref(st)))
        return st.as_dict()
