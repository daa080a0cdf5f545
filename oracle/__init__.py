"""FP64 CPU oracle of the transport sweep -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

``sweep_oracle.c`` follows the paper's Algorithm 2 (Kahn task queue) with the
Sec. 2.6 transport scheme (a), Algorithm 1 (source iteration) and the Sec. 2.7
periodic iteration; ``dense.py`` is an independent second oracle that assembles
and solves the same linear systems directly on small meshes.

Parity status per function (what pins it; see tests/test_oracle_pins.py):
  oracle_levels  -- pinned: brute-force longest paths, the Voronoi ordering invariant (Appendix A);
                    with dc_n > 0 brute-force longest paths of the thinner scheme (b) graph and the
                    paper's dependency counts
  oracle_solve   -- pinned: 1-D column closed form, photon conservation, dense LU solves
                    (plain, scattering, periodic, both at once for the nested and the fused
                    loops), uniform periodic fixed point, linearity, pure streaming; law="exp":
                    the exact transport solution along a column and dense solves of the EXP
                    system; dc_n > 0: scheme (a) where the faces tie and dense solves of the
                    scheme (b) system
  oracle_adjoint -- pinned: central finite differences of oracle_solve (also in kappa_scat, through
                    the source iteration, and through the periodic iteration), dense transposed
                    solve (also of the coupled system, with scattering and periodic faces),
                    reciprocity of the transport operator
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

OK, ERR_ARG, ERR_CYCLE, NOT_CONVERGED, ERR_MEM = 0, 1, 2, 3, 5
LAWS = {"balance": 0, "exp": 1}


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "sweep_oracle.c")
    out = os.path.join(_HERE, "_sweep_oracle.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-o", tmp,
                               src, "-lm", "-lpthread"])
        os.replace(tmp, out)
    return out


class Stats(ctypes.Structure):
    _fields_ = [("it_scat", ctypes.c_int32), ("it_pbc", ctypes.c_int32), ("res_scat", ctypes.c_double),
                ("res_pbc", ctypes.c_double), ("res_pbc_mean", ctypes.c_double), ("emitted", ctypes.c_double),
                ("injected", ctypes.c_double), ("absorbed", ctypes.c_double), ("escaped", ctypes.c_double),
                ("defect", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.oracle_levels.restype = ctypes.c_int
            lib.oracle_levels.argtypes = [I64, I64, P, P, P, P, P, I32, P, ctypes.c_int, P, P, ctypes.c_int]
            lib.oracle_solve.restype = ctypes.c_int
            lib.oracle_solve.argtypes = [I64, I64, P, P, P, P, P, I32, P, P, I32, P, P, P, P, D, I32, D, I32, P,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P,
                                         ctypes.POINTER(Stats)]
            lib.oracle_remap_coeffs.restype = ctypes.c_int
            lib.oracle_remap_coeffs.argtypes = [I32, P, P, I64, P]
            lib.oracle_adjoint.restype = ctypes.c_int
            lib.oracle_adjoint.argtypes = [I64, I64, P, P, P, P, P, I32, P, P, I32, P, P, P, P, P, P, D, I32, D,
                                           I32, ctypes.c_int, P, P, P, P]
            _LIB = lib
    return _LIB


def _c(a, dtype):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _mesh_args(mesh):
    vol = _c(mesh.volume, np.float64)
    fc = _c(mesh.face_cells, np.int32)
    ar = _c(mesh.area, np.float64)
    nr = _c(mesh.normal, np.float64)
    fl = _c(mesh.flags, np.uint8)
    keep = (vol, fc, ar, nr, fl)
    return keep, (mesh.n_cells, mesh.n_faces, _ptr(vol), _ptr(fc), _ptr(ar), _ptr(nr), _ptr(fl))


def levels(mesh, omega, threads: int = 1, dc_n: int = 0):
    """Wavefront level of every cell for every direction, and the depth per direction (dc_n > 0: the
    dependency graph of direction-conserving transport to dc_n neighbours)."""
    om = _c(omega, np.float64).reshape(-1, 3)
    keep, margs = _mesh_args(mesh)
    D = om.shape[0]
    lev = np.zeros((D, mesh.n_cells), np.int32)
    depth = np.zeros(D, np.int32)
    rc = _lib().oracle_levels(*margs, D, _ptr(om), dc_n, _ptr(lev), _ptr(depth), threads)
    return rc, lev, depth


def solve(mesh, omega, weight, kappa_abs, emissivity, kappa_scat=None, bc_inflow=None, tol_scat=1e-6,
          max_it_scat=100, tol_pbc=1e-6, max_it_pbc=100, prev_init=None, threads: int = 1,
          want_intensity: bool = False, fused: bool = False, law: str = "balance", dc_n: int = 0):
    """Mean intensity J[N,G], absorbed rate Gamma[N,G], stats (and I[D,N,G] if asked)."""
    om = _c(omega, np.float64).reshape(-1, 3)
    w = _c(weight, np.float64)
    ka = _c(kappa_abs, np.float64)
    N = mesh.n_cells
    G = ka.reshape(N, -1).shape[1] if N else 1
    ka = ka.reshape(N, G)
    em = _c(emissivity, np.float64).reshape(N, G)
    ks = None if kappa_scat is None else _c(kappa_scat, np.float64).reshape(N, G)
    bc = None if bc_inflow is None else _c(bc_inflow, np.float64)
    pi = None if prev_init is None else _c(prev_init, np.float64)
    keep, margs = _mesh_args(mesh)
    D = om.shape[0]
    J = np.zeros((N, G))
    Gam = np.zeros((N, G))
    I = np.zeros((D, N, G)) if want_intensity else None
    st = Stats()
    rc = _lib().oracle_solve(*margs, D, _ptr(om), _ptr(w), G, _ptr(ka), _ptr(ks), _ptr(em), _ptr(bc), tol_scat,
                             max_it_scat, tol_pbc, max_it_pbc, _ptr(pi), int(fused), LAWS[law], dc_n, threads, _ptr(J),
                             _ptr(Gam),
                             _ptr(I),
                             ctypes.byref(st))
    out = {"rc": rc, "J": J, "Gamma": Gam, "stats": st.as_dict()}
    if want_intensity:
        out["I"] = I
    return out


def adjoint(mesh, omega, weight, kappa_abs, emissivity, dl_dJ=None, dl_dGamma=None, bc_inflow=None,
            threads: int = 1):
    """Gradients (dL/dkappa_abs, dL/demissivity) [N,G] of a loss with the given dL/dJ and dL/dGamma."""
    r = adjoint_full(mesh, omega, weight, kappa_abs, emissivity, dl_dJ=dl_dJ, dl_dGamma=dl_dGamma,
                     bc_inflow=bc_inflow, threads=threads)
    return r["rc"], r["grad_kappa_abs"], r["grad_emissivity"]


def adjoint_full(mesh, omega, weight, kappa_abs, emissivity, kappa_scat=None, dl_dJ=None, dl_dGamma=None,
                 bc_inflow=None, tol_scat=1e-6, max_it_scat=100, tol_pbc=1e-6, max_it_pbc=100, threads: int = 1):
    """The adjoint through the scattering and periodic iterations (their transpose): a dict with rc, the
    gradients in kappa_abs, emissivity and kappa_scat [N,G], and the forward sweep and transposed pass
    counts."""
    om = _c(omega, np.float64).reshape(-1, 3)
    w = _c(weight, np.float64)
    N = mesh.n_cells
    ka = _c(kappa_abs, np.float64).reshape(N, -1)
    G = ka.shape[1]
    em = _c(emissivity, np.float64).reshape(N, G)
    ks = None if kappa_scat is None else _c(kappa_scat, np.float64).reshape(N, G)
    dj = None if dl_dJ is None else _c(dl_dJ, np.float64).reshape(N, G)
    dg = None if dl_dGamma is None else _c(dl_dGamma, np.float64).reshape(N, G)
    bc = None if bc_inflow is None else _c(bc_inflow, np.float64)
    keep, margs = _mesh_args(mesh)
    gk = np.zeros((N, G))
    ge = np.zeros((N, G))
    gs = np.zeros((N, G))
    its = np.zeros(2, np.int32)
    rc = _lib().oracle_adjoint(*margs, om.shape[0], _ptr(om), _ptr(w), G, _ptr(ka), _ptr(ks), _ptr(em), _ptr(bc),
                               _ptr(dj), _ptr(dg), tol_scat, max_it_scat, tol_pbc, max_it_pbc, threads, _ptr(gk),
                               _ptr(ge), _ptr(gs), _ptr(its))
    return {"rc": rc, "grad_kappa_abs": gk, "grad_emissivity": ge, "grad_kappa_scat": gs,
            "it_forward": int(its[0]), "it_adjoint": int(its[1])}


def remap_coeffs(omega_old, omega_new, n_quad: int = 1 << 16):
    """c[i][j] = dS_ij / dS_i between a direction set and its rotation (the rotation paragraph of
    Sec. 2.6): the solid angle that the bin of new direction i shares with the bin of old direction j,
    over the solid angle of bin i, by a Fibonacci-sphere quadrature of n_quad points."""
    a = _c(omega_old, np.float64).reshape(-1, 3)
    b = _c(omega_new, np.float64).reshape(-1, 3)
    D = a.shape[0]
    c = np.zeros((D, D))
    rc = _lib().oracle_remap_coeffs(D, _ptr(a), _ptr(b), n_quad, _ptr(c))
    if rc != OK:
        raise RuntimeError("oracle_remap_coeffs failed: %d" % rc)
    return c


def rotation(theta: float, phi: float) -> np.ndarray:
    """R(theta, phi) = R_z(phi) R_y(theta): a rotation by theta about y, then by phi about z (the two
    spherical angles of the rotation paragraph of Sec. 2.6)."""
    ct, st, cp, sp = np.cos(theta), np.sin(theta), np.cos(phi), np.sin(phi)
    ry = np.array([[ct, 0.0, st], [0.0, 1.0, 0.0], [-st, 0.0, ct]])
    rz = np.array([[cp, -sp, 0.0], [sp, cp, 0.0], [0.0, 0.0, 1.0]])
    return rz @ ry


def rotate(omega, R):
    """Omega'_i = R Omega_i, each component ((R_k0 x + R_k1 y) + R_k2 z) separately rounded."""
    om = _c(omega, np.float64).reshape(-1, 3)
    R = np.asarray(R, np.float64)
    out = np.empty_like(om)
    for k in range(3):
        out[:, k] = (R[k, 0] * om[:, 0] + R[k, 1] * om[:, 1]) + R[k, 2] * om[:, 2]
    return out
