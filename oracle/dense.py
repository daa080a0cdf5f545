"""Dense-matrix second oracle for small meshes (<= ~512 cells) -- TEST INFRASTRUCTURE ONLY.

Independent of ``sweep_oracle.c``: it assembles the discretised transport system
of the paper's Sec. 2.6 transport scheme (a) as an explicit matrix from the face
list and solves it with LU (numpy.linalg.solve), with no ordering, no queue and
no iteration. For one direction Omega (paper Sec. 2.3: ordering the cells makes
this matrix lower triangular; here it is simply solved):

    row c:  (P_c + kappa_t,c V_c) I_c  -  sum_{faces f with inflow into c} |a_f| I_other(f)  =  q_c (+ boundary inflow)
    a_f = A_f n_f . Omega,  P_c = sum over faces with outward n.Omega > 0 of |a_f|

The EXP law (solve_coupled_exp) is the same kind of system with the outgoing intensity
P_c I_c = exp(-tau_c) F_in,c + q_c, tau_c = kappa_t,c V_c / P_c, and J formed from the cell mean
(F_in,c / P_c)(1 - exp(-tau_c)) / tau_c.

Periodic faces enter as ordinary couplings to the partner cell, so the matrix is
cyclic and its solution is the fixed point the periodic iteration of Sec. 2.7
converges to. Isotropic scattering couples the directions through
q_c = eps_c/4pi + kappa_s,c V_c (1/4pi) sum_d' w_d' I_c,d' (Alg. 1's fixed point).
"""
from __future__ import annotations

import math

import numpy as np

FACE_BOUNDARY = 1
FACE_PERIODIC = 2


def _dot(n, om):
    # same rounding order as the classification: ((x) + (y)) + (z)
    return (n[..., 0] * om[0] + n[..., 1] * om[1]) + n[..., 2] * om[2]


def transport_matrix(mesh, om, kappa_t, bc_inflow=None, group=0, periodic_coupling=True):
    """Matrix L (N x N) and boundary right-hand side b (N) for one direction and group."""
    N = mesh.n_cells
    L = np.zeros((N, N))
    b = np.zeros(N)
    t = _dot(mesh.normal, om)
    a = mesh.area * np.abs(t)
    bidx = np.cumsum((mesh.flags & FACE_BOUNDARY) != 0) - 1
    for f in range(mesh.n_faces):
        c0, c1 = int(mesh.face_cells[f, 0]), int(mesh.face_cells[f, 1])
        if t[f] == 0.0:
            continue
        if mesh.flags[f] & FACE_BOUNDARY:
            if t[f] > 0:
                L[c0, c0] += a[f]
            elif bc_inflow is not None:
                b[c0] += a[f] * bc_inflow[bidx[f], group]
            continue
        up, down = (c0, c1) if t[f] > 0 else (c1, c0)
        L[up, up] += a[f]                      # outflow of the upwind cell
        if (mesh.flags[f] & FACE_PERIODIC) and not periodic_coupling:
            continue
        L[down, up] -= a[f]                    # inflow of the downwind cell
    L[np.arange(N), np.arange(N)] += kappa_t[:, group] * mesh.volume
    return L, b


def solve_direction(mesh, om, kappa_abs, emissivity, kappa_scat=None, bc_inflow=None):
    """I[N,G] for one direction with scattering treated as absent."""
    kt = kappa_abs + (0.0 if kappa_scat is None else kappa_scat)
    G = kappa_abs.shape[1]
    I = np.zeros((mesh.n_cells, G))
    for g in range(G):
        L, b = transport_matrix(mesh, om, kt, bc_inflow, g)
        I[:, g] = np.linalg.solve(L, emissivity[:, g] / (4 * math.pi) + b)
    return I


def coupled_matrix(mesh, omega, weight, kappa_t, kappa_scat, group, bc_inflow=None):
    """The whole system of one group, all directions with the isotropic scattering coupling:
    A [D*N, D*N] and the boundary part b of the right-hand side."""
    D, N = omega.shape[0], mesh.n_cells
    A = np.zeros((D * N, D * N))
    b = np.zeros(D * N)
    idx = np.arange(N)
    for d in range(D):
        L, bd = transport_matrix(mesh, omega[d], kappa_t, bc_inflow, group)
        A[d * N:(d + 1) * N, d * N:(d + 1) * N] = L
        b[d * N:(d + 1) * N] = bd
        for d2 in range(D):
            A[d * N + idx, d2 * N + idx] -= kappa_scat[:, group] * mesh.volume * weight[d2] / (4 * math.pi)
    return A, b


def solve_coupled(mesh, omega, weight, kappa_abs, emissivity, kappa_scat=None, bc_inflow=None):
    """All directions at once with isotropic scattering coupling; returns I[D,N,G], J[N,G], Gamma[N,G]."""
    D, N = omega.shape[0], mesh.n_cells
    G = kappa_abs.shape[1]
    ks = np.zeros_like(kappa_abs) if kappa_scat is None else kappa_scat
    kt = kappa_abs + ks
    I = np.zeros((D, N, G))
    for g in range(G):
        A, b = coupled_matrix(mesh, omega, weight, kt, ks, g, bc_inflow)
        rhs = np.tile(emissivity[:, g] / (4 * math.pi), D) + b
        I[:, :, g] = np.linalg.solve(A, rhs).reshape(D, N)
    J = np.einsum("d,dng->ng", weight, I) / (4 * math.pi)
    Gam = kappa_abs * mesh.volume[:, None] * 4 * math.pi * J
    return I, J, Gam


def adjoint_coupled(mesh, omega, weight, kappa_abs, kappa_scat, g_src):
    """lambda[D,N,G] solving A^T lambda = g for the coupled system of every group (no periodic faces)."""
    D, N = omega.shape[0], mesh.n_cells
    G = kappa_abs.shape[1]
    lam = np.zeros((D, N, G))
    for g in range(G):
        A, _ = coupled_matrix(mesh, omega, weight, kappa_abs + kappa_scat, kappa_scat, g, None)
        lam[:, :, g] = np.linalg.solve(A.T, g_src[:, :, g].reshape(D * N)).reshape(D, N)
    return lam


def adjoint_direction(mesh, om, kappa_abs, g_src):
    """lambda[N,G] solving L^T lambda = g for one direction (no scattering, no periodic faces)."""
    G = kappa_abs.shape[1]
    lam = np.zeros((mesh.n_cells, G))
    for g in range(G):
        L, _ = transport_matrix(mesh, om, kappa_abs, None, g)
        lam[:, g] = np.linalg.solve(L.T, g_src[:, g])
    return lam


# ---- the EXP law: outgoing (exp(-tau) F_in + q) / P, cell mean (F_in / P)(1 - exp(-tau)) / tau ----
def inflow_operator(mesh, om, bc_inflow=None, group=0, dc_n=0):
    """For one direction: M (N x N) and b (N) with the inflow flux F_in = M I + b of every cell, and
    the projected outflow area P (N). Periodic faces couple to the partner cell. dc_n > 0: the flux
    of scheme (b) (dc_operator) instead of A |n . Omega| per face."""
    N = mesh.n_cells
    if dc_n > 0:
        L, b, _ = dc_operator(mesh, om, np.zeros((N, group + 1)), dc_n, bc_inflow, group)
        P = np.diag(L).copy()
        M = -(L - np.diag(np.diag(L)))
        return M, b, P
    M = np.zeros((N, N))
    b = np.zeros(N)
    P = np.zeros(N)
    t = _dot(mesh.normal, om)
    a = mesh.area * np.abs(t)
    bidx = np.cumsum((mesh.flags & FACE_BOUNDARY) != 0) - 1
    for f in range(mesh.n_faces):
        c0, c1 = int(mesh.face_cells[f, 0]), int(mesh.face_cells[f, 1])
        if t[f] == 0.0:
            continue
        if mesh.flags[f] & FACE_BOUNDARY:
            if t[f] > 0:
                P[c0] += a[f]
            elif bc_inflow is not None:
                b[c0] += a[f] * bc_inflow[bidx[f], group]
            continue
        up, down = (c0, c1) if t[f] > 0 else (c1, c0)
        P[up] += a[f]
        M[down, up] += a[f]
    return M, b, P


def _exp_factors(kt_V, P):
    tau = kt_V / P
    f = np.where(tau > 0, -np.expm1(-tau) / np.where(tau > 0, tau, 1.0), 1.0)
    return np.exp(-tau), f


def solve_coupled_exp(mesh, omega, weight, kappa_abs, emissivity, kappa_scat=None, bc_inflow=None, dc_n=0):
    """EXP law, all directions with isotropic scattering through the cell-mean J; returns the outgoing
    I[D,N,G], the cell mean Ibar[D,N,G], J[N,G] and Gamma[N,G]. dc_n > 0: scheme (b) transport."""
    D, N = omega.shape[0], mesh.n_cells
    G = kappa_abs.shape[1]
    ks = np.zeros_like(kappa_abs) if kappa_scat is None else kappa_scat
    I = np.zeros((D, N, G))
    Ibar = np.zeros((D, N, G))
    for g in range(G):
        ktV = (kappa_abs[:, g] + ks[:, g]) * mesh.volume
        ops = [inflow_operator(mesh, omega[d], bc_inflow, g, dc_n) for d in range(D)]
        assert all((P > 0).all() for _, _, P in ops)
        A = np.zeros((D * N, D * N))
        rhs = np.zeros(D * N)
        # mean operator of each direction: Ibar_d = diag(f_d / P_d) (M_d I_d + b_d)
        mean_op = []
        for d, (M, b, P) in enumerate(ops):
            e, f = _exp_factors(ktV, P)
            mean_op.append(((f / P)[:, None] * M, (f / P) * b))
            sl = slice(d * N, (d + 1) * N)
            A[sl, sl] = np.diag(P) - e[:, None] * M
            rhs[sl] = emissivity[:, g] / (4 * math.pi) + e * b
        c = ks[:, g] * mesh.volume / (4 * math.pi)
        for d in range(D):
            for d2 in range(D):
                Mm, bm = mean_op[d2]
                A[d * N:(d + 1) * N, d2 * N:(d2 + 1) * N] -= weight[d2] * c[:, None] * Mm
                rhs[d * N:(d + 1) * N] += weight[d2] * c * bm
        I[:, :, g] = np.linalg.solve(A, rhs).reshape(D, N)
        for d in range(D):
            Mm, bm = mean_op[d]
            Ibar[d, :, g] = Mm @ I[d, :, g] + bm
    J = np.einsum("d,dng->ng", weight, Ibar) / (4 * math.pi)
    Gam = kappa_abs * mesh.volume[:, None] * 4 * math.pi * J
    return I, Ibar, J, Gam


# ---- direction-conserving transport, scheme (b): equal parts to the n faces most nearly along Omega ----
def dc_operator(mesh, om, kappa_t, n, bc_inflow=None, group=0):
    """Matrix L (N x N) and boundary right-hand side b (N) of scheme (b) for one direction: row c is
    (P_c + kappa_t,c V_c) I_c - sum over the cells u that chose a face to c of (P_u / n_u) I_u. Also
    returns the downwind dependencies {u: [cells u hands flux to]} over interior, non-periodic faces."""
    N = mesh.n_cells
    t = _dot(mesh.normal, om)
    a = mesh.area * np.abs(t)
    bidx = np.cumsum((mesh.flags & FACE_BOUNDARY) != 0) - 1
    out = [[] for _ in range(N)]  # (n . Omega outward, face, downwind cell or -1)
    L = np.zeros((N, N))
    b = np.zeros(N)
    P = np.zeros(N)
    for f in range(mesh.n_faces):
        c0, c1 = int(mesh.face_cells[f, 0]), int(mesh.face_cells[f, 1])
        if t[f] == 0.0:
            continue
        if mesh.flags[f] & FACE_BOUNDARY:
            if t[f] > 0:
                out[c0].append((t[f], f, -1))
                P[c0] += a[f]
            elif bc_inflow is not None:
                b[c0] += a[f] * bc_inflow[bidx[f], group]
            continue
        up, down, tu = (c0, c1, t[f]) if t[f] > 0 else (c1, c0, -t[f])
        out[up].append((tu, f, down))
        P[up] += a[f]
    deps = {}
    for u in range(N):
        chosen = sorted(out[u], key=lambda x: (-x[0], x[1]))[:n]
        if not chosen:
            continue
        share = P[u] / len(chosen)
        for _, f, down in chosen:
            if down >= 0:
                L[down, u] -= share
                if not (mesh.flags[f] & FACE_PERIODIC):
                    deps.setdefault(u, []).append(down)
    L[np.arange(N), np.arange(N)] += P + kappa_t[:, group] * mesh.volume
    return L, b, deps


def solve_coupled_dc(mesh, omega, weight, kappa_abs, emissivity, n, kappa_scat=None, bc_inflow=None):
    """Scheme (b), BALANCE law, all directions with isotropic scattering; returns I[D,N,G], J, Gamma."""
    D, N = omega.shape[0], mesh.n_cells
    G = kappa_abs.shape[1]
    ks = np.zeros_like(kappa_abs) if kappa_scat is None else kappa_scat
    kt = kappa_abs + ks
    I = np.zeros((D, N, G))
    idx = np.arange(N)
    for g in range(G):
        A = np.zeros((D * N, D * N))
        rhs = np.zeros(D * N)
        for d in range(D):
            L, bd, _ = dc_operator(mesh, omega[d], kt, n, bc_inflow, g)
            A[d * N:(d + 1) * N, d * N:(d + 1) * N] = L
            rhs[d * N:(d + 1) * N] = emissivity[:, g] / (4 * math.pi) + bd
            for d2 in range(D):
                A[d * N + idx, d2 * N + idx] -= ks[:, g] * mesh.volume * weight[d2] / (4 * math.pi)
        I[:, :, g] = np.linalg.solve(A, rhs).reshape(D, N)
    J = np.einsum("d,dng->ng", weight, I) / (4 * math.pi)
    Gam = kappa_abs * mesh.volume[:, None] * 4 * math.pi * J
    return I, J, Gam
