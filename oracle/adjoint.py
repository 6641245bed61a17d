"""Adjoint gradient of a point objective (test infrastructure; no counterpart in the paper,
which has no adjoint -- this differentiates its discretisation).

J = sum_i |u(x_i)|^2 for the solution of the conforming (globally assembled) system.  With
G = 2 u(x_i) at the points (PyTorch's conj(2 dJ/du) convention) and the point-evaluation
functionals e_i, the transposed adjoint A^T lam = sum_i conj(G_i) e_i is an ordinary solve
(A complex symmetric), and dJ/deps_e = k^2 (h_e/2)^2 Re(lam_e^T (M (x) M) u_e).

Pin (tests/test_oracle_adjoint.py): central finite differences of J on direct solves.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import element as el
from . import legendre as lg
from .constraints import element_offsets
from .dd import Conforming, Problem, build_problem, element_geometry, field_at, to_tilde_vec


def solve_load(prob: Problem, b_N: np.ndarray) -> np.ndarray:
    """Conforming solution for an arbitrary element-local load (N basis, [R, n_local])."""
    conf = Conforming(prob)
    Ac = (conf.Zc.T @ conf.A @ conf.Zc).tocsc()
    bt = to_tilde_vec(prob, np.atleast_2d(b_N))
    u = spla.splu(Ac).solve((bt @ conf.Zc).T).T
    return to_tilde_vec(prob, (conf.Zc @ u.T).T)


def point_functionals(prob: Problem, pts: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """sum_i w_i e_i as an element-local vector (N basis): e_i[a + (p+1) b] = N_a(u1) N_b(u2)."""
    mesh = prob.mesh
    off = element_offsets(mesh)
    out = np.zeros(int(off[-1]), complex)
    for (x, y), w in zip(pts, weights):
        for e in range(mesh.n_elem):
            x0, y0, h = element_geometry(mesh, e)
            if x0 <= x <= x0 + h and y0 <= y <= y0 + h:
                p = int(mesh.p[e])
                N1 = lg.N_basis(p, 2 * (x - x0) / h - 1)
                N2 = lg.N_basis(p, 2 * (y - y0) / h - 1)
                out[off[e]:off[e + 1]] += w * np.outer(N1, N2).reshape(-1, order="F")
                break
    return out


def objective(prob: Problem, phi_N: np.ndarray, pts: np.ndarray):
    vals = field_at(prob, phi_N, pts[:, 0], pts[:, 1])
    return float(np.sum(np.abs(vals) ** 2)), vals


def gradient_eps(prob: Problem, pts: np.ndarray):
    """(J, dJ/deps [E], phi) by the adjoint formula on direct solves."""
    phi = solve_load(prob, prob.b_N)[0]
    J, vals = objective(prob, phi, pts)
    G = 2.0 * vals
    g = point_functionals(prob, pts, np.conj(G))
    lam = solve_load(prob, g[None, :])[0]
    mesh = prob.mesh
    off = element_offsets(mesh)
    grad = np.zeros(mesh.n_elem)
    for e in range(mesh.n_elem):
        p = int(mesh.p[e])
        h = float(mesh.h[e])
        M = el.mass_matrix_N(p)
        s = lam[off[e]:off[e + 1]] @ (M @ phi[off[e]:off[e + 1]])
        grad[e] = prob.k ** 2 * (0.5 * h) ** 2 * s.real
    return J, grad, phi


def fd_gradient(w, pts: np.ndarray, index, step: float = 1e-6) -> np.ndarray:
    """Central differences of J in eps_e for the listed elements (direct solves)."""
    out = []
    for e in index:
        vals = []
        for sgn in (1.0, -1.0):
            eps = np.array(w.eps, float).copy()
            eps[e] += sgn * step
            prob = build_problem(w.base_n, w.leaves, w.p, eps, w.k, w.thetas[:1])
            phi = solve_load(prob, prob.b_N)[0]
            vals.append(objective(prob, phi, pts)[0])
        out.append((vals[0] - vals[1]) / (2 * step))
    return np.array(out)
