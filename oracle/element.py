"""Two-dimensional tensor-product element of Section 2.2 (plain FP64, test infrastructure).

The PDE is -div(alpha grad phi) + beta phi = f with Robin data n.(alpha grad phi) + gamma phi = q
(eqs. prototype_pde, prototype_robin).  For the Helmholtz problems here alpha = I,
beta = -k^2 eps_e (constant per element), gamma = -i k and q = g on the boundary of [0,1]^2.

On an axis-aligned square of side h the effective parameters (Sec. 2.2.2) are
alpha_eff = alpha, beta_eff = beta (h/2)^2, gamma_eff = gamma h/2, q_eff = q h/2.
Matrices follow Table 1 with constant coefficients (sum_k alpha_k T_k = I for alpha = 1):
  S11 = M1 (x) K1,  S22 = K1 (x) M1,  S12 = 0 (alpha_12 = 0),  M = beta_eff M1 (x) M1,
where the first Kronecker factor acts on the x2 index and vec(Phi) stacks columns
(x1 index fastest).  Robin matrices R_i and load vectors r_i follow the R_i / r_i cases
with e1 +- e2 selecting N(+-1).

Pins (tests/test_oracle_element.py): the bilinear form against brute-force 2-D Gauss
quadrature of the basis functions; the Galerkin residual of an exactly representable
polynomial; the plane-wave discretisation error decaying spectrally in p.
"""
from __future__ import annotations

import numpy as np

from . import legendre as lg


def side_vector(p: int, side: int) -> np.ndarray:
    """(e1 + (-1)^i e2) for side i = 1 (x=-1), 2 (x=+1), 3 (y=-1), 4 (y=+1)."""
    w = np.zeros(p + 1)
    w[0] = 1.0
    w[1] = 1.0 if side in (2, 4) else -1.0
    return w


def element_matrix_N(p: int, beta_eff: complex, robin: dict[int, complex]) -> np.ndarray:
    """Element matrix in the N basis; robin maps side index -> gamma_eff."""
    M1 = lg.mass_1d(p)
    K1 = lg.stiff_1d(p)
    A = np.kron(M1, K1) + np.kron(K1, M1) + beta_eff * np.kron(M1, M1)
    A = A.astype(complex)
    for side, gam in robin.items():
        w = side_vector(p, side)
        E = 0.5 * np.outer(w, w)
        if side in (1, 2):
            A += gam * np.kron(M1, E)
        else:
            A += gam * np.kron(E, M1)
    return A


def stiffness_matrix_N(p: int) -> np.ndarray:
    """The part of the element matrix from -div(grad phi) only (used by the preconditioner)."""
    M1 = lg.mass_1d(p)
    K1 = lg.stiff_1d(p)
    return np.kron(M1, K1) + np.kron(K1, M1)


def mass_matrix_N(p: int) -> np.ndarray:
    M1 = lg.mass_1d(p)
    return np.kron(M1, M1)


def to_tilde(p: int, A: np.ndarray) -> np.ndarray:
    """(B (x) B) A (B (x) B): the same operator on the interpolatory basis N~ = B N."""
    B = lg.B_matrix(p)
    BB = np.kron(B, B)
    return BB @ A @ BB


def vec_to_tilde(p: int, v: np.ndarray) -> np.ndarray:
    B = lg.B_matrix(p)
    return np.kron(B, B) @ v


def robin_load_N(p: int, side: int, q_of_t, half_h: float, nq: int = 0) -> np.ndarray:
    """r_i = S q_i (x) (e1 +- e2)/sqrt(2) (or the mirrored Kronecker order for i = 3,4),
    with q_i = int q_eff(t) p(t) dt the Legendre coefficients of q_eff = q h/2 along the side,
    computed by Gauss-Legendre quadrature (evaluating the integrals directly, one of the paper's options)."""
    nq = nq or (p + 40)
    t, w = lg.gauss_legendre(nq)
    qi = (lg.legendre_p(p, t) * w) @ (np.asarray(q_of_t(t), dtype=complex) * half_h)
    Sq = lg.S_matrix(p) @ qi
    sv = side_vector(p, side) / np.sqrt(2.0)
    if side in (1, 2):
        return np.kron(Sq, sv)
    return np.kron(sv, Sq)


def volume_load_N(p: int, f_of_xy, x0: float, y0: float, h: float, nq: int = 0) -> np.ndarray:
    """f~ = int N(x) f dOmega with f_eff = f (h/2)^2, by tensor Gauss-Legendre quadrature."""
    nq = nq or (p + 30)
    t, w = lg.gauss_legendre(nq)
    N = lg.N_basis(p, t)                       # (p+1, nq)
    X = x0 + 0.5 * h * (1.0 + t)
    Y = y0 + 0.5 * h * (1.0 + t)
    F = np.asarray(f_of_xy(X[:, None], Y[None, :]), dtype=complex)  # F[i1, i2]
    G = (N * w) @ F @ (N * w).T                # G[a, b] = sum N_a(t1) N_b(t2) f w w
    return (G * (0.5 * h) ** 2).reshape(-1, order="F")


def evaluate_N(p: int, phi: np.ndarray, u1, u2) -> np.ndarray:
    """phi(u) = N(u1)^T Phi N(u2) at canonical points (u1, u2) (arrays of equal shape)."""
    Phi = phi.reshape(p + 1, p + 1, order="F")
    N1 = lg.N_basis(p, np.asarray(u1))
    N2 = lg.N_basis(p, np.asarray(u2))
    return np.einsum("a...,ab,b...->...", N1, Phi, N2)
