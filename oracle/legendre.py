"""One-dimensional polynomial algebra of Section 2.1 (plain FP64, test infrastructure).

Pins (tests/test_oracle_legendre.py): orthonormality under Gauss quadrature; the
derivative matrix against finite differences of the recurrence; N(+-1); the
Jacobi eigen-ODE of N_k; L against pointwise evaluation of p(ax+b); L_kk = a^k.
"""
from __future__ import annotations

import numpy as np


def legendre_p(n: int, x) -> np.ndarray:
    """Orthonormal Legendre polynomials p_0..p_n at x (Sec. 2.1, eq. recurrence_relation),
    p_0 = 1/sqrt(2), p_1 = sqrt(3/2) x.  Returns shape (n+1,) + x.shape."""
    x = np.asarray(x, dtype=float)
    P = np.zeros((n + 1,) + x.shape)
    P[0] = 1.0 / np.sqrt(2.0)
    if n >= 1:
        P[1] = np.sqrt(1.5) * x
    for k in range(2, n + 1):
        P[k] = (np.sqrt((2 * k + 1) * (2 * k - 1)) / k) * x * P[k - 1] \
            - ((k - 1) / k) * np.sqrt((2 * k + 1) / (2 * k - 3)) * P[k - 2]
    return P


def gauss_legendre(m: int):
    """Gauss-Legendre nodes and weights on (-1,1) (library primitive)."""
    return np.polynomial.legendre.leggauss(m)


def D_matrix(n: int) -> np.ndarray:
    """Differentiation d/dx p = D p, d_ij = sqrt((2i-1)(2j-1)) for i>j, i+j odd (1-based)."""
    D = np.zeros((n + 1, n + 1))
    for i in range(1, n + 2):
        for j in range(1, n + 2):
            if i > j and (i + j) % 2 == 1:
                D[i - 1, j - 1] = np.sqrt((2 * i - 1) * (2 * j - 1))
    return D


def g_vector(n: int) -> np.ndarray:
    """g_1 = 1, g_i = 1/sqrt((2i-1)(2i-3)) for i>=2 (1-based), length n+1."""
    g = np.zeros(n + 1)
    g[0] = 1.0
    for i in range(2, n + 2):
        g[i - 1] = 1.0 / np.sqrt((2 * i - 1) * (2 * i - 3))
    return g


def SDL(n: int) -> np.ndarray:
    """Down-shift matrix (s_DL)_ij = delta_{i,j+1}."""
    return np.eye(n + 1, k=-1)


def S_matrix(n: int) -> np.ndarray:
    """N = S p with S = diag(g) - S_DL diag(g) S_DL (eq. define_basis_functions)."""
    g = np.diag(g_vector(n))
    Sd = SDL(n)
    return g - Sd @ g @ Sd


def N_basis(n: int, x) -> np.ndarray:
    """Integrated Legendre basis N_0..N_n at x."""
    return S_matrix(n) @ legendre_p(n, x)


def Q_matrix() -> np.ndarray:
    return np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)


def B_matrix(n: int) -> np.ndarray:
    """B = diag(Q, I): N~ = B N with N~_0 = (1+x)/2, N~_1 = (1-x)/2 (eq. interpolatory_relation)."""
    B = np.eye(n + 1)
    B[:2, :2] = Q_matrix()
    return B


def mass_1d(n: int) -> np.ndarray:
    """int N N^T dx = S S^T (orthonormality of p)."""
    S = S_matrix(n)
    return S @ S.T


def stiff_1d(n: int) -> np.ndarray:
    """int N' N'^T dx = S_DL S_DL^T (eq. differentiation_property)."""
    Sd = SDL(n)
    return Sd @ Sd.T


def affine_L(n: int, a: float, b: float) -> np.ndarray:
    """L with p(ax+b) = L p(x), computed from its defining integral
    L = int p(ax+b) p(x)^T dx by Gauss-Legendre quadrature (exact for these degrees)."""
    x, w = gauss_legendre(n + 4)
    Pa = legendre_p(n, a * x + b)
    P = legendre_p(n, x)
    return (Pa * w) @ P.T


def affine_L_N(n: int, a: float, b: float) -> np.ndarray:
    """Change of basis L_c^f = S L S^{-1} so that N(ax+b) = L_c^f N(x)."""
    S = S_matrix(n)
    return S @ affine_L(n, a, b) @ np.linalg.inv(S)


def affine_L_tilde(n: int, a: float, b: float) -> np.ndarray:
    """The same change of basis for the interpolatory basis: N~(ax+b) = B L_c^f B N~(x)."""
    B = B_matrix(n)
    return B @ affine_L_N(n, a, b) @ B
