"""Axis-aligned perfectly matched layers (Sec. 4, PML paragraph): test infrastructure only.

Complex coordinate stretching s_i = 1 - i sigma_i / k along each axis, with sigma_i piecewise
constant per element (non-zero only in the layer bands), turns -lap phi - k^2 phi = f into

    -div(Lambda grad phi) - k^2 s_1 s_2 phi = f,   Lambda = det(S) S^-2 = diag(s_2/s_1, s_1/s_2),

the scalar form of the paper's eps_PML = Lambda eps, mu_PML = Lambda mu.  (The sign follows the
time convention of the outgoing H0^(2) field of the Dirichlet test: waves exp(-i k x) travel
towards +x and decay as exp(-int sigma) inside a layer.)  On a square element the operator stays
a sum of Kronecker products,

    A_e = (s_2/s_1) K(x1) M(x2) + (s_1/s_2) M(x1) K(x2) - k^2 s_1 s_2 (h/2)^2 M (x) M,

so the element interiors keep a separable fast solver (complex generalized eigenvalues).  The
layered problem is closed by Dirichlet data on the outer boundary and solved by the dual-primal
split of oracle/poisson.py (the constraint rows of oracle/dirichlet.py) with the unscaled
Dirichlet preconditioner on the unstretched stiffness and FGMRES.

Pins in tests/test_oracle_pml.py: with a layer the exact solution of the stretched problem is
exp(-i k x~(x)), x~ = x - (i/k) int sigma_1 -- continuous and smooth per element -- and the field
converges to it spectrally; with zero data beyond the layer the field in the physical region is
the unbounded plane wave up to the layer's round-trip reflection exp(-2 int sigma_1); without
a layer the operator is the plain Helmholtz one of oracle/dirichlet.py.
"""
from __future__ import annotations

import numpy as np

from . import dirichlet as D
from . import poisson as P
from .fgmres import fgmres


def stretch(m: int, k: float, cells: int, sigma: float, axes=(0,)):
    """Per element (e = i + m j) the factors s_1, s_2: 1 - i sigma/k in the last `cells` columns
    (axis 0) and / or rows (axis 1) of the m x m grid, 1 elsewhere."""
    s1 = np.ones(m * m, complex)
    s2 = np.ones(m * m, complex)
    for e in range(m * m):
        i, j = e % m, e // m
        if 0 in axes and i >= m - cells:
            s1[e] = 1.0 - 1j * sigma / k
        if 1 in axes and j >= m - cells:
            s2[e] = 1.0 - 1j * sigma / k
    return s1, s2


def coefficients(m: int, k: float, s1, s2) -> np.ndarray:
    """[E, 3]: (s2/s1, s1/s2, -k^2 s1 s2 (h/2)^2) per element."""
    c = -(k * 0.5 / m) ** 2
    return np.stack([s2 / s1, s1 / s2, c * s1 * s2], axis=1)


def stretched_plane_wave(m: int, k: float, cells: int, sigma: float):
    """exp(-i k x~(x)) with x~ = x - (i/k) sigma max(0, x - x_layer): the exact solution of the
    stretched problem with a layer in the last `cells` columns."""
    x_layer = 1.0 - cells / m
    def f(x, y):
        x = np.asarray(x, float)
        xt = x - 1j * (sigma / k) * np.maximum(0.0, x - x_layer)
        return np.exp(-1j * k * xt) + 0.0 * np.asarray(y)
    return f


class Solver:
    """Dual-primal solve of the stretched problem on 2^n x 2^n squares, Dirichlet data outside."""

    def __init__(self, n: int, p: int, l: int, k: float, s1, s2):
        m = 2 ** n
        self.n, self.p, self.l, self.k = n, p, l, k
        self.coef = coefficients(m, k, s1, s2)
        self.dd = P.build(n, p, l, rho=np.ones(m * m), k=k, coef=self.coef)
        self.S = P.Solver(self.dd, scaled=False)
        from .element import mass_matrix_N
        from . import legendre as lg
        M1, K1 = lg.mass_1d(p), lg.stiff_1d(p)
        self.A_N = [c[0] * np.kron(M1, K1) + c[1] * np.kron(K1, M1) + c[2] * mass_matrix_N(p) for c in self.coef]

    def apply_A_N(self, phi_N):
        N2 = (self.p + 1) ** 2
        return np.concatenate([self.A_N[e] @ phi_N[e * N2:(e + 1) * N2] for e in range(len(self.A_N))])

    def solve(self, b_N, g_N, tol=1e-10, restart=200, maxit=400):
        """phi = g + phi_0 (N basis): g the Dirichlet lifting, phi_0 the zero-data solve."""
        dd, S = self.dd, self.S
        bG = b_N - self.apply_A_N(g_N)
        bh = dd.Z.T @ (dd.B @ bG)
        y1, _ = S.Ahat_solve(bh[:dd.n1], bh[dd.n1:])
        rhs = S.C1 @ y1
        if dd.nd:
            Fop = lambda v: S.apply_F(v)
            Pop = lambda v: S.apply_P(v.real) + 1j * S.apply_P(v.imag)
            nu, its, _ = fgmres(Fop, Pop, rhs.astype(complex), tol=tol, restart=restart, maxit=maxit)
        else:
            nu, its = np.zeros(0, complex), 0
        x1, x2 = S.Ahat_solve(bh[:dd.n1] - S.C1.T @ nu, bh[dd.n1:])
        return g_N + dd.B @ (dd.Z @ np.concatenate([x1, x2])), its


def lifting(n: int, p: int, data):
    """The Dirichlet lifting of oracle/dirichlet.py (vertex values, L^2-projection bubbles)."""
    return D.lifting(n, p, data)
