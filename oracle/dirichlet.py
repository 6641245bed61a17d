"""The Helmholtz test problem with Dirichlet data of Sec. 3.2 (Table 3): test infrastructure only.

-lap phi - k^2 phi = 0 on (-1,1)^2 with phi = -(i/4) H0^(2)(k |x - x_c|) on the boundary,
x_c = (-2, 1), so that the exact solution is that point-source field.  The square maps to the
unit square of the meshes here by x' = (x + 1)/2: the wavenumber becomes 2k and the centre
(-1/2, 1); the element matrices are unchanged (2-D stiffness does not depend on h, and
(k h / 2)^2 is the same).

Dirichlet data enter as constraints C_i phi = d_i on every boundary side (Sec. 2.2.1): the
rows pick the trace coefficients of the side in the N basis, and d_i = sqrt(2) S^-T p_i makes
the trace the L^2 projection of the data onto degree-p polynomials.  Reading of the corners:
the two sides meeting at a boundary vertex both constrain it, which for non-polynomial data
is inconsistent; the build keeps one constraint per boundary vertex, the data's point value
there, and every side's rows for the bubble coefficients m = 2..p (in the N basis these rows
pick the bubble coefficient alone, so they do not involve the vertices).

The solve splits phi = phi_G + phi_0: phi_G is the lifting that carries the boundary trace
(vertex values and bubble coefficients of the boundary sides, zero elsewhere), phi_0 solves
the problem with zero Dirichlet data and load b - A phi_G by the dual-primal method of
oracle/poisson.py (Algorithm 1 discards the boundary vertices and moments 2..l of boundary
sides, moments above l are single-sided dual rows) with the unscaled Dirichlet preconditioner
on the stiffness part (Sec. 2.3.3) and flexible GMRES (the paper uses left-preconditioned
PGMRES; iteration counts are context).

Pins in tests/test_oracle_dirichlet.py: the trace rule against the exact L^2 projection of a
polynomial (exact), spectral convergence of the field to the point-source solution, the
solution against the all-primal split, and Table 3 iteration counts.
"""
from __future__ import annotations

import numpy as np
import scipy.special as ss

from . import legendre as lg
from . import poisson as P
from .fgmres import fgmres
from .mesh import side_slot


def point_source(k: float, xc: float, yc: float):
    """phi(x, y) = -(i/4) H0^(2)(k r), r = |(x, y) - (xc, yc)| (unit-square coordinates)."""
    def f(x, y):
        r = np.hypot(np.asarray(x) - xc, np.asarray(y) - yc)
        return -0.25j * ss.hankel2(0, k * r)
    return f


def table3_problem(k_paper: float):
    """(k, data) on the unit square for the paper's wavenumber on (-1,1)^2 with x_c = (-2, 1)."""
    return 2.0 * k_paper, point_source(2.0 * k_paper, -0.5, 1.0)


def side_bubbles(p: int, data_of_t, nq: int = 0) -> np.ndarray:
    """N-basis coefficients tau = S^-T q of the L^2 projection of data(t) on [-1, 1] onto degree
    p (q_j = int data p_j dt with orthonormal Legendre p_j); entries 2..p are the bubbles."""
    nq = nq or (p + 40)
    t, w = lg.gauss_legendre(nq)
    q = (lg.legendre_p(p, t) * w) @ np.asarray(data_of_t(t), dtype=complex)
    return np.linalg.solve(lg.S_matrix(p).T, q)


def lifting(n: int, p: int, data) -> np.ndarray:
    """phi_G (element-local, N basis) on 2^n x 2^n squares of degree p: boundary vertex values
    = data at the vertex, boundary-side bubble coefficients = the L^2 projection's, zero
    elsewhere (interpolatory basis, then B (x) B back to the N basis)."""
    m = 2 ** n
    h = 1.0 / m
    N = p + 1
    Bl = lg.B_matrix(p)
    BB = np.kron(Bl, Bl)
    out = []
    for e in range(m * m):
        i, j = e % m, e // m
        x0, y0 = i * h, j * h
        phit = np.zeros(N * N, complex)
        # corners: a = 0 is x1 = +1 (x0 + h), a = 1 is x1 = -1 (x0); the same for b along x2
        for a in (0, 1):
            for b in (0, 1):
                on_x = (a == 1 and i == 0) or (a == 0 and i == m - 1)
                on_y = (b == 1 and j == 0) or (b == 0 and j == m - 1)
                if on_x or on_y:
                    phit[a + N * b] = data(x0 + (h if a == 0 else 0.0), y0 + (h if b == 0 else 0.0))
        sides = []
        if i == 0:
            sides.append((1, lambda t: data(x0 + 0 * t, y0 + 0.5 * h * (1 + t))))
        if i == m - 1:
            sides.append((2, lambda t: data(x0 + h + 0 * t, y0 + 0.5 * h * (1 + t))))
        if j == 0:
            sides.append((3, lambda t: data(x0 + 0.5 * h * (1 + t), y0 + 0 * t)))
        if j == m - 1:
            sides.append((4, lambda t: data(x0 + 0.5 * h * (1 + t), y0 + h + 0 * t)))
        for side, f in sides:
            tau = side_bubbles(p, f)
            for mm in range(2, N):
                phit[side_slot(p, side, mm)] = tau[mm]
        out.append(BB @ phit)
    return np.concatenate(out)


class Solver:
    """Dual-primal solve of the Dirichlet Helmholtz problem on 2^n x 2^n squares."""

    def __init__(self, n: int, p: int, l: int, k: float):
        self.n, self.p, self.l, self.k = n, p, l, k
        self.dd = P.build(n, p, l, rho=np.ones(4 ** n), k=k)
        self.S = P.Solver(self.dd, scaled=False)
        E = 4 ** n
        m = 2 ** n
        c = -(k * 0.5 / m) ** 2
        from .element import mass_matrix_N, stiffness_matrix_N
        self.A_N = [stiffness_matrix_N(p) + c * mass_matrix_N(p) for _ in range(E)]

    def _ahat(self, r1, r2):
        """The real block solve of oracle/poisson.py applied to real and imaginary parts."""
        a1, a2 = self.S.Ahat_solve(r1.real, r2.real)
        b1, b2 = self.S.Ahat_solve(r1.imag, r2.imag)
        return a1 + 1j * b1, a2 + 1j * b2

    def apply_A_N(self, phi_N):
        N2 = (self.p + 1) ** 2
        return np.concatenate([self.A_N[e] @ phi_N[e * N2:(e + 1) * N2] for e in range(len(self.A_N))])

    def solve(self, b_N, g_N, tol=1e-10, restart=200, maxit=400):
        """phi = g + phi_0 (N basis) for load b and lifting g; returns (phi, iterations, hist)."""
        dd, S = self.dd, self.S
        bG = b_N - self.apply_A_N(g_N)
        bh = dd.Z.T @ (dd.B @ bG)
        y1, _ = self._ahat(bh[:dd.n1], bh[dd.n1:])
        rhs = S.C1 @ y1
        if dd.nd:
            Fop = lambda v: S.apply_F(v.real) + 1j * S.apply_F(v.imag)
            Pop = lambda v: S.apply_P(v.real) + 1j * S.apply_P(v.imag)
            nu, its, hist = fgmres(Fop, Pop, rhs.astype(complex), tol=tol, restart=restart, maxit=maxit)
        else:
            nu, its, hist = np.zeros(0, complex), 0, [0.0]
        x1, x2 = self._ahat(bh[:dd.n1] - S.C1.T @ nu, bh[dd.n1:])
        phi0 = dd.B @ (dd.Z @ np.concatenate([x1, x2]))
        return g_N + phi0, its, hist
