"""The Poisson convergence test of Sec. 3.1 (Table 2): test infrastructure only, plain and slow.

-div(rho grad phi) = f on (-1,1)^2 with zero Dirichlet data on the whole boundary, split into
2^n x 2^n equal squares of degree p, rho piecewise constant with rho_ij = 10^((i - j)/4) on
element (i, j) (i along x1, j along x2, both from 1).  The dual-primal method of Sec. 2.3 with
zero Dirichlet constraints (Sec. 2.2.1: on a Dirichlet side the constraint rows pick every
trace coefficient; the paper's rows carry +-1 entries on the N-basis pair e1 +- e2, here unit
entries on the interpolatory-basis trace slots, the same rows up to a constant):

* Algorithm 1 with Dirichlet sides: the vertices on the boundary and the edge unknowns of
  moments 2..l on a Dirichlet side are discarded (constrained to zero with the primal rows);
  interface edges keep one coarse unknown per moment 2..min(l, d) and per interior vertex;
* the dual rows: moments l < m <= d of every interface edge (coarse side minus fine side) and
  of every Dirichlet side (the single side's trace slot, right-hand side d = 0);
* the Dirichlet preconditioner with diagonal scaling (Sec. 2.3.3):
  P^-1 = (C1 W1 C1^T)^-T C1 W1^T A11 W1 C1^T (C1 W1 C1^T)^-1 with per-element blocks
  W^(j) = [I 0; -(A_ii)^-1 A_ei^T 0] diag(diag(A_ee)^-1, I) over the edge (e) and interior (i)
  unknowns of A11 (W2 = 0; the mesh is conforming, so C2 = 0);
* PCG on F nu = g, F = C^ A^-1 C^T, with P^-1 (Sec. 2.3.3 Poisson paragraph), and the extreme
  eigenvalues of P^-1 F by a dense eigensolve (small cases);
* the recovered field phi = Z A^-1 (b^ - C^T nu) in the N basis;
* Lanczos estimates of the extreme eigenvalues from the PCG coefficients.

Parity pinned against the paper's Table 2 in tests/test_oracle_poisson.py, and the recovered
field against the exact solution sin(pi x) sin(pi y) of a manufactured problem (rho = 1) and
against the all-primal split (l = p, no dual rows) for piecewise rho.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import legendre as lg
from .element import mass_matrix_N, stiffness_matrix_N, to_tilde
from .mesh import build_mesh, side_corners, side_slot


def uniform_leaves(m: int) -> np.ndarray:
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    return np.stack([np.zeros(m * m, np.int64), ii.ravel(), jj.ravel()], axis=1)


def rho_table2(m: int) -> np.ndarray:
    """rho on element e = i + m j (0-based i, j): 10^((i - j)/4) (the 1-based indices differ by
    the same amount)."""
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    return (10.0 ** ((ii - jj) / 4.0)).ravel()


@dataclass
class PoissonDD:
    n1: int
    n2: int
    nd: int
    A11: sp.csr_matrix
    A12: sp.csr_matrix
    A22: sp.csr_matrix
    C1: sp.csr_matrix
    Z: sp.csr_matrix
    t1_offset: np.ndarray
    t1_edge_mask: list
    B: sp.csr_matrix          # block-diagonal B (x) B: phi~ = B phi (N -> interpolatory basis)
    A11_lap: sp.csr_matrix    # stiffness part of A11 (equal to A11 when k = 0)


def build(n: int, p: int, l: int, rho: np.ndarray | None = None, k: float = 0.0,
          coef: np.ndarray | None = None) -> PoissonDD:
    """The dual-primal pieces for 2^n x 2^n squares of degree p with l primal moments per edge.
    With k > 0 the element operators are those of the Helmholtz problem with the same zero
    Dirichlet constraints (alpha = I, beta = -k^2 on the unit square: S + c_e M, c_e = -k^2 (h/2)^2;
    Sec. 3.2); A11_lap then holds the stiffness part, which the Dirichlet preconditioner uses.
    coef [E, 3] (complex) replaces both: element e's operator is
    a_e K(x1) M(x2) + b_e M(x1) K(x2) + c_e M (x) M (diagonal alpha = diag(a_e, b_e) and
    beta_eff = c_e per element, as a coordinate-stretched PML gives, Sec. 4)."""
    m = 2 ** n
    E = m * m
    leaves = uniform_leaves(m)
    mesh = build_mesh(m, leaves, np.full(E, p))
    rho = rho_table2(m) if rho is None else np.asarray(rho, float)
    N = p + 1
    off = np.arange(E + 1, dtype=np.int64) * N * N
    Xmax = m                                          # vertex coordinates in element units
    on_boundary = lambda xy: xy[0] in (0, Xmax) or xy[1] in (0, Xmax)
    # ---- coarse unknowns: interior vertices, moments 2..min(l, d) of interface edges
    vcol = {}
    for xy in sorted(mesh.vertices):
        if not on_boundary(xy):
            vcol[xy] = len(vcol)
    ecol = {}
    nxt = len(vcol)
    for ei, ed in enumerate(mesh.edges):
        if ed.kind != 'conforming':
            continue
        for mm in range(2, min(l, ed.degree) + 1):
            ecol[(ei, mm)] = nxt
            nxt += 1
    n2 = nxt
    # ---- per element: type-1 slots (interior, then edge moments m > l side by side)
    zr, zc, zv = [], [], []
    t1_offset = np.zeros(E + 1, np.int64)
    t1_edge_mask = []
    n1 = 0
    t1_slot = {}
    coarse_rows = []
    for e in range(E):
        t1, mask = [], []
        for bb in range(2, N):
            for aa in range(2, N):
                t1.append(aa + N * bb); mask.append(False)
        for side in (1, 2, 3, 4):
            ei, _ = mesh.side_edge[(e, side)]
            ed = mesh.edges[ei]
            for mm in range(2, N):
                s = side_slot(p, side, mm)
                if mm > l:
                    t1.append(s); mask.append(True)
                elif ed.kind == 'conforming':
                    coarse_rows.append((off[e] + s, ecol[(ei, mm)]))
                # a Dirichlet side's moments 2..l: discarded (zero)
        for (aa, bb) in ((0, 0), (1, 0), (0, 1), (1, 1)):
            xy = mesh.corner_xy(e, aa, bb)
            if xy in vcol:
                coarse_rows.append((off[e] + aa + N * bb, vcol[xy]))
        for jj, s in enumerate(t1):
            zr.append(off[e] + s); zc.append(n1 + jj); zv.append(1.0)
            t1_slot[(e, s)] = n1 + jj
        t1_edge_mask.append(np.asarray(mask, bool))
        n1 += len(t1)
        t1_offset[e + 1] = n1
    for row, col in coarse_rows:
        zr.append(row); zc.append(n1 + col); zv.append(1.0)
    Z = sp.csr_matrix((zv, (zr, zc)), shape=(int(off[-1]), n1 + n2))
    # ---- dual rows on the type-1 unknowns (C2 = 0: no coarse unknown carries a dual moment)
    dr, dc, dv = [], [], []
    r = 0
    for ei, ed in enumerate(mesh.edges):
        for mm in range(l + 1, ed.degree + 1):
            dr.append(r); dc.append(t1_slot[(ed.elem, side_slot(p, ed.side, mm))]); dv.append(1.0)
            if ed.kind == 'conforming':
                f, fs, _, _ = ed.others[0]
                dr.append(r); dc.append(t1_slot[(f, side_slot(p, fs, mm))]); dv.append(-1.0)
            r += 1
    C1 = sp.csr_matrix((dv, (dr, dc)), shape=(r, n1))
    # ---- element operators rho_e (K (x) M + M (x) K) on the interpolatory basis
    S = to_tilde(p, stiffness_matrix_N(p))
    if coef is not None:
        M1 = lg.mass_1d(p)
        K1 = lg.stiff_1d(p)
        Sx = to_tilde(p, np.kron(M1, K1))     # K along x1 (index a, fastest), M along x2
        Sy = to_tilde(p, np.kron(K1, M1))
        Mt = to_tilde(p, mass_matrix_N(p))
        cf = np.asarray(coef, complex)
        A = sp.block_diag([cf[e, 0] * Sx + cf[e, 1] * Sy + cf[e, 2] * Mt for e in range(E)], format="csr")
    elif k > 0.0:
        c = -(k * 0.5 / m) ** 2
        Ae = S + c * to_tilde(p, mass_matrix_N(p))
        A = sp.block_diag([rho[e] * Ae for e in range(E)], format="csr")
    else:
        A = sp.block_diag([rho[e] * S for e in range(E)], format="csr")
    Ah = (Z.T @ A @ Z).tocsr()
    Bl = lg.B_matrix(p)
    B = sp.block_diag([np.kron(Bl, Bl)] * E, format="csr")
    Z1 = Z[:, :n1]
    A11_lap = (Z1.T @ sp.block_diag([rho[e] * S for e in range(E)], format="csr") @ Z1).tocsr()
    return PoissonDD(n1, n2, r, Ah[:n1, :n1].tocsr(), Ah[:n1, n1:].tocsr(), Ah[n1:, n1:].tocsr(), C1, Z,
                     t1_offset, t1_edge_mask, B, A11_lap)


class Solver:
    """F, the Dirichlet preconditioner and PCG for one PoissonDD.  scaled = True: the diagonally
    scaled Dirichlet preconditioner of the Poisson test (W^(j) with diag(A_ee)^-1, on A11);
    scaled = False: the unscaled Dirichlet preconditioner on the stiffness part of A11 (W^(j) =
    [I; -A_ii^-1 A_ei^T], Sec. 2.3.3), used for the Helmholtz problem."""

    def __init__(self, dd: PoissonDD, scaled: bool = True):
        self.dd = dd
        self.lu11 = spla.splu(dd.A11.tocsc())
        K = dd.A22 - dd.A12.T @ self.lu11.solve(dd.A12.toarray())
        self.K = np.asarray(K)
        self.Klu = sla.lu_factor(self.K) if dd.n2 else None
        # W1 element by element (edge unknowns e, interior unknowns i)
        n1 = dd.n1
        W = np.zeros((n1, n1))
        A11 = (dd.A11 if scaled else dd.A11_lap).toarray().real
        t = dd.t1_offset
        for e in range(len(t) - 1):
            idx = np.arange(t[e], t[e + 1])
            msk = dd.t1_edge_mask[e]
            ie, ii = idx[msk], idx[~msk]
            Aee = A11[np.ix_(ie, ie)]
            Aei = A11[np.ix_(ie, ii)]
            Aii = A11[np.ix_(ii, ii)]
            Dinv = np.diag(1.0 / np.diag(Aee)) if scaled else np.eye(len(ie))
            W[np.ix_(ie, ie)] = Dinv
            W[np.ix_(ii, ie)] = -np.linalg.solve(Aii, Aei.T) @ Dinv
        C1 = dd.C1.toarray()
        self.CWC = C1 @ W @ C1.T
        self.mid = C1 @ W.T @ A11 @ W @ C1.T
        self.C1 = C1

    def Ahat_solve(self, r1, r2):
        """[A11 A12; A12^T A22]^-1 [r1; r2] by block inversion (Sec. 2.3.3)."""
        dd = self.dd
        y1 = self.lu11.solve(r1)
        if dd.n2 == 0:
            return y1, np.zeros(0)
        x2 = sla.lu_solve(self.Klu, r2 - dd.A12.T @ y1)
        x1 = y1 - self.lu11.solve(dd.A12 @ x2)
        return x1, x2

    def apply_F(self, nu):
        x1, _ = self.Ahat_solve(self.C1.T @ nu, np.zeros(self.dd.n2))
        return self.C1 @ x1

    def F_dense(self):
        return np.column_stack([self.apply_F(c) for c in np.eye(self.dd.nd)])

    def apply_P(self, v):
        a = np.linalg.solve(self.CWC, v)
        return np.linalg.solve(self.CWC.T, self.mid @ a)

    def P_dense(self):
        return np.column_stack([self.apply_P(c) for c in np.eye(self.dd.nd)])

    def eigs(self):
        """Extreme eigenvalues of P^-1 F (real and positive for this SPD problem)."""
        ev = np.linalg.eigvals(self.P_dense() @ self.F_dense())
        ev = np.sort(ev.real)
        return float(ev[0]), float(ev[-1])

    def rhs(self, b_N):
        """g = C^ A^-1 b^ with b^ = Z^T B b (the load on the interpolatory basis, d = 0)."""
        bh = self.dd.Z.T @ (self.dd.B @ b_N)
        x1, _ = self.Ahat_solve(bh[:self.dd.n1], bh[self.dd.n1:])
        return self.C1 @ x1

    def solve(self, b_N, tol=1e-12):
        """phi (N basis, element-local) of the Poisson problem with load b_N: PCG on F nu = g,
        then the recovery A^ phi^ = b^ - C^T nu (Sec. 2.3.3) and phi = Z phi^ back in the N basis
        (B (x) B is involutory).  Returns (phi_N, iterations)."""
        dd = self.dd
        bh = dd.Z.T @ (dd.B @ b_N)
        if dd.nd:
            nu, its = self.pcg(self.rhs(b_N), tol=tol)
        else:
            nu, its = np.zeros(0), 0
        x1, x2 = self.Ahat_solve(bh[:dd.n1] - self.C1.T @ nu, bh[dd.n1:])
        return dd.B @ (dd.Z @ np.concatenate([x1, x2])), its

    def pcg(self, g, tol=1e-10, maxit=500, coeffs=None):
        """Preconditioned conjugate gradients on F nu = g from nu = 0; iterations until
        ||g - F nu|| <= tol ||g||.  With a list `coeffs`, appends (alpha_j, beta_j) of every
        iteration (beta of the last one is None)."""
        nu = np.zeros_like(g)
        r = g.copy()
        z = self.apply_P(r)
        d = z.copy()
        rz = r @ z
        g0 = np.linalg.norm(g)
        for it in range(1, maxit + 1):
            Fd = self.apply_F(d)
            a = rz / (d @ Fd)
            nu += a * d
            r -= a * Fd
            if np.linalg.norm(r) <= tol * g0:
                if coeffs is not None:
                    coeffs.append((a, None))
                return nu, it
            z = self.apply_P(r)
            rz_new = r @ z
            if coeffs is not None:
                coeffs.append((a, rz_new / rz))
            d = z + (rz_new / rz) * d
            rz = rz_new
        return nu, maxit


def lanczos_extremes(coeffs):
    """Extreme eigenvalues of the Lanczos matrix of k CG steps (the CG-Lanczos relation, e.g.
    Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.7.3): T_00 = 1/alpha_0,
    T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j-1} = sqrt(beta_{j-1})/alpha_{j-1}; its
    eigenvalues are Ritz values of P^-1 F (Sec. 3.1 reads lambda_max by Lanczos)."""
    k = len(coeffs)
    T = np.zeros((k, k))
    for j in range(k):
        a = coeffs[j][0]
        T[j, j] = 1.0 / a
        if j:
            ap, bp = coeffs[j - 1]
            T[j, j] += bp / ap
            T[j, j - 1] = T[j - 1, j] = np.sqrt(bp) / ap
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])
