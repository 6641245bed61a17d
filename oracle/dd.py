"""Dual-primal domain decomposition of Section 2.3 (plain FP64, test infrastructure).

Saddle system [[A, C^T], [C, 0]] (eq. second_saddle_point_system) with block-diagonal A.
Partial nullspace method (eq. null_space_identity / assembled_saddle_point_system):
phi = Z phi_p, A^ = Z^T A Z, C^ = C_d Z, b^ = Z^T b (phi_z = 0, no Dirichlet data).
Dual Schur system C^ A^-1 C^T nu = C^ A^-1 b^ (eq. schur_complement_system), with A^-1
applied by block inversion (eq. block_matrix_inversion):
  y1 = A11^-1 r1,  t = r2 - A12^T y1,  x2 = K^-1 t,  x1 = y1 - A11^-1 A12 x2,
K = A22 - A12^T A11^-1 A12.  Local solves use a dense LU of each element block of A11
(plain; the fast-diagonalisation solver is pinned separately).  Recovery
A^ phi_p = b^ - C^T nu, phi = Z phi_p.

Preconditioner (eqs. general_preconditioner, weight_matrix; Sec. 2.3.3 choices):
P^-1 = D^-1 [C1 blockdiag(S_e^Lap) C1^T + C2 K^Lap C2^T] D^-1 with
D = C1_E C1_E^T + C2 C2^T (W1 Dirichlet, W2 = I on non-conforming meshes, the term
-C1 A11^-1 A12 W2 C2^T dropped), every operator in it built from the stiffness part only
(the -div(grad) term; mass and Robin terms dropped).

The Krylov method is FGMRES on the dual system with the true relative residual as the
stopping test.

Pins (tests/test_oracle_dd.py): the DD solution equals the direct globally assembled
solve; it is independent of l and of the preconditioner; C phi = 0; F is complex symmetric.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import element as el
from . import legendre as lg
from .constraints import Split, classify, dispersion_l, element_offsets, paper_constraints
from .fgmres import fgmres
from .mesh import Mesh, build_mesh, weak_two_colouring


# ------------------------------------------------------------------ problem definition

def plane_wave(k: float, theta: float):
    d = (np.cos(theta), np.sin(theta))
    return lambda x, y: np.exp(1j * k * (x * d[0] + y * d[1]))


def impedance_data(k: float, theta: float, side: int):
    """g = du/dn - i k u of the plane wave on the side of [0,1]^2 with the element side
    index (1: x=0, 2: x=1, 3: y=0, 4: y=1); returns g(x, y)."""
    u = plane_wave(k, theta)
    nd = {1: -np.cos(theta), 2: np.cos(theta), 3: -np.sin(theta), 4: np.sin(theta)}[side]
    return lambda x, y: (1j * k * nd - 1j * k) * u(x, y)


@dataclass
class Problem:
    mesh: Mesh
    k: float
    eps: np.ndarray
    A_N: list           # element matrices, N basis
    Alap_N: list        # stiffness parts, N basis
    b_N: np.ndarray     # [R, n_local] loads, N basis


def element_geometry(mesh: Mesh, e: int):
    lev, i, j = (int(v) for v in mesh.leaves[e])
    h = float(mesh.h[e])
    return i * h, j * h, h


def build_problem(base_n, leaves, p, eps, k, thetas, f_list=None, robin_modified=False) -> Problem:
    """Element matrices and loads for -lap u - k^2 eps u = f, du/dn - i k u = g(theta).

    robin_modified: the Robin-modified local problems of Sec. 2.3.4.  Elements get signs from
    the weak 2-colouring; an element of sign s adds the Robin term with gamma = s i k on each
    side it shares, across a conforming edge, with an element of the opposite sign (reading:
    no terms across hanging edges).  The two sides of such an edge add opposite terms, so the
    assembled conforming system, hence the primal solution, is unchanged; the loads are too."""
    mesh = build_mesh(base_n, leaves, p)
    sign = weak_two_colouring(mesh) if robin_modified else None
    eps = np.asarray(eps, float)
    thetas = np.atleast_1d(np.asarray(thetas, float))
    A_N, Alap_N = [], []
    off = element_offsets(mesh)
    R = len(thetas)
    b = np.zeros((R, int(off[-1])), complex)
    for e in range(mesh.n_elem):
        pe = int(mesh.p[e])
        x0, y0, h = element_geometry(mesh, e)
        beta_eff = -k * k * eps[e] * (0.5 * h) ** 2
        robin, loads = {}, []
        for side in (1, 2, 3, 4):
            ei, role = mesh.side_edge[(e, side)]
            ed = mesh.edges[ei]
            if ed.kind == 'boundary':
                robin[side] = -1j * k * 0.5 * h
                loads.append(side)
            elif sign is not None and ed.kind == 'conforming':
                nb = ed.others[0][0] if role == 'c' else ed.elem
                if sign[nb] != sign[e]:
                    robin[side] = sign[e] * 1j * k * 0.5 * h
        A_N.append(el.element_matrix_N(pe, beta_eff, robin))
        Alap_N.append(el.stiffness_matrix_N(pe))
        for r, th in enumerate(thetas):
            be = np.zeros((pe + 1) ** 2, complex)
            for side in loads:
                gfun = impedance_data(k, th, side)
                if side == 1:
                    q = lambda t, g=gfun: g(0.0 * t + x0, y0 + 0.5 * h * (1 + t))
                elif side == 2:
                    q = lambda t, g=gfun: g(0.0 * t + x0 + h, y0 + 0.5 * h * (1 + t))
                elif side == 3:
                    q = lambda t, g=gfun: g(x0 + 0.5 * h * (1 + t), 0.0 * t + y0)
                else:
                    q = lambda t, g=gfun: g(x0 + 0.5 * h * (1 + t), 0.0 * t + y0 + h)
                be += el.robin_load_N(pe, side, q, 0.5 * h)
            if f_list is not None:
                be += el.volume_load_N(pe, f_list[r], x0, y0, h)
            b[r, off[e]:off[e + 1]] = be
    return Problem(mesh, k, eps, A_N, Alap_N, b)


def problem_from_workload(w, thetas=None, robin_modified=False) -> Problem:
    return build_problem(w.base_n, w.leaves, w.p, w.eps, w.k,
                         w.thetas if thetas is None else thetas, robin_modified=robin_modified)


def tilde_blocks(prob: Problem, mats):
    return [el.to_tilde(int(prob.mesh.p[e]), mats[e]) for e in range(prob.mesh.n_elem)]


def to_tilde_vec(prob: Problem, v: np.ndarray) -> np.ndarray:
    """Element-wise (B (x) B) v (B is involutory, so the same map goes back)."""
    off = element_offsets(prob.mesh)
    out = np.empty_like(v)
    for e in range(prob.mesh.n_elem):
        pe = int(prob.mesh.p[e])
        out[..., off[e]:off[e + 1]] = (el.vec_to_tilde(pe, v[..., off[e]:off[e + 1]].T)).T
    return out


# ------------------------------------------------------------------ direct solve

def direct_solve(prob: Problem) -> np.ndarray:
    """Globally assembled conforming solve: Z_c = null(C) from an SVD of the paper's C,
    A_c = Z_c^T A Z_c, b_c = Z_c^T b, phi = Z_c A_c^-1 b_c.  Returns [R, n_local], N basis."""
    C, _ = paper_constraints(prob.mesh)
    Zc = sla.null_space(C.toarray(), rcond=1e-11)
    A = sp.block_diag(prob.A_N, format="csr")
    Ac = Zc.T @ (A @ Zc)
    bc = prob.b_N @ Zc
    u = np.linalg.solve(Ac, bc.T).T
    return u @ Zc.T


# ------------------------------------------------------------------ DD operator

class DDSolver:
    """Dual-primal operator pieces for a fixed split (primal-constraint count l)."""

    def __init__(self, prob: Problem, l: int | None = None, precond: str = "dirichlet"):
        self.prob = prob
        mesh = prob.mesh
        self.l = dispersion_l(mesh, prob.k, prob.eps) if l is None else l
        self.split: Split = classify(mesh, self.l)
        s = self.split
        self.precond = precond
        At = tilde_blocks(prob, prob.A_N)
        Alt = tilde_blocks(prob, prob.Alap_N)
        A = sp.block_diag(At, format="csr")
        Al = sp.block_diag(Alt, format="csr")
        Z = s.Z
        Ah = (Z.T @ A @ Z).tocsr()
        Ahl = (Z.T @ Al @ Z).tocsr()
        n1 = s.n1
        self.n1, self.n2 = n1, s.n2
        self.A12 = Ah[:n1, n1:].tocsr()
        self.A22 = Ah[n1:, n1:].tocsr()
        A11 = Ah[:n1, :n1].tocsr()
        self.A11 = A11
        self.Z = Z
        self.Ch = (s.Cd @ Z).tocsr()
        self.C1 = self.Ch[:, :n1].tocsr()
        self.C2 = self.Ch[:, n1:].tocsr()
        self.nd = self.Ch.shape[0]
        # element blocks of A11 (block diagonal by construction: checked)
        t1o = s.t1_offset
        self.lu11 = []
        blk_nnz = 0
        for e in range(mesh.n_elem):
            blk = A11[t1o[e]:t1o[e + 1], t1o[e]:t1o[e + 1]].toarray()
            blk_nnz += np.count_nonzero(blk)
            self.lu11.append(sla.lu_factor(blk))
        assert blk_nnz == A11.count_nonzero(), "A11 is not block diagonal"
        self.K = self._schur(self.A12, self.A22)
        self.Klu = spla.splu(self.K.tocsc()) if self.n2 else None
        # preconditioner pieces (stiffness part only)
        A11l = Ahl[:n1, :n1].tocsr()
        A12l = Ahl[:n1, n1:].tocsr()
        A22l = Ahl[n1:, n1:].tocsr()
        rows, cols, vals = [], [], []
        for e in range(mesh.n_elem):
            blk = A11l[t1o[e]:t1o[e + 1], t1o[e]:t1o[e + 1]].toarray()
            mE = s.t1_edge_mask[e]
            iE = np.nonzero(mE)[0]
            iI = np.nonzero(~mE)[0]
            Aee = blk[np.ix_(iE, iE)]
            Aei = blk[np.ix_(iE, iI)]
            Aii = blk[np.ix_(iI, iI)]
            Slap = Aee - Aei @ np.linalg.solve(Aii, Aei.T)
            gi = t1o[e] + iE
            rr, cc = np.meshgrid(gi, gi, indexing="ij")
            rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(Slap.ravel())
        if rows:
            Sbd = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(n1, n1))
        else:
            Sbd = sp.csr_matrix((n1, n1))
        self.Slap_bd = Sbd
        emask = np.zeros(n1, bool)
        for e in range(mesh.n_elem):
            emask[t1o[e]:t1o[e + 1]] = s.t1_edge_mask[e]
        C1E = self.C1[:, np.nonzero(emask)[0]]
        Dm = (C1E @ C1E.T + self.C2 @ self.C2.T).astype(complex).tocsc()
        self.Dlu = spla.splu(Dm) if self.nd else None
        self.mid = (self.C1 @ Sbd @ self.C1.T)
        if self.C2.count_nonzero() > 0:
            self.lu11_lap = []
            for e in range(mesh.n_elem):
                blk = A11l[t1o[e]:t1o[e + 1], t1o[e]:t1o[e + 1]].toarray()
                self.lu11_lap.append(sla.lu_factor(blk))
            Klap = self._schur(A12l, A22l, lus=self.lu11_lap)
            self.mid = self.mid + self.C2 @ Klap @ self.C2.T
        self.mid = self.mid.tocsr()

    # -- pieces
    def _schur(self, A12, A22, lus=None):
        """K = A22 - A12^T A11^-1 A12, accumulated element by element."""
        lus = self.lu11 if lus is None else lus
        t1o = self.split.t1_offset
        K = A22.tocoo()
        rows, cols, vals = [K.row], [K.col], [K.data.astype(complex)]
        for e in range(self.prob.mesh.n_elem):
            blk = A12[t1o[e]:t1o[e + 1], :].tocsc()
            nz = np.unique(blk.nonzero()[1])
            if nz.size == 0:
                continue
            Bd = blk[:, nz].toarray()
            X = sla.lu_solve(lus[e], Bd)
            contrib = -(Bd.T @ X)
            rr, cc = np.meshgrid(nz, nz, indexing="ij")
            rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(contrib.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=A22.shape)

    def A11_solve(self, r1: np.ndarray) -> np.ndarray:
        t1o = self.split.t1_offset
        out = np.empty_like(r1, dtype=complex)
        for e in range(self.prob.mesh.n_elem):
            out[t1o[e]:t1o[e + 1]] = sla.lu_solve(self.lu11[e], r1[t1o[e]:t1o[e + 1]])
        return out

    def Ahat_solve(self, r1, r2):
        y1 = self.A11_solve(r1)
        if self.n2 == 0:
            return y1, np.zeros(0, complex)
        t = r2 - self.A12.T @ y1
        x2 = self.Klu.solve(t)
        x1 = y1 - self.A11_solve(self.A12 @ x2)
        return x1, x2

    def apply_F(self, nu):
        x1, x2 = self.Ahat_solve(self.C1.T @ nu, self.C2.T @ nu)
        return self.C1 @ x1 + self.C2 @ x2

    def apply_P(self, v):
        if self.precond == "none":
            return v.copy()
        if self.precond == "lumped":
            return v.copy() if self.Dlu is None else self.Dlu.solve(v)
        w = self.Dlu.solve(v)
        return self.Dlu.solve(self.mid @ w)

    def bhat(self, b_tilde):
        bh = self.Z.T @ b_tilde
        return bh[: self.n1], bh[self.n1:]

    def rhs(self, b_tilde):
        x1, x2 = self.Ahat_solve(*self.bhat(b_tilde))
        return self.C1 @ x1 + self.C2 @ x2

    def recover(self, b_tilde, nu):
        b1, b2 = self.bhat(b_tilde)
        x1, x2 = self.Ahat_solve(b1 - self.C1.T @ nu, b2 - self.C2.T @ nu)
        return self.Z @ np.concatenate([x1, x2])

    def solve(self, tol=1e-10, restart=100, maxit=300):
        """Solve every RHS.  Returns dict with phi_N [R, n_local], iterations, histories."""
        prob = self.prob
        bt = to_tilde_vec(prob, prob.b_N)
        phis, its, hists, nus = [], [], [], []
        for r in range(bt.shape[0]):
            g = self.rhs(bt[r])
            if self.nd:
                nu, it, hist = fgmres(self.apply_F, self.apply_P, g, tol, restart, maxit)
            else:
                nu, it, hist = np.zeros(0, complex), 0, [0.0]
            phit = self.recover(bt[r], nu)
            phis.append(phit)
            its.append(it); hists.append(hist); nus.append(nu)
        phit = np.array(phis)
        return {"phi_N": to_tilde_vec(prob, phit), "phi_tilde": phit, "iterations": its,
                "history": hists, "nu": nus}


# ------------------------------------------------------------------ conforming yardstick

class Conforming:
    """The globally assembled basis (all constraints primal).  Primal residual yardstick:
    phi is projected onto the conforming space (u_c = argmin ||Z_c u - phi||, least squares),
    then r = ||Z_c^T (b - A Z_c u_c)|| / ||Z_c^T b|| on the interpolatory basis.  (For an
    iterate of the dual method Z_c^T (b - A phi) vanishes identically, whatever the dual
    variable, so phi itself cannot be used.)"""

    def __init__(self, prob: Problem):
        self.prob = prob
        self.split = classify(prob.mesh, None)
        self.Zc = self.split.Z
        self.A = sp.block_diag(tilde_blocks(prob, prob.A_N), format="csr")

    def residual(self, phi_N: np.ndarray, b_N: np.ndarray | None = None) -> np.ndarray:
        prob = self.prob
        b = prob.b_N if b_N is None else b_N
        bt = to_tilde_vec(prob, np.atleast_2d(b))
        pt = to_tilde_vec(prob, np.atleast_2d(phi_N))
        ZtZ = (self.Zc.T @ self.Zc).astype(complex).tocsc()
        uc = spla.splu(ZtZ).solve((pt @ self.Zc).T)
        pc = (self.Zc @ uc).T
        r = (bt - (self.A @ pc.T).T) @ self.Zc
        bc = bt @ self.Zc
        return np.linalg.norm(r, axis=1) / np.linalg.norm(bc, axis=1)

    def solve_direct(self) -> np.ndarray:
        """A_c u = b_c with the slaving basis (sparse LU); phi = Z_c u, N basis."""
        Ac = (self.Zc.T @ self.A @ self.Zc).tocsc()
        bt = to_tilde_vec(self.prob, self.prob.b_N)
        u = spla.splu(Ac).solve((bt @ self.Zc).T).T
        return to_tilde_vec(self.prob, (self.Zc @ u.T).T)


def field_at(prob: Problem, phi_N: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Evaluate the element-local field at physical points (leaf lookup by position)."""
    mesh = prob.mesh
    off = element_offsets(mesh)
    out = np.zeros(np.shape(x), complex)
    X = np.ravel(x); Y = np.ravel(y)
    res = np.zeros(X.shape, complex)
    for e in range(mesh.n_elem):
        x0, y0, h = element_geometry(mesh, e)
        inside = (X >= x0) & (X <= x0 + h) & (Y >= y0) & (Y <= y0 + h)
        todo = inside & (res == 0)
        if not np.any(todo):
            continue
        pe = int(mesh.p[e])
        u1 = 2 * (X[todo] - x0) / h - 1
        u2 = 2 * (Y[todo] - y0) / h - 1
        res[todo] = el.evaluate_N(pe, phi_N[off[e]:off[e + 1]], u1, u2)
    out[...] = res.reshape(np.shape(x))
    return out
