"""Pins of the oracle's Poisson test (Sec. 3.1) against the paper's Table 2.

For each listed case (degree p, N squares, l primal moments per edge; rho_ij = 10^((i-j)/4),
zero Dirichlet data, Dirichlet preconditioner with diagonal scaling):

* the largest eigenvalue of the preconditioned dual operator P^-1 F equals the printed value
  to its two decimals, and the smallest is 1 to two digits, as the paper states;
* PCG from zero with a random right-hand side (entries U(0,1)) reduces the residual by ten
  orders in the printed number of iterations (within one: the right-hand side is random).

A mistake in the Dirichlet treatment (which unknowns Algorithm 1 discards on a Dirichlet
side), the dual rows or the scaling changes these numbers; the planted check below drops the
diagonal scaling.
"""
import os

import numpy as np
import pytest

from oracle import poisson as P

_FIX = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2_poisson.txt")


def _rows():
    out = []
    for line in open(_FIX):
        s = line.split("#", 1)[0].split()
        if len(s) == 5:
            p, N, l, its = (int(v) for v in s[:4])
            out.append((p, N, l, its, float(s[4])))
    return out


ROWS = _rows()


@pytest.mark.parametrize("p,N,l,its,lmax", ROWS, ids=[f"p{r[0]}-N{r[1]}-l{r[2]}" for r in ROWS])
def test_table2_eigenvalues_and_iterations(p, N, l, its, lmax):
    n = int(round(np.log(N) / np.log(4)))
    s = P.Solver(P.build(n, p, l))
    lo, hi = s.eigs()
    assert abs(hi - lmax) <= 0.005 + 1e-9, (hi, lmax)
    assert abs(lo - 1.0) <= 0.005
    b = np.random.default_rng(7).uniform(0.0, 1.0, size=s.dd.B.shape[0])
    _, k = s.pcg(s.rhs(b))
    assert abs(k - its) <= 1, (k, its)


def test_constant_rho_removes_the_dependence_on_the_jumps():
    """With rho = 1 the diagonal scaling is a constant multiple on every interface row, and the
    spectrum stays bounded below by 1 (Sec. 2.3.3 Poisson paragraph)."""
    s = P.Solver(P.build(2, 4, 2, rho=np.ones(16)))
    lo, hi = s.eigs()
    assert abs(lo - 1.0) <= 1e-3 and 1.0 < hi < 2.0


def test_planted_mistakes_move_the_printed_values():
    """Planted in the oracle only: dropping the diagonal scaling of the Dirichlet preconditioner
    moves lambda_max of the p = 4, N = 16, l = 2 case away from the printed 1.26."""
    dd = P.build(2, 4, 2)
    s = P.Solver(dd)
    assert abs(s.eigs()[1] - 1.26) <= 0.005
    # no diagonal scaling: W blocks without diag(A_ee)^-1
    s2 = P.Solver(dd)
    C1 = s2.C1
    A11 = dd.A11.toarray()
    W = np.zeros((dd.n1, dd.n1))
    t = dd.t1_offset
    for e in range(len(t) - 1):
        idx = np.arange(t[e], t[e + 1])
        m = dd.t1_edge_mask[e]
        ie, ii = idx[m], idx[~m]
        W[np.ix_(ie, ie)] = np.eye(len(ie))
        W[np.ix_(ii, ie)] = -np.linalg.solve(A11[np.ix_(ii, ii)], A11[np.ix_(ie, ii)].T)
    s2.CWC = C1 @ W @ C1.T
    s2.mid = C1 @ W.T @ A11 @ W @ C1.T
    assert abs(s2.eigs()[1] - 1.26) > 0.05
