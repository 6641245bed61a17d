"""Flexible GMRES (right preconditioned, restarted, classical Gram-Schmidt applied twice).

The paper uses left-preconditioned PGMRES (Sec. 2.3.4); this implementation uses the
flexible, right-preconditioned variant so that the stopping test measures the true residual
||b - A x|| / ||b|| (zero initial guess, as in Sec. 3).  Complex Givens rotations
G = [[c, s], [-conj(s), c]] with real c.

Pins (tests/test_oracle_dd.py): on random well-conditioned complex systems the iterate
matches numpy.linalg.solve, the residual estimate after every iteration equals the true
residual of the iterate formed there, a preconditioner that changes from one application to
the next still converges to the same solution, and with the identity preconditioner the
residual history is monotone.
"""
from __future__ import annotations

import numpy as np


def givens(a: complex, b: complex):
    if b == 0:
        return 1.0, 0.0
    if a == 0:
        return 0.0, 1.0
    den = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / den
    s = (a / abs(a)) * np.conj(b) / den
    return c, s


def fgmres(apply_A, apply_M, b: np.ndarray, tol: float = 1e-10, restart: int = 100,
           maxit: int = 300):
    """Solve A x = b.  Returns (x, iterations, history of relative residual estimates)."""
    n = b.shape[0]
    x = np.zeros(n, dtype=complex)
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    r = b.astype(complex).copy()
    it = 0
    while True:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, n), dtype=complex)
        Zs = np.zeros((m, n), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        done = False
        for j in range(m):
            Zs[j] = apply_M(V[j])
            w = apply_A(Zs[j])
            h = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            H[: j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                t1 = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j], H[i + 1, j] = t0, t1
            c, s = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = c * H[j, j] + s * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j], g[j + 1] = c * g[j], -np.conj(s) * g[j]
            it += 1
            rel = abs(g[j + 1]) / bnorm
            hist.append(rel)
            j_end = j + 1
            if rel <= tol or it >= maxit:
                done = True
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + Zs[:j_end].T @ y
        if done:
            return x, it, hist
        r = b - apply_A(x)
