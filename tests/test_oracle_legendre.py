"""Pins of the oracle's one-dimensional algebra (Sec. 2.1) against textbook facts."""
import numpy as np
import pytest

from oracle import legendre as lg


def test_recurrence_matches_numpy_legendre():
    x = np.linspace(-1, 1, 37)
    P = lg.legendre_p(20, x)
    for k in range(21):
        ck = np.zeros(k + 1); ck[k] = 1.0
        ref = np.polynomial.legendre.legval(x, ck) * np.sqrt((2 * k + 1) / 2.0)
        assert np.allclose(P[k], ref, atol=1e-12)


def test_orthonormal():
    x, w = lg.gauss_legendre(40)
    P = lg.legendre_p(30, x)
    assert np.allclose((P * w) @ P.T, np.eye(31), atol=1e-13)


def test_derivative_matrix():
    n = 15
    x = np.linspace(-0.9, 0.9, 11)
    D = lg.D_matrix(n)
    dP = np.zeros((n + 1, x.size))
    for k in range(n + 1):
        ck = np.zeros(k + 1); ck[k] = np.sqrt((2 * k + 1) / 2.0)
        dP[k] = np.polynomial.legendre.legval(x, np.polynomial.legendre.legder(ck))
    assert np.allclose(D @ lg.legendre_p(n, x), dP, atol=1e-10)


def test_integrated_basis_is_antiderivative():
    n = 14
    x = np.linspace(-1, 1, 23)
    N = lg.N_basis(n, x)
    for k in range(2, n + 1):
        ck = np.zeros(k); ck[k - 1] = np.sqrt((2 * (k - 1) + 1) / 2.0)
        ref = np.polynomial.legendre.legval(x, np.polynomial.legendre.legint(ck, lbnd=-1))
        assert np.allclose(N[k], ref, atol=1e-12)
    assert np.allclose(N[0], 1 / np.sqrt(2)) and np.allclose(N[1], x / np.sqrt(2))


def test_boundary_values():
    n = 12
    e1 = np.zeros(n + 1); e1[0] = 1
    e2 = np.zeros(n + 1); e2[1] = 1
    assert np.allclose(lg.N_basis(n, 1.0), (e1 + e2) / np.sqrt(2), atol=1e-14)
    assert np.allclose(lg.N_basis(n, -1.0), (e1 - e2) / np.sqrt(2), atol=1e-14)


def test_jacobi_eigen_ode():
    n = 12
    x = np.linspace(-0.8, 0.8, 9)
    S = lg.S_matrix(n)
    D = lg.D_matrix(n)
    N2 = S @ D @ D @ lg.legendre_p(n, x)
    N = lg.N_basis(n, x)
    for k in range(2, n + 1):
        assert np.allclose(N2[k] * (1 - x) * (1 + x) + k * (k - 1) * N[k], 0, atol=1e-10)


def test_mass_and_stiffness_closed_forms():
    n = 10
    g = lg.g_vector(n)
    M = lg.mass_1d(n)
    K = lg.stiff_1d(n)
    assert np.allclose(K, np.diag([0] + [1] * n))
    for i in range(2, n + 1):            # 0-based i >= 2
        assert np.isclose(M[i, i], g[i] ** 2 + g[i - 1] ** 2)
        assert np.isclose(M[i, i - 2], -g[i - 1] * g[i - 2])
    assert np.allclose(M[np.abs(np.subtract.outer(range(n + 1), range(n + 1))) == 1], 0)
    x, w = lg.gauss_legendre(30)
    N = lg.N_basis(n, x)
    assert np.allclose((N * w) @ N.T, M, atol=1e-13)


def test_interpolatory_basis():
    n = 6
    B = lg.B_matrix(n)
    assert np.allclose(B @ B, np.eye(n + 1))
    x = np.linspace(-1, 1, 7)
    Nt = B @ lg.N_basis(n, x)
    assert np.allclose(Nt[0], (1 + x) / 2) and np.allclose(Nt[1], (1 - x) / 2)


@pytest.mark.parametrize("a,b", [(0.5, 0.5), (0.5, -0.5), (0.25, -0.75), (0.25, 0.25), (0.125, 0.375)])
def test_affine_re_expansion(a, b):
    n = 16
    L = lg.affine_L(n, a, b)
    x = np.linspace(-1, 1, 13)
    assert np.allclose(lg.legendre_p(n, a * x + b), L @ lg.legendre_p(n, x), atol=1e-11)
    assert np.allclose(np.diag(L), a ** np.arange(n + 1), atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0, atol=1e-13)
    Lt = lg.affine_L_tilde(n, a, b)
    Nt = lg.B_matrix(n) @ lg.N_basis(n, x)
    Nta = lg.B_matrix(n) @ lg.N_basis(n, a * x + b)
    assert np.allclose(Nta, Lt @ Nt, atol=1e-11)


def test_one_dimensional_dispersion_relation():
    """Condensed 1-D element on an infinite uniform grid: cos(k_h h) = -alpha/beta.
    The discrete dispersion error is O(1) below p = (kh + (kh)^(1/3) - 1)/2 and decays
    super-exponentially above it (Sec. 2.3.4)."""
    def err(p, kh):
        A = 2.0 * lg.stiff_1d(p) - kh * kh * 0.5 * lg.mass_1d(p)
        V, Bi = [0, 1], list(range(2, p + 1))
        S = A[np.ix_(V, V)] - A[np.ix_(V, Bi)] @ np.linalg.solve(A[np.ix_(Bi, Bi)], A[np.ix_(Bi, V)])
        Av = lg.Q_matrix() @ S @ lg.Q_matrix()
        return abs(-Av[0, 0] / Av[0, 1] - np.cos(kh))
    kh = 20.0
    thr = 0.5 * (kh + kh ** (1 / 3) - 1)
    below = [err(p, kh) for p in range(2, int(thr), 2)]
    above = [err(p, kh) for p in range(int(thr) + 2, 22, 2)]
    assert max(below) > 0.3
    assert all(a / b > 10 for a, b in zip(above[:-1], above[1:]))
    assert above[-1] < 1e-8


def test_dispersion_threshold_golden():
    from tests.golden_values import golden
    k, h = 10.75, 1.0
    assert abs(0.5 * (k * h + (k * h) ** (1 / 3) - 1) - golden("dispersion_threshold_k10.75_h1")) < 1e-4
