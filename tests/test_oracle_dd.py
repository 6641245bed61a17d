"""Pins of the oracle's constraints, nullspace basis and dual-primal solve (Sec. 2.2.4, 2.3)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dd
from oracle.constraints import B_z, classify, paper_constraints, split_rows
from oracle.fgmres import fgmres

MESHES = {
    "uniform3": lambda: W.small_uniform(3, 6, 8.0, seed=2, eps_range=(1, 2)),
    "uniform3_mixed_p": lambda: W.small_uniform(3, 6, 8.0, seed=2, eps_range=(1, 2), p_range=(4, 8)),
    "hanging_1level": lambda: W.small_hanging(3, refine=[(1, 1)], levels=1, p=6, k=5.0),
    "hanging_2level": lambda: W.small_hanging(3, refine=[(1, 1)], levels=2, p=6, k=5.0),
    "hanging_mixed_p": lambda: W.small_hanging(3, refine=[(1, 1)], levels=2, p=6, k=5.0, seed=1,
                                               p_range=(4, 8), eps_in=2.0),
    "multilevel": lambda: W.multilevel_hanging(p=5, k=3.0),
}


@pytest.fixture(scope="module", params=list(MESHES))
def case(request):
    w = MESHES[request.param]()
    prob = dd.problem_from_workload(w)
    return request.param, w, prob


def test_nullspace_basis_against_paper_constraints(case):
    name, w, prob = case
    C, tags = paper_constraints(prob.mesh)
    Bz = B_z(prob.mesh)
    for l in (1, 2, 3):
        s = classify(prob.mesh, l)
        isp, isd = split_rows(tags, prob.mesh, l)
        Cp = (C[isp] @ Bz).toarray()
        Z = s.Z.toarray()
        assert np.abs(Cp @ Z).max() < 1e-12
        assert np.linalg.matrix_rank(Z) == Z.shape[1]
        assert sla.null_space(Cp, rcond=1e-11).shape[1] == Z.shape[1]
        # dual rows: the paper's C_d rows scaled by 1/sqrt(2), on range(Z)
        Cdp = (C[isd] @ Bz @ s.Z).toarray() / np.sqrt(2)
        Cdm = (s.Cd @ s.Z).toarray()
        assert Cdp.shape == Cdm.shape and np.abs(Cdp - Cdm).max() < 1e-12
    # the conforming basis spans null(C)
    sc = classify(prob.mesh, None)
    Cf = (C @ Bz).toarray()
    assert np.abs(Cf @ sc.Z.toarray()).max() < 1e-12
    assert sla.null_space(Cf, rcond=1e-11).shape[1] == sc.Z.shape[1]


def test_dd_equals_direct_and_independent_of_l_and_preconditioner(case):
    name, w, prob = case
    ref = dd.Conforming(prob).solve_direct()
    for l, pc in ((1, "dirichlet"), (2, "dirichlet"), (3, "dirichlet"), (2, "lumped"), (2, "none")):
        res = dd.DDSolver(prob, l=l, precond=pc).solve(tol=1e-13)
        err = np.linalg.norm(res["phi_N"] - ref) / np.linalg.norm(ref)
        assert err < 1e-11, (l, pc, err)
    if name != "hanging_mixed_p":
        # the paper's literal constraints with an SVD null space agree as well; with mixed
        # degrees on hanging edges the decayed diagonal of L makes that route lose digits
        ref2 = dd.direct_solve(prob)
        assert np.linalg.norm(ref2 - ref) / np.linalg.norm(ref) < 1e-11
    else:
        ref2 = dd.direct_solve(prob)
        assert np.linalg.norm(ref2 - ref) / np.linalg.norm(ref) < 1e-7


def test_constraints_satisfied_and_primal_residual(case):
    name, w, prob = case
    res = dd.DDSolver(prob, l=2).solve(tol=1e-12)
    C, _ = paper_constraints(prob.mesh)
    assert np.abs(C @ res["phi_N"][0]).max() < 1e-10
    assert dd.Conforming(prob).residual(res["phi_N"])[0] < 1e-10


def test_dual_operator_complex_symmetric():
    prob = dd.problem_from_workload(MESHES["hanging_2level"]())
    s = dd.DDSolver(prob, l=2)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(s.nd) + 1j * rng.standard_normal(s.nd)
    y = rng.standard_normal(s.nd) + 1j * rng.standard_normal(s.nd)
    assert abs(y @ s.apply_F(x) - x @ s.apply_F(y)) < 1e-10 * abs(y @ s.apply_F(x))


def test_l_at_least_p_leaves_no_dual_problem():
    w = W.small_uniform(2, 4, 3.0)
    prob = dd.problem_from_workload(w)
    s = dd.DDSolver(prob, l=4)
    assert s.nd == 0
    res = s.solve()
    ref = dd.Conforming(prob).solve_direct()
    assert np.linalg.norm(res["phi_N"] - ref) / np.linalg.norm(ref) < 1e-12


def test_dispersion_rule_values():
    from oracle.constraints import dispersion_l
    from oracle.mesh import build_mesh
    got = []
    for f in (W.plane_2x2, W.plane_16x16, W.random_eps_64, W.lens_48):
        w = f()
        m = build_mesh(w.base_n, w.leaves[:1], w.p[:1])
        m.h = np.array([1.0 / w.base_n])
        got.append(dispersion_l(m, w.k, np.array([w.eps.max()])))
    assert got == [3, 4, 5, 5]


def test_fgmres_against_dense_solve():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, restart=15, maxit=200)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-11)
    assert all(a >= b - 1e-15 for a, b in zip(hist[:15], hist[1:16]))


def test_fgmres_residual_estimate_is_the_true_residual():
    # stopping after k iterations (no restart) forms x_k from the same least-squares problem
    # whose residual |g_{k+1}| the estimate reports, so the two agree to rounding
    rng = np.random.default_rng(5)
    n = 40
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    D = np.diag(1.0 / np.diag(A))
    for k in (1, 3, 7, 12):
        x, it, hist = fgmres(lambda v: A @ v, lambda v: D @ v, b, tol=0.0, restart=50, maxit=k)
        assert it == k
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert abs(hist[-1] - true) <= 1e-12 * max(1.0, true)


def test_fgmres_flexible_preconditioner():
    # a preconditioner that differs on every application (a few Jacobi sweeps, one more each
    # call): flexible GMRES keeps Z_j and still reaches the dense solution
    rng = np.random.default_rng(6)
    n = 50
    A = np.eye(n) * 5 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    d = np.diag(A)
    calls = [0]

    def prec(v):
        calls[0] += 1
        z = v / d
        for _ in range(calls[0] % 4):
            z = z + (v - A @ z) / d
        return z

    x, it, hist = fgmres(lambda v: A @ v, prec, b, tol=1e-12, restart=30, maxit=200)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-11
