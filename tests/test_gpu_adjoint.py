"""GPU differentiation against the oracle: point evaluation / injection, the adjoint
permittivity gradient (per-element accumulation kernel), dJ/dk, autograd, and finite
differences at the 48x48 lens size."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import adjoint as adj  # noqa: E402
from oracle import dd  # noqa: E402
from paper_1808_04713_gb300 import ddh  # noqa: E402
from paper_1808_04713_gb300.autograd import PlaneWaveSolve, PointEval, make_solver  # noqa: E402


def _small_lens():
    w = W.small_uniform(3, 7, 9.0, seed=5, eps_range=(1.0, 4.0))
    w.thetas = np.array([0.0])
    return w


PTS = np.stack([np.full(6, 0.9), np.linspace(0.4, 0.6, 6)], axis=1)


def test_point_evaluation_and_injection():
    w = _small_lens()
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    s.factor(tol=1e-12)
    prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k, w.thetas)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((2, s.n_local)) + 1j * rng.standard_normal((2, s.n_local))
    pts = np.array([[0.13, 0.77], [0.5, 0.25], [0.91, 0.05], [1.0, 1.0], [0.0, 0.3]])
    y = s.eval_points(pts, torch.tensor(phi, device="cuda")).cpu().numpy()
    for r in range(2):
        assert np.allclose(y[r], dd.field_at(prob, phi[r], pts[:, 0], pts[:, 1]), atol=1e-12)
    wts = rng.standard_normal((1, 5)) + 1j * rng.standard_normal((1, 5))
    e = s.inject_points(pts, torch.tensor(wts, device="cuda")).cpu().numpy()[0]
    assert np.allclose(e, adj.point_functionals(prob, pts, wts[0]), atol=1e-12)
    s.close()


def _oracle_fd_k(w, step=1e-6):
    """Central difference in k of the oracle's objective (direct FP64 solves; the load's own
    k dependence included)."""
    Js = []
    for sgn in (1, -1):
        prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k + sgn * step, w.thetas)
        phi = adj.solve_load(prob, prob.b_N)[0]
        Js.append(adj.objective(prob, phi, PTS)[0])
    return (Js[0] - Js[1]) / (2 * step)


def test_adjoint_gradient_matches_oracle_and_autograd():
    w = _small_lens()
    prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k, w.thetas)
    J0, g0, _ = adj.gradient_eps(prob, PTS)
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    eps = torch.tensor(w.eps, dtype=torch.float64, requires_grad=True)
    k = torch.tensor(w.k, dtype=torch.float64, requires_grad=True)
    u = PlaneWaveSolve.apply(eps, k, s, w.thetas, 1e-12, None)
    y = PointEval.apply(u, s, PTS)
    J = (y.abs() ** 2).sum()
    J.backward()
    g = eps.grad.numpy()
    assert abs(J.item() - J0) <= 1e-9 * J0
    assert np.linalg.norm(g - g0) <= 1e-8 * np.linalg.norm(g0)
    # dJ/dk through autograd against the oracle's central difference in k
    fd = _oracle_fd_k(w)
    assert abs(k.grad.item() - fd) <= 1e-6 * abs(fd), (k.grad.item(), fd)
    s.close()


def test_autograd_raises_when_a_solve_misses_its_tolerance():
    w = _small_lens()
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    eps = torch.tensor(w.eps, dtype=torch.float64, requires_grad=True)
    with pytest.raises(ddh.DDHError) as ei:
        PlaneWaveSolve.apply(eps, w.k, s, w.thetas, 1e-14, {"maxit": 2})
    assert ei.value.status == ddh.ERR_NO_CONVERGENCE
    # an explicit opt-out returns the best iterate instead
    u = PlaneWaveSolve.apply(eps, w.k, s, w.thetas, 1e-14, {"maxit": 2}, True)
    assert torch.isfinite(u.abs()).all()
    s.close()


def test_grad_k_matches_finite_differences():
    w = _small_lens()
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    s.factor(tol=1e-12)
    b = s.rhs_planewave(w.thetas)
    u, _ = s.solve(b, tol=1e-12)
    y = s.eval_points(PTS, u)
    G = 2.0 * y
    lam, _ = s.solve(s.inject_points(PTS, torch.conj(G).resolve_conj()), tol=1e-12)
    gk = s.grad_k(u, lam, w.thetas)
    s.close()
    fd = _oracle_fd_k(w)
    assert abs(gk - fd) <= 1e-6 * abs(fd)


def test_lens_48_gradient_against_finite_differences():
    """48x48 squares, p = 16, k = 200, eps ~ U[1,4], theta = 0, J over 32 points on x = 0.9:
    the adjoint gradient (FP64 forward and adjoint solves to the workload's relative residual
    1e-10) against central differences of FP64 solves on all 16 seeded parameters.

    The FD's own accuracy sets the bounds.  J changes by g h between the two solves and each
    J carries about 1e-11 relative solve error, so step 1e-6 resolves g to about 1e-5 relative
    (bound 1e-4 relative, or 1e-6 of the largest entry), while step 2e-4 resolves it to 1e-7
    (bound 1e-6 relative where |g| is at least 1e-2 of the largest entry, 1e-7 of the largest
    entry absolute everywhere)."""
    w = W.lens_48()
    tol = 1e-10
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    eps = torch.tensor(w.eps, dtype=torch.float64, requires_grad=True)
    u = PlaneWaveSolve.apply(eps, w.k, s, w.thetas, tol, None)
    y = PointEval.apply(u, s, w.points)
    J = (y.abs() ** 2).sum()
    J.backward()
    g = eps.grad.numpy()
    assert len(w.fd_index) == 16

    def J_at(ep):
        s.set_coefficients(w.k, ep)
        s.factor(tol=tol)
        uu, _ = s.solve(s.rhs_planewave(w.thetas), tol=tol)
        return float((s.eval_points(w.points, uu).abs() ** 2).sum())

    gmax = float(np.abs(g).max())
    rows = []
    for e in w.fd_index:
        fd = {}
        for h in (1e-6, 2e-4):
            ep, em = np.array(w.eps).copy(), np.array(w.eps).copy()
            ep[e] += h
            em[e] -= h
            fd[h] = (J_at(ep) - J_at(em)) / (2 * h)
        rows.append((int(e), float(g[e]), fd[1e-6], fd[2e-4]))
    s.close()
    print("lens_48 gradient (element, adjoint, FD step 1e-6, FD step 2e-4):", rows)
    for e, ge, f6, f4 in rows:
        assert abs(ge - f6) <= 1e-4 * max(abs(f6), 1e-2 * gmax), (e, ge, f6)
        assert abs(ge - f4) <= 1e-7 * gmax, (e, ge, f4)
        if abs(ge) >= 1e-2 * gmax:
            assert abs(ge - f4) <= 1e-6 * abs(f4), (e, ge, f4)
