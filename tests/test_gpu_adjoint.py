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


def test_adjoint_gradient_matches_oracle_and_autograd():
    w = _small_lens()
    prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k, w.thetas)
    J0, g0, _ = adj.gradient_eps(prob, PTS)
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    eps = torch.tensor(w.eps, dtype=torch.float64, requires_grad=True)
    u = PlaneWaveSolve.apply(eps, s, w.thetas, 1e-13, None)
    y = PointEval.apply(u, s, PTS)
    J = (y.abs() ** 2).sum()
    J.backward()
    g = eps.grad.numpy()
    assert abs(J.item() - J0) <= 1e-9 * J0
    assert np.linalg.norm(g - g0) <= 1e-8 * np.linalg.norm(g0)
    s.close()


def test_grad_k_matches_finite_differences():
    w = _small_lens()
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    s.factor(tol=1e-13)
    b = s.rhs_planewave(w.thetas)
    u, _ = s.solve(b, tol=1e-13, allow_noconv=True)
    y = s.eval_points(PTS, u)
    G = 2.0 * y
    lam, _ = s.solve(s.inject_points(PTS, torch.conj(G).resolve_conj()), tol=1e-13, allow_noconv=True)
    gk = s.grad_k(u, lam, w.thetas)
    s.close()
    step = 1e-6
    Js = []
    for sgn in (1, -1):
        prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k + sgn * step, w.thetas)
        phi = adj.solve_load(prob, prob.b_N)[0]
        Js.append(adj.objective(prob, phi, PTS)[0])
    fd = (Js[0] - Js[1]) / (2 * step)
    assert abs(gk - fd) <= 1e-6 * abs(fd)


def test_lens_48_gradient_against_finite_differences():
    """48x48 squares, p = 16, k = 200, eps ~ U[1,4], theta = 0, J over 32 points on x = 0.9:
    adjoint gradient vs central differences (step 1e-6) on 4 of the seeded parameters."""
    w = W.lens_48()
    opts = dict(precision=ddh.PREC_MIXED_FP32, inner_iters=12)
    s = make_solver(0, w.base_n, w.leaves, w.p, w.k, w.eps)
    eps = torch.tensor(w.eps, dtype=torch.float64, requires_grad=True)
    u = PlaneWaveSolve.apply(eps, s, w.thetas, 1e-13, opts)
    y = PointEval.apply(u, s, w.points)
    J = (y.abs() ** 2).sum()
    J.backward()
    g = eps.grad.numpy()
    for e in w.fd_index[:4]:
        Js = []
        for sgn in (1, -1):
            ep = np.array(w.eps).copy()
            ep[e] += sgn * 1e-6
            s.set_coefficients(w.k, ep)
            s.factor(tol=1e-13, **opts)
            uu, _ = s.solve(s.rhs_planewave(w.thetas), tol=1e-13, allow_noconv=True)
            Js.append(float((s.eval_points(w.points, uu).abs() ** 2).sum()))
        fd = (Js[0] - Js[1]) / 2e-6
        assert abs(g[e] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), (e, g[e], fd)
    s.close()
