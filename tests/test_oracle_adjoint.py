"""Pin of the oracle's adjoint gradient: central finite differences of direct solves."""
import numpy as np

import workloads as W
from oracle import adjoint as adj
from oracle import dd


def _small_lens():
    w = W.small_uniform(3, 7, 9.0, seed=5, eps_range=(1.0, 4.0))
    w.thetas = np.array([0.0])
    return w


def test_adjoint_gradient_matches_finite_differences():
    w = _small_lens()
    pts = np.stack([np.full(6, 0.9), np.linspace(0.4, 0.6, 6)], axis=1)
    prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k, w.thetas)
    J, g, _ = adj.gradient_eps(prob, pts)
    idx = [0, 4, 8]
    fd = adj.fd_gradient(w, pts, idx, step=1e-6)
    assert np.allclose(g[idx], fd, rtol=1e-6, atol=1e-9 * np.abs(g).max())


def test_point_functional_is_transpose_of_evaluation():
    w = _small_lens()
    prob = dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k, w.thetas)
    pts = np.array([[0.13, 0.77], [0.5, 0.25], [0.91, 0.05]])
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(prob.b_N.shape[1]) + 1j * rng.standard_normal(prob.b_N.shape[1])
    wts = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    vals = dd.field_at(prob, phi, pts[:, 0], pts[:, 1])
    e = adj.point_functionals(prob, pts, wts)
    assert np.isclose(e @ phi, wts @ vals)
