"""Full-size workloads (random_eps_64: 1.64 M DoF, 8 RHS; lens_48: 0.59 M DoF) checked by
properties the oracle computes one sampled unknown at a time.

The oracle cannot solve these meshes in seconds, so instead:
- the conforming residual r_c = Z_c^T (b - A phi) is evaluated at sampled interior vertex and
  edge-bubble unknowns from the oracle's own element matrices (Table 1 Kronecker products)
  applied to the GPU solution, and ||b_c|| from the oracle's impedance loads.  Every entry
  must satisfy |r_c[q]| <= ||r_c|| <= 1e-10 ||b_c||, which also checks the library's yardstick;
- the traces of the two elements of sampled interior edges agree (continuity of the
  conforming solution, eq. final_constraint with all moments).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dd, element as el, legendre as lg  # noqa: E402
from oracle.mesh import side_slot  # noqa: E402
from paper_1808_04713_gb300 import ddh  # noqa: E402


def _uniform_index(n):
    return lambda i, j: i + n * j          # workloads.uniform_leaves order


def _residual_tilde(w, e, phi_e, cache):
    """(B x B)(A_e phi_e) for an interior element (no Robin sides)."""
    n = w.base_n
    h = 1.0 / n
    p = int(w.p[e])
    if e not in cache:
        A = el.element_matrix_N(p, -w.k * w.k * w.eps[e] * (0.5 * h) ** 2, {})
        B = lg.B_matrix(p)
        cache[e] = np.kron(B, B) @ A
    return cache[e] @ phi_e


def _vertex_residual(w, idx, phi, i, j, cache):
    """r_c at the interior grid vertex (i h, j h): the corner entries of the four elements."""
    total = 0
    for (ei, ej, a, b2) in ((i, j, 1, 1), (i - 1, j, 0, 1), (i, j - 1, 1, 0), (i - 1, j - 1, 0, 0)):
        e = idx(ei, ej)
        N = int(w.p[e]) + 1
        total = total + _residual_tilde(w, e, phi(e), cache)[a + N * b2]
    return total


def _boundary_load_norm(w, r):
    """||b_c|| of the assembled impedance load for right-hand side r (oracle quadrature)."""
    n = w.base_n
    h = 1.0 / n
    idx = _uniform_index(n)
    acc = {}
    th = float(w.thetas[r])
    for j in range(n):
        for i in range(n):
            sides = [s for s, cond in ((1, i == 0), (2, i == n - 1), (3, j == 0), (4, j == n - 1)) if cond]
            if not sides:
                continue
            e = idx(i, j)
            p = int(w.p[e])
            x0, y0 = i * h, j * h
            bN = np.zeros((p + 1) ** 2, complex)
            for side in sides:
                g = dd.impedance_data(w.k, th, side)
                if side == 1:
                    q = lambda t: g(0.0 * t + x0, y0 + 0.5 * h * (1 + t))
                elif side == 2:
                    q = lambda t: g(0.0 * t + x0 + h, y0 + 0.5 * h * (1 + t))
                elif side == 3:
                    q = lambda t: g(x0 + 0.5 * h * (1 + t), 0.0 * t + y0)
                else:
                    q = lambda t: g(x0 + 0.5 * h * (1 + t), 0.0 * t + y0 + h)
                bN += el.robin_load_N(p, side, q, 0.5 * h)
            B = lg.B_matrix(p)
            bt = np.kron(B, B) @ bN
            N = p + 1
            # corners by grid point, edge bubbles by (edge, m)
            for (a, b2), (gx, gy) in (((1, 1), (i, j)), ((0, 1), (i + 1, j)), ((1, 0), (i, j + 1)), ((0, 0), (i + 1, j + 1))):
                acc[("v", gx, gy)] = acc.get(("v", gx, gy), 0) + bt[a + N * b2]
            for side in sides:
                for m in range(2, p + 1):
                    acc[("e", i, j, side, m)] = bt[side_slot(p, side, m)]
    return float(np.sqrt(sum(abs(v) ** 2 for v in acc.values())))


@pytest.mark.parametrize("name,prec", [("random_eps_64", ddh.PREC_FP64), ("random_eps_64", ddh.PREC_MIXED_FP32),
                                       ("lens_48", ddh.PREC_FP64)])
def test_full_size_sampled_conforming_residual(name, prec):
    w = W.WORKLOADS[name]()
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(tol=1e-10, precision=prec)
    b = s.rhs_planewave(w.thetas)
    u, st = s.solve(b, tol=1e-10)
    off = s.elem_offsets()
    uh = u.cpu().numpy()
    s.close()
    n = w.base_n
    idx = _uniform_index(n)
    rng = np.random.default_rng(2024)
    verts = [(int(a), int(c)) for a, c in rng.integers(1, n, size=(12, 2))]
    vedges = [(int(a), int(c)) for a, c in zip(rng.integers(1, n, 8), rng.integers(0, n, 8))]   # x = a h, cell row c
    cache = {}
    R = uh.shape[0]
    for r in range(R):
        assert st[r].primal_residual <= 1e-10
        bnorm = _boundary_load_norm(w, r)
        phi = lambda e: uh[r, off[e]:off[e + 1]]
        worst = 0.0
        for (i, j) in verts:
            worst = max(worst, abs(_vertex_residual(w, idx, phi, i, j, cache)))
        for (i, j) in vedges:
            eL, eR = idx(i - 1, j), idx(i, j)
            pL, pR = int(w.p[eL]), int(w.p[eR])
            rl = _residual_tilde(w, eL, phi(eL), cache)
            rr = _residual_tilde(w, eR, phi(eR), cache)
            for m in range(2, min(pL, pR) + 1):
                worst = max(worst, abs(rl[side_slot(pL, 2, m)] + rr[side_slot(pR, 1, m)]))
            # continuity of the traces along the edge
            t = np.array([-0.7, 0.1, 0.9])
            uL = el.evaluate_N(int(w.p[eL]), phi(eL), np.ones_like(t), t)
            uR = el.evaluate_N(int(w.p[eR]), phi(eR), -np.ones_like(t), t)
            assert np.max(np.abs(uL - uR)) <= 1e-8 * max(1.0, np.max(np.abs(uL)))
        assert worst <= 1.5e-10 * bnorm, (name, r, worst / bnorm)
