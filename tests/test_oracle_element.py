"""Pins of the oracle's element operator (Sec. 2.2.1) and discretisation."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dd, element as el, legendre as lg
from tests.golden_values import golden


def _basis_numpy(p, x):
    """N_k and N_k' built with numpy.polynomial.legendre (independent of S and D)."""
    vals = np.zeros((p + 1, x.size)); ders = np.zeros((p + 1, x.size))
    vals[0] = 1 / np.sqrt(2); vals[1] = x / np.sqrt(2); ders[1] = 1 / np.sqrt(2)
    for k in range(2, p + 1):
        ck = np.zeros(k); ck[k - 1] = np.sqrt((2 * (k - 1) + 1) / 2.0)
        vals[k] = np.polynomial.legendre.legval(x, np.polynomial.legendre.legint(ck, lbnd=-1))
        ders[k] = np.polynomial.legendre.legval(x, ck)
    return vals, ders


@pytest.mark.parametrize("p,h,beta,sides", [(5, 0.5, -30.0, (1, 3)), (7, 0.25, -120.0, (2, 4)),
                                            (4, 1.0, 3.0, ())])
def test_bilinear_form_brute_force(p, h, beta, sides):
    gam = -1j * 7.0
    t, w = lg.gauss_legendre(p + 6)
    V, Dv = _basis_numpy(p, t)
    n = p + 1
    A = np.zeros((n * n, n * n), complex)
    J = h / 2
    for a1 in range(n):
        for a2 in range(n):
            for b1 in range(n):
                for b2 in range(n):
                    i, j = a1 + n * a2, b1 + n * b2
                    gx = np.sum(w * Dv[a1] * Dv[b1]) * np.sum(w * V[a2] * V[b2])
                    gy = np.sum(w * V[a1] * V[b1]) * np.sum(w * Dv[a2] * Dv[b2])
                    mm = np.sum(w * V[a1] * V[b1]) * np.sum(w * V[a2] * V[b2])
                    A[i, j] = gx + gy + beta * J * J * mm
    Vp, _ = _basis_numpy(p, np.array([1.0, -1.0]))
    for s in sides:
        end = 0 if s in (2, 4) else 1
        for a1 in range(n):
            for a2 in range(n):
                for b1 in range(n):
                    for b2 in range(n):
                        if s in (1, 2):
                            val = Vp[a1, end] * Vp[b1, end] * np.sum(w * V[a2] * V[b2])
                        else:
                            val = Vp[a2, end] * Vp[b2, end] * np.sum(w * V[a1] * V[b1])
                        A[a1 + n * a2, b1 + n * b2] += gam * J * val
    mine = el.element_matrix_N(p, beta * J * J, {s: gam * J for s in sides})
    assert np.allclose(mine, A, atol=1e-12)


def test_element_resonance_golden():
    """The smallest resonant wavenumber of an interior element's A11 block (type-1 unknowns:
    interior bubbles and edge bubbles above l) for p = 32, l = 3, h = 0.25."""
    p, l, h = 32, 3, 0.25
    n = p + 1
    Kt = el.to_tilde(p, el.stiffness_matrix_N(p)).real
    Mt = el.to_tilde(p, el.mass_matrix_N(p)).real
    idx = [a + n * b for b in range(n) for a in range(n)
           if (a >= 2 and b >= 2) or (a < 2 and b > l) or (b < 2 and a > l)]
    lam = sla.eigh(Kt[np.ix_(idx, idx)], Mt[np.ix_(idx, idx)], eigvals_only=True)
    k0 = np.sqrt(lam[0]) / (h / 2)
    assert abs(k0 - golden("resonant_k_p32_l3_h0.25")) < 1e-9


def test_plane_wave_spectral_convergence():
    w = W.plane_2x2()
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, 300), rng.uniform(0, 1, 300)
    ex = dd.plane_wave(w.k, w.thetas[0])(x, y)
    errs = []
    for p in (6, 8, 10, 12):
        prob = dd.build_problem(2, w.leaves, np.full(4, p), w.eps, w.k, w.thetas)
        phi = dd.Conforming(prob).solve_direct()
        errs.append(np.abs(dd.field_at(prob, phi[0], x, y) - ex).max())
    assert all(a / b > 20 for a, b in zip(errs[:-1], errs[1:]))
    assert errs[-1] < 1e-8


def test_manufactured_solution_with_volume_load():
    """u = sin(3x) cos(2y) + i x y^2 with f = -lap u - k^2 u and g = du/dn - i k u."""
    k = 4.0
    u = lambda x, y: np.sin(3 * x) * np.cos(2 * y) + 1j * x * y * y
    lap = lambda x, y: -13 * np.sin(3 * x) * np.cos(2 * y) + 2j * x
    f = lambda x, y: -lap(x, y) - k * k * u(x, y)
    grad = lambda x, y: (3 * np.cos(3 * x) * np.cos(2 * y) + 1j * y * y,
                         -2 * np.sin(3 * x) * np.sin(2 * y) + 2j * x * y)
    w = W.small_uniform(2, 8, k)
    errs = []
    for p in (6, 9, 12):
        prob = dd.build_problem(2, w.leaves, np.full(4, p), np.ones(4), k, [0.0], f_list=[f])
        # replace the plane-wave boundary load by the manufactured impedance data
        from oracle.constraints import element_offsets
        off = element_offsets(prob.mesh)
        b = np.zeros_like(prob.b_N)
        for e in range(4):
            x0, y0, h = dd.element_geometry(prob.mesh, e)
            be = el.volume_load_N(p, f, x0, y0, h)
            for side in (1, 2, 3, 4):
                ei, _ = prob.mesh.side_edge[(e, side)]
                if prob.mesh.edges[ei].kind != 'boundary':
                    continue
                nrm = {1: (-1, 0), 2: (1, 0), 3: (0, -1), 4: (0, 1)}[side]
                def q(t, side=side, nrm=nrm, x0=x0, y0=y0, h=h):
                    if side in (1, 2):
                        X = x0 + (h if side == 2 else 0) + 0 * t; Y = y0 + h / 2 * (1 + t)
                    else:
                        X = x0 + h / 2 * (1 + t); Y = y0 + (h if side == 4 else 0) + 0 * t
                    gx, gy = grad(X, Y)
                    return nrm[0] * gx + nrm[1] * gy - 1j * k * u(X, Y)
                be += el.robin_load_N(p, side, q, h / 2)
            b[0, off[e]:off[e + 1]] = be
        prob.b_N = b
        phi = dd.Conforming(prob).solve_direct()
        rng = np.random.default_rng(2)
        x, y = rng.uniform(0, 1, 200), rng.uniform(0, 1, 200)
        errs.append(np.abs(dd.field_at(prob, phi[0], x, y) - u(x, y)).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9
