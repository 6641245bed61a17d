"""Pins of the oracle's axis-aligned PML (Sec. 4, complex coordinate stretching).

* with layers the exact solution of the stretched problem is exp(-i k x~(x)) (x~ = x minus
  (i/k) times the integral of sigma_1); it is smooth per element and the field converges to it
  spectrally in p, with a layer along x1 and with layers along both axes (the corner elements
  carry both stretches; the coefficients of the two stiffness terms swapped would fail here);
* with zero data beyond the layer the field in the physical region is the unbounded plane
  wave up to a reflection that falls by orders of magnitude as sigma grows (no layer: the
  wave is fully reflected);
* with s = 1 the stretched element operators are the plain Helmholtz ones.
"""
import numpy as np
import pytest

from oracle import element as el
from oracle import pml
from oracle import poisson as P


def _field_error(phi, n, p, f, pts):
    m = 2 ** n
    h = 1.0 / m
    N2 = (p + 1) ** 2
    err = 0.0
    for x, y in pts:
        i, j = min(int(x / h), m - 1), min(int(y / h), m - 1)
        e = i + m * j
        v = el.evaluate_N(p, phi[e * N2:(e + 1) * N2], np.array([2 * (x - i * h) / h - 1]),
                          np.array([2 * (y - j * h) / h - 1]))[0]
        err = max(err, abs(v - f(x, y)))
    return err


@pytest.mark.parametrize("axes", [(0,), (0, 1)], ids=["x1_layer", "both_layers"])
def test_field_converges_to_the_stretched_plane_wave(axes):
    k, cells, sigma, n = 20.0, 1, 30.0, 2
    m = 2 ** n
    s1, s2 = pml.stretch(m, k, cells, sigma, axes=axes)
    f = pml.stretched_plane_wave(m, k, cells, sigma)
    pts = np.random.default_rng(1).uniform(0.0, 1.0, size=(40, 2))
    errs = []
    for p, l in ((6, 2), (9, 3), (12, 3)):
        S = pml.Solver(n, p, l, k, s1, s2)
        g = pml.lifting(n, p, f)
        phi, _ = S.solve(np.zeros_like(g), g, tol=1e-12)
        errs.append(_field_error(phi, n, p, f, pts))
    assert all(a / b > 20 for a, b in zip(errs[:-1], errs[1:])), errs
    assert errs[-1] < 1e-5, errs


def test_layer_absorbs_the_outgoing_wave():
    k, n, p, l = 20.0, 3, 10, 3
    m = 2 ** n
    pts = np.random.default_rng(2).uniform([0.0, 0.0], [1.0 - 2.0 / m, 1.0], size=(40, 2))
    errs = []
    for sigma in (0.0, 20.0, 40.0):
        s1, s2 = pml.stretch(m, k, 2, sigma)
        f = pml.stretched_plane_wave(m, k, 2, sigma)
        data = lambda x, y, f=f: np.where(np.asarray(x) > 1.0 - 1e-12, 0.0, f(x, y))
        S = pml.Solver(n, p, l, k, s1, s2)
        g = pml.lifting(n, p, data)
        phi, _ = S.solve(np.zeros_like(g), g, tol=1e-12)
        errs.append(_field_error(phi, n, p, f, pts))
    assert errs[0] > 0.5, errs
    assert errs[1] < 1e-3 and errs[2] < 1e-5 and errs[2] < 0.05 * errs[1], errs


def test_unit_stretch_is_the_helmholtz_operator():
    k, n, p, l = 15.0, 1, 7, 2
    m = 2 ** n
    s1, s2 = np.ones(m * m, complex), np.ones(m * m, complex)
    a = P.build(n, p, l, rho=np.ones(m * m), k=k, coef=pml.coefficients(m, k, s1, s2))
    b = P.build(n, p, l, rho=np.ones(m * m), k=k)
    for x, y in ((a.A11, b.A11), (a.A12, b.A12), (a.A22, b.A22)):
        assert abs(x - y).max() <= 1e-13 * abs(y).max()
