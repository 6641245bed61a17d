"""Pins of the oracle's hanging-node geometry against what the mathematics fixes.

Every hanging-mesh parity result rests on the sub-edge affine parameters (a, b) of
eq. affine_parameters (Sec. 2.2.4) and on the slaving basis built from them.  Two checks
that use neither (a, b) nor the re-expansion matrices L:

* the conforming Galerkin solution on a hanging mesh converges spectrally in p to the
  exact plane wave (the plane wave solves the impedance problem exactly, Sec. 2.2.4 /
  Sec. 3 discretisation; measured with ``field_at``, i.e. each element's own polynomial);
* the field is continuous across every hanging edge: at points of a fine side, the coarse
  element's polynomial and the fine element's polynomial, each evaluated from its own
  element geometry by ``evaluate_N``, agree to rounding.

A planted mistake (one sub-edge's offset b negated, which is the same as ordering the
children the wrong way along the coarse side) must fail both checks.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dd
from oracle import element as el
from oracle.constraints import element_offsets

MESHES = {
    "hanging_1level": lambda p: W.small_hanging(3, refine=[(1, 1)], levels=1, p=p, k=5.0),
    "hanging_2level": lambda p: W.small_hanging(3, refine=[(1, 1)], levels=2, p=p, k=5.0),
    "hanging_mixed_p": lambda p: W.small_hanging(3, refine=[(1, 1)], levels=2, p=p, k=5.0, seed=1,
                                                 p_range=(p - 1, p + 2)),
    "multilevel": lambda p: W.multilevel_hanging(p=p, k=5.0),
}


def _problem(w):
    return dd.build_problem(w.base_n, w.leaves, w.p, w.eps, w.k, w.thetas)


def _side_point(prob, e, side, t):
    """Physical point of edge coordinate t in [-1, 1] on side `side` of element e
    (sides: 1 left, 2 right, 3 bottom, 4 top; t runs with y on 1, 2 and with x on 3, 4)."""
    x0, y0, h = dd.element_geometry(prob.mesh, e)
    s = 0.5 * h * (1 + t)
    if side == 1:
        return np.full_like(t, x0), y0 + s
    if side == 2:
        return np.full_like(t, x0 + h), y0 + s
    if side == 3:
        return x0 + s, np.full_like(t, y0)
    return x0 + s, np.full_like(t, y0 + h)


def _eval_on_element(prob, phi_N, e, x, y):
    """Element e's own polynomial at physical points (reference coordinates from its geometry)."""
    off = element_offsets(prob.mesh)
    x0, y0, h = dd.element_geometry(prob.mesh, e)
    pe = int(prob.mesh.p[e])
    return el.evaluate_N(pe, phi_N[off[e]:off[e + 1]], 2 * (x - x0) / h - 1, 2 * (y - y0) / h - 1)


def _hanging_trace_gap(prob, phi_N):
    """max over hanging edges, fine sides and sample points of |u_coarse - u_fine| / max|u|."""
    t = np.linspace(-1.0, 1.0, 9)
    gap, scale, n_fine = 0.0, 0.0, 0
    for ed in prob.mesh.edges:
        if ed.kind != "hanging":
            continue
        for (f, fs, _a, _b) in ed.others:
            x, y = _side_point(prob, f, fs, t)
            uf = _eval_on_element(prob, phi_N, f, x, y)
            uc = _eval_on_element(prob, phi_N, ed.elem, x, y)
            gap = max(gap, float(np.abs(uf - uc).max()))
            scale = max(scale, float(np.abs(uc).max()))
            n_fine += 1
    assert n_fine > 0
    return gap / scale


def _plane_wave_error(prob, phi_N, k, theta):
    rng = np.random.default_rng(11)
    x, y = rng.uniform(0, 1, 400), rng.uniform(0, 1, 400)
    ex = dd.plane_wave(k, theta)(x, y)
    return float(np.abs(dd.field_at(prob, phi_N, x, y) - ex).max())


@pytest.mark.parametrize("name", list(MESHES))
def test_plane_wave_spectral_convergence_on_hanging_meshes(name):
    errs = []
    for p in (5, 7, 9, 11):
        w = MESHES[name](p)
        prob = _problem(w)
        phi = dd.Conforming(prob).solve_direct()
        errs.append(_plane_wave_error(prob, phi[0], w.k, w.thetas[0]))
    # spectral decay: each step of 2 in p gains more than a factor 10, and p ~ 11 reaches 1e-7
    assert all(a / b > 10 for a, b in zip(errs[:-1], errs[1:])), errs
    assert errs[-1] < 1e-7, errs


@pytest.mark.parametrize("name", list(MESHES))
def test_field_is_continuous_across_hanging_edges(name):
    w = MESHES[name](7)
    prob = _problem(w)
    phi = dd.Conforming(prob).solve_direct()
    assert _hanging_trace_gap(prob, phi[0]) < 1e-12
    # the DD solution (dual-primal, the method itself) is continuous there too
    r = dd.DDSolver(prob).solve(tol=1e-13)
    assert _hanging_trace_gap(prob, r["phi_N"][0]) < 1e-10


def _negate_one_offset(prob):
    for ed in prob.mesh.edges:
        if ed.kind == "hanging":
            f, fs, a, b = ed.others[0]
            assert b != 0.0
            ed.others[0] = (f, fs, a, -b)
            return
    raise AssertionError("no hanging edge")


@pytest.mark.parametrize("name", ["hanging_1level", "multilevel"])
def test_pins_catch_a_negated_subedge_offset(name):
    """A planted mistake in the oracle's mesh bookkeeping fails both pins."""
    w = MESHES[name](9)
    prob = _problem(w)
    _negate_one_offset(prob)
    phi = dd.Conforming(prob).solve_direct()
    assert _hanging_trace_gap(prob, phi[0]) > 1e-3
    assert _plane_wave_error(prob, phi[0], w.k, w.thetas[0]) > 1e-3
