"""Pins of the oracle's Robin-modified local problems (Sec. 2.3.4) against what the paper and
the mathematics fix.

* The weak 2-colouring gives every element that has a neighbour a neighbour of the opposite
  sign.
* The added Robin terms cancel in the assembled conforming system, so the primal solution is
  unchanged: the paper states that only the A block changes and the primal solution does not.
* The dual-primal solve with the modified local problems equals the direct solve of the
  unmodified conforming system.
* At the element resonant wavenumber the paper prints (h = 0.25, p = 32, l = 3) the unmodified
  local block A11 of an interior element is singular, the modified one is not.
"""
import warnings

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from tests.golden_values import golden
from oracle import dd
from oracle.constraints import classify
from oracle.mesh import element_neighbours, weak_two_colouring

MESHES = {
    "uniform3_eps": lambda: W.small_uniform(3, 6, 8.0, seed=2, eps_range=(1, 2)),
    "uniform4_mixed_p": lambda: W.small_uniform(4, 6, 9.0, seed=7, eps_range=(1, 2), p_range=(4, 9)),
    "hanging_2level": lambda: W.small_hanging(3, refine=[(1, 1)], levels=2, p=6, k=5.0),
    "multilevel": lambda: W.multilevel_hanging(p=5, k=3.0),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_colouring_gives_every_element_an_opposite_neighbour(name):
    w = MESHES[name]()
    prob = dd.problem_from_workload(w)
    sign = weak_two_colouring(prob.mesh)
    assert set(np.unique(sign)) <= {-1, 1}
    for e in range(prob.mesh.n_elem):
        nb = element_neighbours(prob.mesh, e)
        assert nb and any(sign[f] != sign[e] for f in nb), e


@pytest.mark.parametrize("name", list(MESHES))
def test_added_robin_terms_cancel_in_the_conforming_system(name):
    w = MESHES[name]()
    p0 = dd.problem_from_workload(w)
    p1 = dd.problem_from_workload(w, robin_modified=True)
    # some element matrices really changed (interior Robin terms) ...
    changed = sum(np.abs(a - b).max() > 1e-12 for a, b in zip(p0.A_N, p1.A_N))
    assert changed >= 2
    # ... but the assembled conforming system and the loads did not
    Z = classify(p0.mesh, None).Z
    A0 = sp.block_diag(dd.tilde_blocks(p0, p0.A_N), format="csr")
    A1 = sp.block_diag(dd.tilde_blocks(p1, p1.A_N), format="csr")
    Ac0 = (Z.T @ A0 @ Z).toarray()
    Ac1 = (Z.T @ A1 @ Z).toarray()
    assert np.abs(Ac1 - Ac0).max() <= 1e-13 * np.abs(Ac0).max()
    assert np.array_equal(p0.b_N, p1.b_N)


@pytest.mark.parametrize("name", list(MESHES))
def test_robin_modified_dd_equals_unmodified_direct_solve(name):
    w = MESHES[name]()
    ref = dd.Conforming(dd.problem_from_workload(w)).solve_direct()
    p1 = dd.problem_from_workload(w, robin_modified=True)
    r = dd.DDSolver(p1).solve(tol=1e-12)
    assert np.linalg.norm(r["phi_N"] - ref) <= 1e-10 * np.linalg.norm(ref)


def _interior_block_cond(prob, l, e):
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        s = dd.DDSolver(prob, l=l)
    t = s.split.t1_offset
    blk = s.A11[t[e]:t[e + 1], t[e]:t[e + 1]].toarray()
    sv = np.linalg.svd(blk, compute_uv=False)
    return sv[-1] / sv[0]


def test_robin_modification_removes_the_element_resonance():
    """4 x 4 squares of [0,1]^2 (h = 0.25), p = 32, l = 3, at the paper's resonant wavenumber:
    the unmodified A11 block of interior element (1, 1) is singular to rounding, the modified
    block is well conditioned."""
    k = golden("resonant_k_p32_l3_h0.25")
    w = W.small_uniform(4, 32, k)
    e = 1 + 4 * 1
    r0 = _interior_block_cond(dd.problem_from_workload(w), 3, e)
    r1 = _interior_block_cond(dd.problem_from_workload(w, robin_modified=True), 3, e)
    assert r0 < 1e-11, r0
    assert r1 > 1e-6, r1
