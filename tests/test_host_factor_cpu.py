"""Host-only setup and factorisation of the native library (no GPU) against the oracle.

The library classifies slots, builds the dual rows and the coarse matrix K, and factors K
by nested dissection in its own C++ code. The oracle builds the same objects from
eq. final_constraint and Algorithm 1 with dense and sparse linear algebra. They share no
code, so equal sizes and the same l (eq. dispersion_criterion) check the host logic. The
library's self-checks are also bounded: one coarse solve K x = t with a seeded random t,
and S_E S_E^-1 = I for every element."""
import numpy as np
import pytest

import workloads as W
from oracle import dd


@pytest.fixture(scope="module")
def ddh():
    from paper_1808_04713_gb300 import build as b
    b.build()
    from paper_1808_04713_gb300 import ddh as m
    return m


CASES = {
    "plane_2x2": W.plane_2x2,
    "uniform3_eps": lambda: W.small_uniform(3, 8, 6.0, seed=1, eps_range=(1.0, 2.0)),
    "uniform4_mixed_p": lambda: W.small_uniform(4, 8, 5.0, seed=2, p_range=(5, 9)),
    "hanging4": lambda: W.small_hanging(4, refine=((1, 1),), levels=2, p=8, k=6.0),
    "hanging_mixed_p": lambda: W.small_hanging(3, refine=((0, 0), (2, 1)), levels=1, p=7, k=5.0,
                                               seed=3, p_range=(5, 9)),
    "multilevel": W.multilevel_hanging,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_factor_matches_oracle(ddh, name):
    w = CASES[name]()
    sizes, secs, l = ddh.host_factor(w.base_n, w.leaves, w.p, w.k, w.eps)
    S = dd.DDSolver(dd.problem_from_workload(w))
    assert l == S.l
    assert sizes["n_local"] == int(np.sum((np.asarray(w.p) + 1) ** 2))
    assert sizes["n_dual"] == S.nd
    assert sizes["n_coarse"] == S.n2
    assert sizes["n_e1"] + sizes["n_t"] > 0
    assert 0 < sizes["max_block"] <= sizes["n_coarse"]
    assert secs[2] <= 1e-12, secs          # ||K x - t|| / ||t|| of one coarse solve
    assert secs[3] <= 1e-10, secs          # max_e ||S_E S_E^-1 - I||_max
    assert secs[4] > 0                     # no interior block at resonance


@pytest.mark.parametrize("l", [2, 3, 5])
def test_host_factor_l_override(ddh, l):
    w = W.small_hanging(4, refine=((1, 1),), levels=1, p=8, k=6.0)
    sizes, secs, l_used = ddh.host_factor(w.base_n, w.leaves, w.p, w.k, w.eps, l_override=l)
    S = dd.DDSolver(dd.problem_from_workload(w), l=l)
    assert l_used == l
    assert (sizes["n_dual"], sizes["n_coarse"]) == (S.nd, S.n2)
    assert secs[2] <= 1e-12


@pytest.mark.parametrize("n,p,l", [(1, 3, 1), (1, 4, 3), (2, 3, 2), (2, 8, 2), (1, 16, 4)])
def test_host_factor_poisson_split_matches_oracle(ddh, n, p, l):
    """Poisson mode (k = 0, rho_ij = 10^((i - j)/4), zero Dirichlet data): the library's
    Dirichlet split (discarded boundary vertices and moments 2..l of boundary sides, single-sided
    dual rows above l) has the oracle's sizes, and its factor passes the self-checks."""
    from oracle import poisson as P
    m = 2 ** n
    leaves = P.uniform_leaves(m)
    rho = P.rho_table2(m)
    sizes, secs, l_used = ddh.host_factor(m, leaves, np.full(m * m, p), 0.0, rho, l_override=l)
    D = P.build(n, p, l)
    interior = m * m * (p - 1) ** 2
    assert l_used == l
    assert sizes["n_dual"] == D.nd
    assert sizes["n_coarse"] == D.n2
    assert sizes["n_e1"] + interior == D.n1
    # conforming unknowns: interior vertices, interior edge bubbles, element interiors
    assert sizes["n_conforming"] == (m - 1) ** 2 + 2 * m * (m - 1) * (p - 1) + interior
    assert secs[2] <= 1e-12, secs
    assert secs[3] <= 1e-10, secs


def test_dispersion_l_reproduces_the_bold_cells_of_table3(ddh):
    """The library's l from the dispersion criterion (eq. dispersion_criterion) is the smallest l
    the paper's Table 3 marks bold for every (N, k) it prints: bold exactly when l >= the
    library's choice.  The criterion reads kh only; the paper's kh = k * 2/sqrt(N) on (-1,1)^2 is
    set on a 2 x 2 mesh of the unit square (h = 1/2) by the wavenumber 2 kh."""
    import os
    fix = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table3_helmholtz.txt")
    rows = [tuple(int(v) for v in ln.split()) for ln in open(fix) if ln[:1].isdigit()]
    seen = {}
    for p, N, k, l, its, bold in rows:
        if (N, k) not in seen:
            kh = k * 2.0 / np.sqrt(N)
            _, _, l_lib = ddh.host_factor(2, W.uniform_leaves(2), np.full(4, 3), 2.0 * kh, np.ones(4))
            seen[(N, k)] = l_lib
        assert bool(bold) == (l >= seen[(N, k)]), (p, N, k, l, seen[(N, k)])


@pytest.mark.parametrize("n,p,l,kp", [(1, 8, 1, 11.0), (2, 8, 3, 21.0), (2, 12, 2, 31.0)])
def test_host_factor_dirichlet_helmholtz_split_matches_oracle(ddh, n, p, l, kp):
    """Helmholtz with Dirichlet data (k < 0 selects it here; Sec. 3.2): the library's split has the
    sizes of the oracle's, and its factor (indefinite A11 blocks) passes the self-checks."""
    from oracle import dirichlet as D
    m = 2 ** n
    k, _ = D.table3_problem(kp)
    sizes, secs, l_used = ddh.host_factor(m, W.uniform_leaves(m), np.full(m * m, p), -k, np.ones(m * m),
                                          l_override=l)
    ref = D.Solver(n, p, l, k)
    assert l_used == l
    assert (sizes["n_dual"], sizes["n_coarse"]) == (ref.dd.nd, ref.dd.n2)
    assert sizes["n_e1"] + m * m * (p - 1) ** 2 == ref.dd.n1
    assert secs[2] <= 1e-11, secs
    assert secs[3] <= 1e-10, secs
