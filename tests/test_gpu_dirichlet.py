"""GPU parity of the Helmholtz problem with Dirichlet data (Sec. 3.2, Table 3) against the oracle.

-lap phi - k^2 phi = 0 with phi = -(i/4) H0^(2)(k |x - x_c|) on the boundary of the unit square
(the paper's (-1,1)^2 with x_c = (-2, 1), mapped: k doubled, x_c = (-1/2, 1)).  Checked here:

* the device lifting of the data (boundary vertex values, L^2-projection bubbles of each
  boundary side, N basis) against the oracle's, relative 1e-10 (Bessel function rounding);
* one application of F and of the unscaled Dirichlet preconditioner P^-1 (single-sided rows of
  the boundary sides divided by 1, interface rows by 2) against the oracle, relative 1e-12;
* complete solves against the oracle's solution (plain FP64 relative 1e-9 with both sides to
  1e-12; the mixed form relative 1e-8) and against the exact point-source field;
* the printed Table 3 iteration counts (the paper's criterion: dual residual reduced by ten
  orders, option dual_stop) on 132 cells with p <= 32 (the library's limit; p = 8 all, p = 16
  with N <= 256, p = 32 with N = 16 and 1024), within two iterations or 6 % (FGMRES here,
  left-preconditioned PGMRES in the paper), at least 95 where the table prints a dash.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dirichlet as D  # noqa: E402
from oracle import poisson as P  # noqa: E402
from paper_1808_04713_gb300 import ddh  # noqa: E402

_FIX = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table3_helmholtz.txt")
SRC = np.array([[-0.5, 1.0]])


def _rows():
    out = []
    for line in open(_FIX):
        s = line.split("#", 1)[0].split()
        if len(s) == 6:
            out.append(tuple(int(v) for v in s))
    return out


def _solver(n, p, l, k, **opt):
    m = 2 ** n
    s = ddh.DDH(0)
    s.set_mesh(m, P.uniform_leaves(m), np.full(m * m, p))
    s.set_coefficients(k, np.ones(m * m))
    s.set_boundary(ddh.BOUNDARY_DIRICHLET)
    s.factor(l_override=l, **opt)
    return s


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,p,kp", [(1, 8, 11.0), (2, 12, 21.0), (1, 32, 31.0)])
def test_lifting_matches_oracle(n, p, kp):
    k, data = D.table3_problem(kp)
    s = _solver(n, p, 2, k)
    g = s.dirichlet_point_source(SRC).cpu().numpy()[0]
    ref = D.lifting(n, p, data)
    # CUDA's j0 / y0 and scipy's Hankel function agree to a few units in the last place; the
    # high-degree bubble moments are small differences of such values
    assert _rel(g, ref) <= 1e-10, _rel(g, ref)
    s.close()


@pytest.mark.parametrize("n,p,l,kp", [(1, 8, 3, 11.0), (2, 8, 2, 21.0), (2, 12, 4, 11.0)])
def test_operator_and_preconditioner_match_oracle(n, p, l, kp):
    k, _ = D.table3_problem(kp)
    s = _solver(n, p, l, k)
    ref = D.Solver(n, p, l, k)
    info = s.info()
    assert (info.n_dual, info.n_coarse) == (ref.dd.nd, ref.dd.n2)
    rng = np.random.default_rng(9)
    nu = rng.standard_normal((2, ref.dd.nd)) + 1j * rng.standard_normal((2, ref.dd.nd))
    v = torch.tensor(nu, device="cuda:0")
    Fv = s.apply_dual_operator(0, v, ddh.PREC_FP64).cpu().numpy()
    Pv = s.apply_dual_operator(1, v, ddh.PREC_FP64).cpu().numpy()
    for r in range(2):
        fo = ref.S.apply_F(nu[r].real) + 1j * ref.S.apply_F(nu[r].imag)
        po = ref.S.apply_P(nu[r].real) + 1j * ref.S.apply_P(nu[r].imag)
        assert _rel(Fv[r], fo) <= 1e-12, ("F", _rel(Fv[r], fo))
        assert _rel(Pv[r], po) <= 1e-12, ("P", _rel(Pv[r], po))
    s.close()


@pytest.mark.parametrize("n,p,l,kp,prec", [(1, 12, 4, 11.0, ddh.PREC_FP64), (2, 10, 3, 21.0, ddh.PREC_FP64),
                                           (2, 10, 3, 21.0, ddh.PREC_MIXED_FP32)],
                         ids=["fp64_2x2", "fp64_4x4", "mixed_4x4"])
def test_solution_matches_oracle(n, p, l, kp, prec):
    k, data = D.table3_problem(kp)
    s = _solver(n, p, l, k, precision=prec)
    g = s.dirichlet_point_source(SRC)
    b = torch.zeros_like(g)
    u, st = s.solve_dirichlet(b, g, tol=1e-12 if prec == ddh.PREC_FP64 else 1e-10)
    ref = D.Solver(n, p, l, k)
    gr = D.lifting(n, p, data)
    phi, _, _ = ref.solve(np.zeros_like(gr), gr, tol=1e-12)
    tol = 1e-9 if prec == ddh.PREC_FP64 else 1e-8
    assert _rel(u.cpu().numpy()[0], phi) <= tol, _rel(u.cpu().numpy()[0], phi)
    assert st[0].primal_residual <= 1e-10, st[0].primal_residual
    s.close()


def test_helmholtz_dirichlet_solves_run_fgmres_not_pcg():
    """The Helmholtz problem with Dirichlet data is indefinite: the solve runs FGMRES (its
    iteration count equals the oracle's FGMRES on the same problem), and the PCG spectrum of the
    Poisson mode is not available."""
    k, data = D.table3_problem(11.0)
    s = _solver(1, 8, 1, k, dual_stop=1, maxit=110, restart=110)
    g = s.dirichlet_point_source(SRC)
    _, st = s.solve_dirichlet(torch.zeros_like(g), g, tol=1e-10)
    gr = D.lifting(1, 8, data)
    _, its, _ = D.Solver(1, 8, 1, k).solve(np.zeros_like(gr), gr, tol=1e-10, maxit=110)
    assert abs(st[0].iterations - its) <= 2, (st[0].iterations, its)
    with pytest.raises(ddh.DDHError):
        s.pcg_spectrum(0)
    s.close()


def test_field_is_the_point_source():
    """p = 16 on 4 x 4 squares at the paper's k = 21: the field at seeded points equals
    -(i/4) H0^(2)(k |x - x_c|) to the discretisation error."""
    k, data = D.table3_problem(21.0)
    s = _solver(2, 16, 4, k)
    g = s.dirichlet_point_source(SRC)
    u, _ = s.solve_dirichlet(torch.zeros_like(g), g, tol=1e-12)
    xy = np.random.default_rng(6).uniform(0.0, 1.0, size=(64, 2))
    vals = s.eval_points(xy, u).cpu().numpy()[0]
    ex = data(xy[:, 0], xy[:, 1])
    assert np.max(np.abs(vals - ex)) <= 1e-6 * np.max(np.abs(ex)), np.max(np.abs(vals - ex))
    s.close()


GPU_ROWS = [r for r in _rows() if r[0] == 8 or (r[0] == 16 and r[1] <= 256) or (r[0] == 32 and r[1] in (16, 1024))]


@pytest.mark.parametrize("p,N,k,l,its,bold", GPU_ROWS, ids=[f"p{r[0]}-N{r[1]}-k{r[2]}-l{r[3]}" for r in GPU_ROWS])
def test_table3_iterations(p, N, k, l, its, bold):
    n = int(round(np.log(N) / np.log(4)))
    kk, _ = D.table3_problem(float(k))
    s = _solver(n, p, l, kk, dual_stop=1, maxit=110, restart=110)
    g = s.dirichlet_point_source(SRC)
    _, st = s.solve_dirichlet(torch.zeros_like(g), g, tol=1e-10, allow_noconv=True)
    got = st[0].iterations
    if its < 0:
        assert got >= 95, got
    else:
        # runs of 40-110 iterations on an indefinite problem are sensitive to rounding (the
        # oracle itself gives 59 or 61 for p = 8, N = 4, k = 11, l = 1 on two hosts) and the
        # paper's PGMRES is left-preconditioned: two iterations or 6 %
        assert abs(got - its) <= max(2.0, 0.06 * its), (got, its)
    s.close()
