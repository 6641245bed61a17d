"""GPU parity of the axis-aligned PML (Sec. 4, complex coordinate stretching) against the oracle.

The stretched element operators (s2/s1) K(x1) M(x2) + (s1/s2) M(x1) K(x2) - k^2 (h/2)^2 s1 s2 M (x) M
enter the host factor (explicit edge operators, coarse matrix), the element fast solver of the RHS
pass and the recovery (complex divide, anisotropic frame coupling) and the FP64 yardstick.  Checked
against oracle/pml.py, which is pinned to the exact stretched plane wave and to the layer's
absorption, on meshes closed by zero Dirichlet data beyond the layers:

* one application of F and of the (unstretched) Dirichlet preconditioner, relative 1e-12, with a
  layer along x1 and with layers along both axes (corner elements stretched twice), in the
  explicit-edge-operator form and in the FDM form of the Krylov loop;
* complete solves with seeded random loads: FP64 relative 1e-9 of the oracle's field (both sides
  to 1e-12), the mixed form relative 1e-8, and the FP64 primal residual of the stretched system.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import pml  # noqa: E402
from oracle import poisson as P  # noqa: E402
from paper_1808_04713_gb300 import ddh  # noqa: E402

K, SIGMA = 20.0, 30.0


def _case(n, p, l, axes, **opt):
    m = 2 ** n
    s1, s2 = pml.stretch(m, K, 1, SIGMA, axes=axes)
    s = ddh.DDH(0)
    s.set_mesh(m, P.uniform_leaves(m), np.full(m * m, p))
    s.set_coefficients(K, np.ones(m * m))
    s.set_pml(s1, s2)
    s.set_boundary(ddh.BOUNDARY_DIRICHLET)
    s.factor(l_override=l, **opt)
    return s, pml.Solver(n, p, l, K, s1, s2)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("axes,opt", [((0,), {}), ((0, 1), {}), ((0, 1), {"local_form": ddh.LOCAL_FDM})],
                         ids=["x1_layer", "both_layers", "both_layers_fdm_form"])
def test_operator_and_preconditioner_match_oracle(axes, opt):
    s, ref = _case(2, 8, 2, axes, **opt)
    info = s.info()
    assert (info.n_dual, info.n_coarse) == (ref.dd.nd, ref.dd.n2)
    rng = np.random.default_rng(12)
    nu = rng.standard_normal((2, ref.dd.nd)) + 1j * rng.standard_normal((2, ref.dd.nd))
    v = torch.tensor(nu, device="cuda:0")
    Fv = s.apply_dual_operator(0, v, ddh.PREC_FP64).cpu().numpy()
    Pv = s.apply_dual_operator(1, v, ddh.PREC_FP64).cpu().numpy()
    for r in range(2):
        fo = ref.S.apply_F(nu[r])
        po = ref.S.apply_P(nu[r].real) + 1j * ref.S.apply_P(nu[r].imag)
        assert _rel(Fv[r], fo) <= 1e-12, ("F", _rel(Fv[r], fo))
        assert _rel(Pv[r], po) <= 1e-12, ("P", _rel(Pv[r], po))
    s.close()


@pytest.mark.parametrize("axes,prec", [((0,), ddh.PREC_FP64), ((0, 1), ddh.PREC_FP64), ((0, 1), ddh.PREC_MIXED_FP32)],
                         ids=["x1_fp64", "both_fp64", "both_mixed"])
def test_solution_matches_oracle(axes, prec):
    n, p, l = 2, 9, 3
    s, ref = _case(n, p, l, axes, precision=prec)
    N2 = (p + 1) ** 2
    b = np.random.default_rng(31).uniform(-1.0, 1.0, size=(2, 16 * N2)).astype(np.complex128)
    u, st = s.solve(torch.tensor(b, device="cuda:0"), tol=1e-12 if prec == ddh.PREC_FP64 else 1e-10)
    u = u.cpu().numpy()
    tol = 1e-9 if prec == ddh.PREC_FP64 else 1e-8
    for r in range(2):
        phi, _ = ref.solve(b[r], np.zeros(16 * N2, complex), tol=1e-12)
        assert _rel(u[r], phi) <= tol, (r, _rel(u[r], phi))
        assert st[r].primal_residual <= 1e-10, st[r].primal_residual
    s.close()


def test_gradients_are_refused_with_a_layer():
    s, _ = _case(1, 6, 2, (0,))
    u = torch.zeros((1, s.info().n_local), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(ddh.DDHError):
        s.grad_eps(u, u)
    s.close()
