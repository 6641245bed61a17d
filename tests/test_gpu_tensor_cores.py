"""The tensor-core Krylov-loop pass 1 (tcgen05, TF32) of the mixed-precision inner solves.

* One application of the interface operator F with the TF32 pass matches the oracle's F to the
  TF32 rounding of the element operators and of the right-hand sides (10-bit mantissas:
  relative 2^-11 per operand, bound 2e-3 on the result), on meshes with mixed degrees and
  hanging nodes, for 1, 8 and 20 right-hand sides (MMA widths 16 and 32 with padding).
* Solves with it still meet the FP64 primal residual 1e-10 (the outer FGMRES is FP64) and match
  the FP64 oracle's solution to 1e-8.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dd  # noqa: E402
from paper_1808_04713_gb300 import ddh  # noqa: E402

MESHES = {
    "plane_2x2": W.plane_2x2,
    "uniform4_mixed_p": lambda: W.small_uniform(4, 6, 9.0, seed=7, eps_range=(1, 2), p_range=(4, 9)),
    "hanging_corner": lambda: W.small_hanging(4, refine=[(0, 0), (3, 2)], levels=2, p=7, k=9.0, seed=4,
                                              p_range=(5, 9), n_rhs=3),
    "multilevel": lambda: W.multilevel_hanging(p=5, k=3.0),
    "wide_p20": lambda: W.small_uniform(3, 20, 12.0, seed=9, eps_range=(1, 2), n_rhs=3),
}


def _solver(w, **opt):
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(**opt)
    return s


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("R", [1, 8, 20])
def test_tensor_core_interface_operator_matches_oracle(name, R):
    w = MESHES[name]()
    s = _solver(w, tol=1e-10, precision=ddh.PREC_MIXED_FP32, tensor_cores=1)
    ref = dd.DDSolver(dd.problem_from_workload(w), l=s.info().l)
    rng = np.random.default_rng(R)
    nu = rng.standard_normal((R, ref.nd)) + 1j * rng.standard_normal((R, ref.nd))
    Fv = s.apply_dual_operator(0, torch.tensor(nu, device="cuda:0"), ddh.PREC_MIXED_FP32).cpu().numpy()
    worst = max(_rel(Fv[r], ref.apply_F(nu[r])) for r in range(R))
    assert worst <= 2e-3, worst
    # the complex64 CUDA-core pass of the same context is more accurate than the TF32 one
    s2 = _solver(w, tol=1e-10, precision=ddh.PREC_MIXED_FP32, tensor_cores=0)
    F2 = s2.apply_dual_operator(0, torch.tensor(nu, device="cuda:0"), ddh.PREC_MIXED_FP32).cpu().numpy()
    assert max(_rel(F2[r], ref.apply_F(nu[r])) for r in range(R)) <= 1e-5
    s.close()
    s2.close()


@pytest.mark.parametrize("name", list(MESHES))
def test_tensor_core_solve_meets_fp64_yardstick(name):
    w = MESHES[name]()
    s = _solver(w, tol=1e-10, precision=ddh.PREC_MIXED_FP32, tensor_cores=1)
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-10)
    ref = dd.Conforming(dd.problem_from_workload(w)).solve_direct()
    got = u.cpu().numpy()
    for r in range(got.shape[0]):
        assert st[r].primal_residual <= 1e-10
        assert _rel(got[r], ref[r]) <= 1e-8, (name, r)
    s.close()
