"""The allocation-free primal-residual entry point, called through the C ABI.

Callers that cannot allocate device memory at the point of the call (stream capture into a
CUDA graph, fixed device-memory budgets) use ddh_primal_residual_noalloc, which works in a
file-scope device scratch array instead of context work buffers.  It must give the same
residuals as ddh_primal_residual, on two calls in a row (the shared scratch keeps the last
call's contents), and reject problems larger than its scratch with a clear error.
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1808_04713_gb300 import ddh  # noqa: E402


def _residual_noalloc(s, b, u):
    R = b.shape[0]
    out = np.zeros(R)
    st = s.lib.ddh_primal_residual_noalloc(s.h, b.data_ptr(), u.data_ptr(), R, out.ctypes.data)
    return st, out


def test_noalloc_matches_allocating_entry_point_twice():
    w = W.small_hanging(4, refine=[(0, 0), (3, 2)], levels=2, p=7, k=9.0, seed=4, p_range=(5, 9), n_rhs=3)
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(tol=1e-10)
    b = s.rhs_planewave(w.thetas)
    u, _ = s.solve(b, tol=1e-10)
    ref = s.primal_residual(b, u)
    for call in range(2):
        st, got = _residual_noalloc(s, b, u)
        assert st == ddh.OK, s.lib.ddh_last_error(s.h).decode()
        assert np.allclose(got, ref, rtol=1e-12, atol=0.0), (call, got, ref)
    # a second, different input through the same scratch: a perturbed solution
    u2 = u.clone()
    u2[:, ::7] += 1e-3
    ref2 = s.primal_residual(b, u2)
    st, got2 = _residual_noalloc(s, b, u2)
    assert st == ddh.OK and np.allclose(got2, ref2, rtol=1e-12)
    assert np.all(got2 > ref)
    s.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    w = W.plane_16x16()
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(tol=1e-10)
    R = 8                      # 16 R (4 n_local + n_conforming) bytes > 32 MiB
    b = s.rhs_planewave(np.linspace(0.1, 1.0, R))
    st, _ = _residual_noalloc(s, b, b)
    assert st == ddh.ERR_INVALID_ARG
    assert "32 MiB" in s.lib.ddh_last_error(s.h).decode()
    st, got = _residual_noalloc(s, b[:1].contiguous(), b[:1].contiguous())
    assert st == ddh.OK
    s.close()
