"""The allocation-free primal-residual entry point, called through the C ABI.

Some callers cannot allocate device memory where they need the FP64 residual: applications
that reserve their whole device-memory budget at start-up and forbid later cudaMalloc calls,
and callers in latency-critical loops that avoid cudaMalloc/cudaFree because those can
synchronise the whole device.  They use ddh_primal_residual_noalloc, which works in a
file-scope device scratch array instead of the context's work buffers.  It must give the same
residuals as ddh_primal_residual on consecutive calls (the shared scratch keeps the last call's
contents), leave free device memory unchanged, and reject problems larger than its scratch,
too many right-hand sides and calls before factor with clear errors.
This file is collected last on purpose."""
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


def _context(w):
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(tol=1e-10)
    return s


def test_noalloc_matches_allocating_entry_point_and_allocates_nothing():
    w = W.small_hanging(4, refine=[(0, 0), (3, 2)], levels=2, p=7, k=9.0, seed=4, p_range=(5, 9), n_rhs=3)
    s = _context(w)
    b = s.rhs_planewave(w.thetas)
    u, _ = s.solve(b, tol=1e-10)
    torch.cuda.synchronize()
    # the allocation-free call comes first on this context: it cannot lean on the residual's
    # work buffers, which ddh_primal_residual creates on its first call
    got = []
    free_after = []
    for call in range(3):
        st, r = _residual_noalloc(s, b, u)
        assert st == ddh.OK, s.lib.ddh_last_error(s.h).decode()
        got.append(r)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info(0)[0])
    # the first call may load kernel code; the later ones must not change free device memory
    assert free_after[1] == free_after[0] and free_after[2] == free_after[0], free_after
    ref = s.primal_residual(b, u)
    for call, r in enumerate(got):
        assert np.allclose(r, ref, rtol=1e-12, atol=0.0), (call, r, ref)
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
    s = _context(w)
    R = 8                      # 16 R (4 n_local + n_conforming) bytes > 32 MiB
    b = s.rhs_planewave(np.linspace(0.1, 1.0, R))
    st, _ = _residual_noalloc(s, b, b)
    assert st == ddh.ERR_INVALID_ARG
    assert "32 MiB" in s.lib.ddh_last_error(s.h).decode()
    st, got = _residual_noalloc(s, b[:1].contiguous(), b[:1].contiguous())
    assert st == ddh.OK
    s.close()


def test_noalloc_rejects_too_many_rhs_and_calls_before_factor():
    w = W.plane_2x2()
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    x = torch.zeros((1, 324), dtype=torch.complex128, device="cuda:0")
    st, _ = _residual_noalloc(s, x, x)
    assert st == ddh.ERR_NOT_READY
    assert "factor first" in s.lib.ddh_last_error(s.h).decode()
    s.factor(tol=1e-10)
    R = 513                    # one more than the entry point's limit, well inside 32 MiB here
    b = torch.zeros((R, s.info().n_local), dtype=torch.complex128, device="cuda:0")
    st, _ = _residual_noalloc(s, b, b)
    assert st == ddh.ERR_INVALID_ARG
    assert "at most 512 right-hand sides" in s.lib.ddh_last_error(s.h).decode()
    s.close()
