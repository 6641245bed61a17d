"""CPU-side checks of the native library: it loads, exports every symbol declared in
include/ddh.h, and its host-only tables agree with the oracle's independent definitions."""
import os
import re

import numpy as np
import pytest

from oracle import legendre as lg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_04713_gb300 import build as b
    b.build()
    from paper_1808_04713_gb300 import ddh
    return ddh.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "ddh.h")).read()
    names = set(re.findall(r"\b(ddh_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("n,a,b", [(12, 0.5, 0.5), (16, 0.5, -0.5), (20, 0.25, -0.75), (24, 0.25, 0.25)])
def test_affine_recurrence_matches_quadrature(lib, n, a, b):
    from paper_1808_04713_gb300 import ddh
    assert np.abs(ddh.table_affine(n, a, b) - lg.affine_L_tilde(n, a, b)).max() < 5e-12


@pytest.mark.parametrize("p", [3, 8, 16, 24, 32])
def test_fdm_table(lib, p):
    from paper_1808_04713_gb300 import ddh
    V, mu = ddh.table_fdm(p)
    Mb = (lg.B_matrix(p) @ lg.mass_1d(p) @ lg.B_matrix(p))[2:, 2:]
    assert np.abs(V @ np.diag(mu) @ V.T - Mb).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(p - 1)).max() < 1e-13
    par = np.add.outer(np.arange(p - 1), np.arange(p - 1)) % 2 == 1
    assert np.all(V[par] == 0.0)
    assert np.allclose(np.sort(mu), np.linalg.eigvalsh(Mb), atol=1e-14)


def test_gauss_rule(lib):
    from paper_1808_04713_gb300 import ddh
    x, w = ddh.table_gauss(40)
    xo, wo = np.polynomial.legendre.leggauss(40)
    assert np.abs(x - xo).max() < 1e-14 and np.abs(w - wo).max() < 1e-14


def test_missing_library_fails_loudly(tmp_path):
    # the product path has no fallback: without the built library every entry point raises
    from paper_1808_04713_gb300 import ddh
    with pytest.raises(ImportError, match="not built"):
        ddh.load_library(str(tmp_path / "libddh.so"))


def test_context_without_gpu_reports_an_error(lib):
    # with no CUDA device visible, creating a solver context fails with a status, not a crash
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    from paper_1808_04713_gb300 import ddh
    with pytest.raises(ddh.DDHError, match="create failed"):
        ddh.DDH(0)
