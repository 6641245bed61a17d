"""ctypes binding of libddh.so (argument marshalling only; every step runs in the library).

The library must have been built (``paper_1808_04713_gb300.build.build()``); loading fails
loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libddh.so")
_lib = None

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_READY, ERR_NO_CONVERGENCE, ERR_SINGULAR, \
    WARN_NEAR_RESONANT, ERR_DEVICE_FLAG = range(9)
PREC_FP64, PREC_MIXED_FP32 = 0, 1
PRECOND_DIRICHLET, PRECOND_LUMPED, PRECOND_NONE = 0, 1, 2
LOCAL_EDGE, LOCAL_FDM = 0, 1
BOUNDARY_IMPEDANCE, BOUNDARY_DIRICHLET = 0, 1
COARSE_AUTO, COARSE_DENSE, COARSE_ND, COARSE_ND_LEVELS = 0, 1, 2, 3
EDGE_LAUNCH_AUTO, EDGE_LAUNCH_PER_TASK, EDGE_LAUNCH_PERSISTENT = 0, 1, 2


class DDHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ddh status {status}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("restart", C.c_int32),
                ("l_override", C.c_int32), ("precision", C.c_int32), ("precond", C.c_int32),
                ("inner_iters", C.c_int32), ("check_every", C.c_int32), ("use_graph", C.c_int32),
                ("coarse_fp32", C.c_int32), ("local_form", C.c_int32),
                ("inner_tol", C.c_double), ("coarse_form", C.c_int32), ("robin_modified", C.c_int32),
                ("tensor_cores", C.c_int32), ("inner_krylov_fp32", C.c_int32), ("edge_launch", C.c_int32),
                ("nd_chains", C.c_int32), ("inner_passes_fp64", C.c_int32), ("split_pass1", C.c_int32),
                ("nd_pdl", C.c_int32), ("dual_stop", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("l", C.c_int32), ("n_local", C.c_int64),
                ("n_dual", C.c_int64), ("n_coarse", C.c_int64), ("n_conforming", C.c_int64),
                ("n_coarse_blocks", C.c_int32), ("max_block", C.c_int32),
                ("min_resonance_gap", C.c_double), ("factor_seconds", C.c_double),
                ("coarse_nd_flops", C.c_double), ("coarse_form", C.c_int32), ("coarse_subtrees", C.c_int32)]


class RhsStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("inner_iterations", C.c_int32),
                ("dual_residual", C.c_double), ("primal_residual", C.c_double)]


_SIGS = {
    "ddh_default_options": (None, [C.POINTER(Options)]),
    "ddh_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "ddh_set_mesh": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "ddh_set_coefficients": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "ddh_set_poisson": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ddh_set_boundary": (C.c_int, [C.c_void_p, C.c_int32]),
    "ddh_set_pml": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ddh_dirichlet_point_source": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ddh_solve_dirichlet": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                      C.c_void_p]),
    "ddh_pcg_spectrum": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "ddh_factor": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "ddh_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "ddh_elem_offsets": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ddh_rhs_planewave": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ddh_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p]),
    "ddh_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p]),
    "ddh_adjoint_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p]),
    "ddh_grad_eps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ddh_eval_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "ddh_grad_k": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ddh_primal_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ddh_primal_residual_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ddh_apply_dual_operator": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "ddh_get_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "ddh_kernel_launches": (C.c_int64, [C.c_void_p]),
    "ddh_profile_op": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "ddh_last_error": (C.c_char_p, [C.c_void_p]),
    "ddh_destroy": (None, [C.c_void_p]),
    "ddh_table_affine": (C.c_int, [C.c_int32, C.c_double, C.c_double, C.c_void_p]),
    "ddh_table_fdm": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p]),
    "ddh_table_gauss": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p]),
    "ddh_host_factor": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                  C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
}


def load_library(path: str | None = None):
    """Load libddh.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libddh.so not built at {p}; run paper_1808_04713_gb300.build.build()")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def default_options(**kw) -> Options:
    o = Options()
    load_library().ddh_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return int(t.data_ptr())


class DDH:
    """One solver context on one CUDA device (names follow the C ABI)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load_library()
        self.torch = torch
        self.device = device
        self.h = C.c_void_p()
        s = None if stream is None else C.c_void_p(stream.cuda_stream)
        self._check(self.lib.ddh_create(C.byref(self.h), device, s))
        self.n_elem = 0
        self.n_local = 0
        self.last_status = OK

    def _check(self, st: int, allow=(OK,)):
        self.last_status = st
        if st not in allow:
            msg = self.lib.ddh_last_error(self.h).decode() if self.h else "create failed"
            raise DDHError(st, msg)
        return st

    def close(self):
        if self.h:
            self.lib.ddh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup
    def set_mesh(self, base_n: int, leaves, p):
        lv = np.ascontiguousarray(leaves, dtype=np.int32)
        pp = np.ascontiguousarray(p, dtype=np.int32)
        self._check(self.lib.ddh_set_mesh(self.h, int(base_n), lv.ctypes.data, pp.ctypes.data, int(lv.shape[0])))
        self.n_elem = int(lv.shape[0])

    def set_coefficients(self, k: float, eps):
        e = np.ascontiguousarray(eps, dtype=np.float64)
        self._check(self.lib.ddh_set_coefficients(self.h, float(k), e.ctypes.data))

    def set_poisson(self, rho):
        """Poisson mode: -div(rho grad phi) = f, zero Dirichlet data, rho per element."""
        r = np.ascontiguousarray(rho, dtype=np.float64)
        self._check(self.lib.ddh_set_poisson(self.h, r.ctypes.data))

    def set_pml(self, s1, s2):
        """Complex stretch factors per element along x1 and x2 (1 outside the layers)."""
        a = np.asarray(s1, dtype=np.complex128)
        b = np.asarray(s2, dtype=np.complex128)
        v = np.ascontiguousarray(np.stack([a.real, a.imag, b.real, b.imag], axis=1).ravel(), dtype=np.float64)
        self._check(self.lib.ddh_set_pml(self.h, v.ctypes.data))

    def set_boundary(self, kind: int):
        """BOUNDARY_IMPEDANCE (default) or BOUNDARY_DIRICHLET for the Helmholtz problem."""
        self._check(self.lib.ddh_set_boundary(self.h, int(kind)))

    def dirichlet_point_source(self, src):
        """Lifting [R, n_local] of the data -(i/4) H0^(2)(k |x - x_c|) for centres src [R, 2]."""
        c = np.ascontiguousarray(np.atleast_2d(src), dtype=np.float64)
        g = self._vec(c.shape[0])
        self._check(self.lib.ddh_dirichlet_point_source(self.h, c.ctypes.data, int(c.shape[0]), _ptr(g)))
        return g

    def solve_dirichlet(self, b, g, tol: float = 0.0, out=None, stats: bool = True, allow_noconv: bool = False):
        """phi = g + phi_0 for load b and Dirichlet lifting g (both [R, n_local])."""
        b = b.contiguous()
        g = g.contiguous()
        R = b.shape[0]
        u = self._vec(R) if out is None else out
        st = (RhsStats * R)() if stats else None
        allow = (OK, ERR_NO_CONVERGENCE) if allow_noconv else (OK,)
        self._check(self.lib.ddh_solve_dirichlet(self.h, _ptr(b), _ptr(g), _ptr(u), R, float(tol),
                                                 C.cast(st, C.c_void_p) if stats else None), allow=allow)
        return u, (list(st) if stats else None)

    def pcg_spectrum(self, r: int = 0):
        """(lambda_min, lambda_max) Lanczos estimates of P^-1 F from the last Poisson solve."""
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.ddh_pcg_spectrum(self.h, int(r), C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def factor(self, **opts) -> int:
        o = default_options(**opts)
        st = self._check(self.lib.ddh_factor(self.h, C.byref(o)), allow=(OK, WARN_NEAR_RESONANT))
        self.n_local = self.info().n_local
        return st

    def info(self) -> Info:
        i = Info()
        self._check(self.lib.ddh_get_info(self.h, C.byref(i)))
        return i

    def elem_offsets(self) -> np.ndarray:
        o = np.zeros(self.n_elem + 1, np.int64)
        self._check(self.lib.ddh_elem_offsets(self.h, o.ctypes.data))
        return o

    def _vec(self, R):
        return self.torch.zeros((R, self.n_local), dtype=self.torch.complex128, device=f"cuda:{self.device}")

    def rhs_planewave(self, thetas):
        th = np.ascontiguousarray(np.atleast_1d(thetas), dtype=np.float64)
        b = self._vec(th.size)
        self._check(self.lib.ddh_rhs_planewave(self.h, th.ctypes.data, int(th.size), _ptr(b)))
        return b

    def solve(self, b, tol: float = 0.0, out=None, stats: bool = True, allow_noconv: bool = False):
        b = b.contiguous()
        R = b.shape[0]
        u = self._vec(R) if out is None else out
        st = (RhsStats * R)() if stats else None
        allow = (OK, ERR_NO_CONVERGENCE) if allow_noconv else (OK,)
        self._check(self.lib.ddh_solve(self.h, _ptr(b), _ptr(u), R, float(tol),
                                       C.cast(st, C.c_void_p) if stats else None), allow=allow)
        return u, (list(st) if stats else None)

    def solve_host(self, b_host: np.ndarray, tol: float = 0.0, stats: bool = False):
        b = np.ascontiguousarray(b_host, dtype=np.complex128)
        u = np.zeros_like(b)
        R = b.shape[0]
        st = (RhsStats * R)() if stats else None
        self._check(self.lib.ddh_solve_host(self.h, b.ctypes.data, u.ctypes.data, R, float(tol),
                                            C.cast(st, C.c_void_p) if stats else None))
        return u, (list(st) if stats else None)

    def adjoint_solve(self, g, tol: float = 0.0):
        g = g.contiguous()
        R = g.shape[0]
        lam = self._vec(R)
        st = (RhsStats * R)()
        self._check(self.lib.ddh_adjoint_solve(self.h, _ptr(g), _ptr(lam), R, float(tol), C.cast(st, C.c_void_p)))
        return lam, list(st)

    def grad_eps(self, u, lam):
        """dJ/deps_e = k^2 (h_e/2)^2 Re(lam_e^T M_e u_e) summed over right-hand sides."""
        g = self.torch.zeros(self.n_elem, dtype=self.torch.float64, device=f"cuda:{self.device}")
        R = u.shape[0]
        self._check(self.lib.ddh_grad_eps(self.h, _ptr(u.contiguous()), _ptr(lam.contiguous()), R, _ptr(g)))
        return g

    def grad_k(self, u, lam, thetas) -> float:
        th = np.ascontiguousarray(np.atleast_1d(thetas), dtype=np.float64)
        out = C.c_double()
        self._check(self.lib.ddh_grad_k(self.h, _ptr(u.contiguous()), _ptr(lam.contiguous()), th.ctypes.data,
                                        int(th.size), C.byref(out)))
        return out.value

    def eval_points(self, xy, u):
        """u(x_i) for points xy [n, 2]; u: [R, n_local] -> [R, n] complex."""
        pts = np.ascontiguousarray(xy, dtype=np.float64)
        R = u.shape[0]
        out = self.torch.zeros((R, pts.shape[0]), dtype=self.torch.complex128, device=f"cuda:{self.device}")
        self._check(self.lib.ddh_eval_points(self.h, pts.ctypes.data, pts.shape[0], R, _ptr(u.contiguous()), _ptr(out), 0))
        return out

    def inject_points(self, xy, w):
        """Transpose of eval_points: w [R, n] -> local vector [R, n_local]."""
        pts = np.ascontiguousarray(xy, dtype=np.float64)
        R = w.shape[0]
        out = self._vec(R)
        self._check(self.lib.ddh_eval_points(self.h, pts.ctypes.data, pts.shape[0], R, _ptr(w.contiguous()), _ptr(out), 1))
        return out

    def primal_residual(self, b, u) -> np.ndarray:
        R = b.shape[0]
        out = np.zeros(R)
        self._check(self.lib.ddh_primal_residual(self.h, _ptr(b.contiguous()), _ptr(u.contiguous()), R, out.ctypes.data))
        return out

    def apply_dual_operator(self, which: int, v, precision: int = PREC_FP64):
        """F v (which = 0) or P^-1 v (which = 1) for dual vectors v [R, n_dual] (complex128)."""
        v = v.contiguous()
        out = self.torch.zeros_like(v)
        self._check(self.lib.ddh_apply_dual_operator(self.h, int(which), _ptr(v), _ptr(out), int(v.shape[0]),
                                                     int(precision)))
        return out

    def get_tuning(self, R: int, precision: int = PREC_FP64) -> dict:
        """Autotuner choices for R right-hand sides: the launch form of the edge pass (1
        persistent, 0 one CTA per task, -1 untuned), its threads per output row by degree, the
        right-hand-side block of each nested-dissection level launch and the number of level
        chains (1, 2 or 4, over equal right-hand-side shares on forked streams)."""
        tpr = np.zeros(33, np.int32)
        nd = np.zeros(128, np.int32)
        L = C.c_int32()
        ep = C.c_int32()
        ent = C.c_int32()
        ch = C.c_int32()
        fs = np.zeros(4, np.int32)
        self._check(self.lib.ddh_get_tuning(self.h, int(R), int(precision), C.byref(ep), C.byref(ent),
                                            tpr.ctypes.data, nd.ctypes.data, C.byref(L), C.byref(ch), fs.ctypes.data))
        return {"edge_persistent": int(ep.value), "edge_cta_threads": int(ent.value),
                "tpr_by_degree": {int(p): int(t) for p, t in enumerate(tpr) if t},
                "nd_chains": int(ch.value),
                "fdm_pass1": {"batch": int(fs[0]), "staged": int(fs[1])},
                "fdm_pass2": {"batch": int(fs[2]), "staged": int(fs[3])},
                "nd_rb_forward": nd[:L.value].tolist(), "nd_rb_backward": nd[L.value:2 * L.value].tolist()}

    def profile_op(self, R: int, precision: int = PREC_FP64, reps: int = 20) -> np.ndarray:
        """Average ms per launch: pass1, coarse assembly, coarse solve, pass2, jump gather, precond."""
        out = np.zeros(6)
        self._check(self.lib.ddh_profile_op(self.h, R, precision, reps, out.ctypes.data))
        return out

    def kernel_launches(self) -> int:
        return int(self.lib.ddh_kernel_launches(self.h))


# -- host-only tables (no GPU needed)
def table_affine(n: int, a: float, b: float) -> np.ndarray:
    out = np.zeros((n + 1, n + 1))
    st = load_library().ddh_table_affine(n, a, b, out.ctypes.data)
    if st:
        raise DDHError(st, "table_affine")
    return out


def table_fdm(p: int):
    n = p - 1
    V = np.zeros((n, n))
    mu = np.zeros(n)
    st = load_library().ddh_table_fdm(p, V.ctypes.data, mu.ctypes.data)
    if st:
        raise DDHError(st, "table_fdm")
    return V, mu


def table_gauss(m: int):
    x = np.zeros(m)
    w = np.zeros(m)
    st = load_library().ddh_table_gauss(m, x.ctypes.data, w.ctypes.data)
    if st:
        raise DDHError(st, "table_gauss")
    return x, w


def host_factor(base_n, leaves, p, k, eps, l_override: int = 0):
    """Host-only setup + factorisation; returns (sizes dict, seconds, l)."""
    lv = np.ascontiguousarray(leaves, dtype=np.int32)
    pp = np.ascontiguousarray(p, dtype=np.int32)
    ee = np.ascontiguousarray(eps, dtype=np.float64)
    sizes = np.zeros(8, np.int64)
    secs = np.zeros(5)
    l = C.c_int32()
    st = load_library().ddh_host_factor(int(base_n), lv.ctypes.data, pp.ctypes.data, int(lv.shape[0]), float(k),
                                        ee.ctypes.data, int(l_override), sizes.ctypes.data, secs.ctypes.data,
                                        C.byref(l))
    if st:
        raise DDHError(st, "host_factor")
    keys = ["n_local", "n_dual", "n_coarse", "n_conforming", "n_e1", "n_t", "blocks", "max_block"]
    return dict(zip(keys, sizes.tolist())), secs, l.value
