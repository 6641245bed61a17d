"""GPU parity on the paths the full-size workloads take, element by element against the oracle.

* the nested-dissection coarse solve (forced on small meshes: the default uses a dense K^-1
  below 6144 coarse unknowns), in its one-launch form (work items in elimination-tree order)
  and its per-level form, the latter with the subtree launches (fewer than 4 right-hand sides
  on a tree with a level of at least 300 fronts) and without (4 or more right-hand sides);
* a reduced batching workload: the disk refinement (2 levels, 3 hanging nodes per coarse
  edge), p ~ U{8..24}, eps = 4 in the disk, the element k h of the full workload, 16 right-hand
  sides, in both precisions;
* wide element rows (p = 20: two threads per output row of the edge pass and one per row of the
  FDM-form S_E^-1 product; p = 24 in FP64: S_E^-1 staged only with the smaller interior batches
  the FDM-pass autotuner tries; p = 32: S_E^-1 too large to stage in shared memory);
* the two operators of the dual iteration applied once: F nu (eq. complicated_schur_system) and
  the Dirichlet preconditioner P^-1 v (eqs. general_preconditioner, weight_matrix).

Tolerances: FP64 relative L2 <= 1e-10 over the element-local N-basis coefficients with both
sides solved to relative residual 1e-12; the mixed form (complex64 inner solves) <= 1e-8 with
the FP64 primal residual <= 1e-10; one operator application <= 1e-12 (FP64) and <= 1e-5
(complex64 element arithmetic, about 100 units of FP32 rounding).
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


def _solver(w, **opt):
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(**opt)
    return s


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _with_rhs(w, R, seed=21):
    w.thetas = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, size=R)
    return w


# ---------------------------------------------------------------- nested-dissection coarse solve
ND_SMALL = {
    "uniform4_mixed_p": lambda: W.small_uniform(4, 6, 9.0, seed=7, eps_range=(1, 2), p_range=(4, 9)),
    "hanging_corner": lambda: W.small_hanging(4, refine=[(0, 0), (3, 2)], levels=2, p=7, k=9.0, seed=4,
                                              p_range=(5, 9)),
    "multilevel": lambda: W.multilevel_hanging(p=5, k=3.0),
}


@pytest.mark.parametrize("name", list(ND_SMALL))
@pytest.mark.parametrize("R", [1, 8])
@pytest.mark.parametrize("form", [ddh.COARSE_ND, ddh.COARSE_ND_LEVELS])
def test_nested_dissection_coarse_path_matches_oracle(name, R, form):
    w = _with_rhs(ND_SMALL[name](), R)
    s = _solver(w, tol=1e-12, coarse_form=form)
    info = s.info()
    assert info.coarse_form == form and info.n_coarse_blocks > 1
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-12)
    prob = dd.problem_from_workload(w)
    ref = dd.DDSolver(prob, l=info.l).solve(tol=1e-12)
    got = u.cpu().numpy()
    for r in range(R):
        assert _rel(got[r], ref["phi_N"][r]) <= 1e-10, (name, R, r)
        assert ref["iterations"][r] - 1 <= st[r].iterations <= ref["iterations"][r] + 6
    s.close()


@pytest.mark.parametrize("R", [1, 4])
@pytest.mark.parametrize("form", [ddh.COARSE_ND, ddh.COARSE_ND_LEVELS])
def test_nested_dissection_on_a_deep_tree(R, form):
    """48 x 48 squares, p = 6, l = 2 (the elimination tree of the 48 x 48 base grid with edge
    unknowns in the coarse space: 2491 fronts).  One launch per level: with one right-hand side
    the bottom levels run as one subtree launch per direction, with four as one launch per
    level.  One launch in all: every front's work items in dependency order."""
    w = _with_rhs(W.small_uniform(48, 6, 40.0, seed=3, eps_range=(1, 2)), R)
    s = _solver(w, tol=1e-12, coarse_form=form, l_override=2)
    info = s.info()
    assert info.coarse_form == form
    if form == ddh.COARSE_ND_LEVELS:
        assert info.coarse_subtrees > 0
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-12)
    prob = dd.problem_from_workload(w)
    ref = dd.Conforming(prob).solve_direct()
    got = u.cpu().numpy()
    for r in range(R):
        assert _rel(got[r], ref[r]) <= 1e-10, (R, r)
        assert st[r].primal_residual <= 1e-11
    s.close()


@pytest.mark.parametrize("R", [1, 8])
def test_nested_dissection_forms_agree_at_full_size(R):
    """lens_48 (21217 coarse unknowns, 2491 fronts): the one-launch and per-level coarse solves
    apply the same factor, so the solutions agree to the solve tolerance."""
    w = _with_rhs(W.lens_48(), R)
    out = {}
    for form in (ddh.COARSE_ND, ddh.COARSE_ND_LEVELS):
        s = _solver(w, tol=1e-10, coarse_form=form)
        u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-10)
        out[form] = (u.cpu().numpy(), [x.iterations for x in st], [x.primal_residual for x in st])
        s.close()
    a, b = out[ddh.COARSE_ND], out[ddh.COARSE_ND_LEVELS]
    assert np.linalg.norm(a[0] - b[0]) <= 1e-9 * np.linalg.norm(b[0])
    assert abs(max(a[1]) - max(b[1])) <= 1 and max(a[2]) <= 1e-10 and max(b[2]) <= 1e-10


@pytest.mark.parametrize("name", ["uniform4_mixed_p", "multilevel"])
@pytest.mark.parametrize("chains", [1, 2, 4])
def test_nested_dissection_chains_match_oracle(name, chains):
    """The per-level solve split into 1, 2 or 4 chains over equal shares of 8 right-hand sides
    (forked streams, each chain with the level tuning of its share) solves the same systems."""
    w = _with_rhs(ND_SMALL[name](), 8)
    s = _solver(w, tol=1e-12, coarse_form=ddh.COARSE_ND_LEVELS, nd_chains=chains)
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-12)
    assert s.get_tuning(8, ddh.PREC_FP64)["nd_chains"] == chains
    ref = dd.DDSolver(dd.problem_from_workload(w), l=s.info().l).solve(tol=1e-12)
    got = u.cpu().numpy()
    for r in range(8):
        assert _rel(got[r], ref["phi_N"][r]) <= 1e-10, (name, chains, r)
    s.close()


@pytest.mark.parametrize("launch", [ddh.EDGE_LAUNCH_PER_TASK, ddh.EDGE_LAUNCH_PERSISTENT])
@pytest.mark.parametrize("prec", [ddh.PREC_FP64, ddh.PREC_MIXED_FP32])
def test_edge_pass_launch_forms_match_oracle(launch, prec):
    """Both launch forms of the Krylov-loop edge pass (one CTA per task; one persistent launch
    over the degree-sorted element list with tuned threads per row) on a mixed-degree hanging
    mesh with 8 right-hand sides."""
    w = _with_rhs(ND_SMALL["hanging_corner"](), 8)
    s = _solver(w, tol=1e-12, precision=prec, edge_launch=launch)
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-12 if prec == ddh.PREC_FP64 else 1e-10)
    assert s.get_tuning(8, prec)["edge_persistent"] == (1 if launch == ddh.EDGE_LAUNCH_PERSISTENT else 0)
    got = u.cpu().numpy()
    if prec == ddh.PREC_FP64:
        ref = dd.DDSolver(dd.problem_from_workload(w), l=s.info().l).solve(tol=1e-12)["phi_N"]
        bound = 1e-10
    else:
        ref = dd.Conforming(dd.problem_from_workload(w)).solve_direct()
        bound = 1e-8
    for r in range(8):
        assert _rel(got[r], ref[r]) <= bound, (launch, prec, r)
    s.close()


@pytest.mark.parametrize("prec", [ddh.PREC_FP64, ddh.PREC_MIXED_FP32])
def test_tuned_launch_shapes_do_not_change_the_bits(prec):
    """Every shape an autotuner picks (edge-pass launch form and threads per row, coarse-solve
    chains and right-hand sides per CTA), and the split of pass 1 into its t_T rows and its x_E
    rows on a forked stream, leave each sum in a fixed order: solves pinned to
    different shapes agree bit for bit, so the tuners' timing noise cannot change iteration
    counts."""
    w = _with_rhs(ND_SMALL["hanging_corner"](), 8)
    outs = []
    for opts in ({}, {"edge_launch": ddh.EDGE_LAUNCH_PER_TASK, "nd_chains": 1},
                 {"edge_launch": ddh.EDGE_LAUNCH_PERSISTENT, "nd_chains": 2}, {"nd_chains": 4},
                 {"edge_launch": ddh.EDGE_LAUNCH_PER_TASK, "split_pass1": 1, "nd_pdl": 0}):
        s = _solver(w, tol=1e-10, precision=prec, coarse_form=ddh.COARSE_ND_LEVELS, **opts)
        u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-10)
        outs.append((u.cpu(), [x.iterations for x in st], [x.inner_iterations for x in st]))
        s.close()
    for u, its, inner in outs[1:]:
        assert torch.equal(u, outs[0][0])
        assert its == outs[0][1] and inner == outs[0][2]


# ---------------------------------------------------------------- reduced batching workload
@pytest.fixture(scope="module")
def disk_reduced():
    w = W.disk_hanging(8, 16)
    prob = dd.problem_from_workload(w)
    return w, prob, dd.Conforming(prob).solve_direct()


def test_reduced_disk_batch_fp64(disk_reduced):
    w, prob, ref = disk_reduced
    assert w.n_elem == 244 and int(w.p.min()) >= 8 and int(w.p.max()) <= 24
    s = _solver(w, tol=1e-12)
    assert s.info().l == 3
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-12)
    got = u.cpu().numpy()
    for r in range(w.n_rhs):
        assert _rel(got[r], ref[r]) <= 1e-10, r
    assert dd.Conforming(prob).residual(got).max() <= 1e-10
    s.close()


def test_reduced_disk_batch_mixed(disk_reduced):
    w, prob, ref = disk_reduced
    s = _solver(w, tol=1e-10, precision=ddh.PREC_MIXED_FP32)
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-10)
    got = u.cpu().numpy()
    for r in range(w.n_rhs):
        assert st[r].primal_residual <= 1e-10
        assert _rel(got[r], ref[r]) <= 1e-8, r
    s.close()


# ---------------------------------------------------------------- wide element rows
@pytest.mark.parametrize("p", [20, 24, 32])
@pytest.mark.parametrize("prec", [ddh.PREC_FP64, ddh.PREC_MIXED_FP32])
@pytest.mark.parametrize("form", [ddh.LOCAL_EDGE, ddh.LOCAL_FDM])
def test_wide_rows_match_oracle(p, prec, form):
    w = W.small_uniform(3, p, 12.0, seed=9, eps_range=(1, 2), n_rhs=3)
    s = _solver(w, tol=1e-12 if prec == ddh.PREC_FP64 else 1e-10, precision=prec, local_form=form, l_override=2)
    u, st = s.solve(s.rhs_planewave(w.thetas), tol=1e-12 if prec == ddh.PREC_FP64 else 1e-10)
    ref = dd.Conforming(dd.problem_from_workload(w)).solve_direct()
    got = u.cpu().numpy()
    for r in range(w.n_rhs):
        assert _rel(got[r], ref[r]) <= (1e-10 if prec == ddh.PREC_FP64 else 1e-8), (p, prec, form, r)
    s.close()


# ---------------------------------------------------------------- one application of F and P^-1
OPS = {
    "plane_2x2": W.plane_2x2,
    "uniform4_mixed_p": ND_SMALL["uniform4_mixed_p"],
    "hanging_mixed_p": lambda: W.small_hanging(3, refine=[(1, 1)], levels=2, p=6, k=5.0, seed=1,
                                               p_range=(4, 8), eps_in=2.0),
    "hanging_corner": ND_SMALL["hanging_corner"],
    "multilevel": ND_SMALL["multilevel"],
}


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("prec", [ddh.PREC_FP64, ddh.PREC_MIXED_FP32])
def test_interface_operator_and_preconditioner_match_oracle(name, prec):
    w = OPS[name]()
    s = _solver(w, tol=1e-12)
    info = s.info()
    prob = dd.problem_from_workload(w)
    ref = dd.DDSolver(prob, l=info.l)
    assert ref.nd == info.n_dual and ref.n2 == info.n_coarse
    rng = np.random.default_rng(17)
    R = 3
    nu = rng.standard_normal((R, ref.nd)) + 1j * rng.standard_normal((R, ref.nd))
    v = torch.tensor(nu, device="cuda:0")
    Fv = s.apply_dual_operator(0, v, prec).cpu().numpy()
    Pv = s.apply_dual_operator(1, v, prec).cpu().numpy()
    tol = 1e-12 if prec == ddh.PREC_FP64 else 1e-5
    for r in range(R):
        assert _rel(Fv[r], ref.apply_F(nu[r])) <= tol, (name, "F", r)
        assert _rel(Pv[r], ref.apply_P(nu[r])) <= tol, (name, "P", r)
    s.close()
