"""Seeded synthetic workloads for the dual-primal DD spectral-element Helmholtz solver.

This module is shared by the CPU oracle and the GPU library's tests and bench. It holds
only problem *inputs* (meshes, degrees, permittivities, wavenumbers, incident angles,
observation points); none of the method's arithmetic lives here.

A mesh is a list of quadtree leaves over a base grid of ``base_n x base_n`` squares
covering [0,1]^2.  Leaf ``(level, i, j)`` is the square of side
``h = 1 / (base_n * 2**level)`` with lower-left corner ``(i*h, j*h)``.

The five named workloads are:

* ``plane_2x2``    -- 2x2 squares, p=8, k=10, eps=1, theta=pi/7, one RHS.
* ``plane_16x16``  -- 16x16 squares, p=16, k=100, eps=1, theta=pi/7, one RHS.
* ``disk_hanging`` -- 32x32 base grid, base cells whose centre lies in the disk
  r<0.25 about (0.5,0.5) refined two levels (hanging nodes, 3 per coarse edge);
  eps=4 for leaves centred in the disk, else 1; k=150; p ~ U{8..24} per leaf
  (seed 3); 64 incident angles ~ U[0, 2pi) (seed 33).
* ``random_eps_64`` -- 64x64 squares, p=20, k=400, eps ~ U[1,2] i.i.d. (seed 4),
  8 angles ~ U[0, 2pi) (seed 44).
* ``lens_48``      -- 48x48 squares, p=16, k=200, eps ~ U[1,4] (seed 5), theta=0,
  32 observation points on x=0.9, y in [0.4, 0.6]; 16 finite-difference
  parameter indices (seed 55).

``poisson_table2(p, N, l)`` gives the Poisson test problem of the paper's Table 2 (rho_ij =
10^((i-j)/4) on sqrt(N) x sqrt(N) squares, zero Dirichlet data, loads ~ U(0,1), seed 7).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    base_n: int
    leaves: np.ndarray          # int32 [E,3] (level, i, j)
    p: np.ndarray               # int32 [E]
    eps: np.ndarray             # float64 [E]
    k: float
    thetas: np.ndarray          # float64 [R] incident angles of the plane waves
    points: np.ndarray | None = None       # float64 [P,2] observation points
    fd_index: np.ndarray | None = None     # int64 [16] parameters checked by finite differences
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return int(self.leaves.shape[0])

    @property
    def n_rhs(self) -> int:
        return int(self.thetas.shape[0])


def uniform_leaves(n: int) -> np.ndarray:
    """Leaves of a uniform n x n grid, element index e = i + n*j (x fastest)."""
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([np.zeros(n * n, np.int32), ii.ravel().astype(np.int32),
                     jj.ravel().astype(np.int32)], axis=1).astype(np.int32)


def disk_leaves(base_n: int = 32, radius: float = 0.25, levels: int = 2,
                centre=(0.5, 0.5)) -> np.ndarray:
    """Base grid with every base cell whose centre lies inside the disk refined
    ``levels`` times (4**levels children).  Leaves are ordered by base cell
    (x fastest), children of a refined cell in (j, i) order, x fastest."""
    out = []
    cx, cy = centre
    m = 2 ** levels
    for bj in range(base_n):
        for bi in range(base_n):
            xc = (bi + 0.5) / base_n
            yc = (bj + 0.5) / base_n
            if (xc - cx) ** 2 + (yc - cy) ** 2 < radius ** 2:
                for sj in range(m):
                    for si in range(m):
                        out.append((levels, bi * m + si, bj * m + sj))
            else:
                out.append((0, bi, bj))
    return np.asarray(out, np.int32)


def leaf_centres(base_n: int, leaves: np.ndarray) -> np.ndarray:
    lev, i, j = leaves[:, 0], leaves[:, 1], leaves[:, 2]
    h = 1.0 / (base_n * 2.0 ** lev)
    return np.stack([(i + 0.5) * h, (j + 0.5) * h], axis=1)


def leaf_sizes(base_n: int, leaves: np.ndarray) -> np.ndarray:
    return 1.0 / (base_n * 2.0 ** leaves[:, 0])


def plane_2x2() -> Workload:
    lv = uniform_leaves(2)
    E = lv.shape[0]
    return Workload("plane_2x2", 2, lv, np.full(E, 8, np.int32), np.ones(E), 10.0,
                    np.array([math.pi / 7]))


def plane_16x16() -> Workload:
    lv = uniform_leaves(16)
    E = lv.shape[0]
    return Workload("plane_16x16", 16, lv, np.full(E, 16, np.int32), np.ones(E), 100.0,
                    np.array([math.pi / 7]))


def disk_hanging(base_n: int = 32, n_rhs: int = 64) -> Workload:
    """The batching workload on a base_n x base_n grid (32 by default).  Smaller grids keep the
    refinement rule, the degree and angle distributions and the element k h (k = 150 base_n/32)."""
    lv = disk_leaves(base_n, 0.25, 2)
    E = lv.shape[0]
    c = leaf_centres(base_n, lv)
    inside = (c[:, 0] - 0.5) ** 2 + (c[:, 1] - 0.5) ** 2 < 0.25 ** 2
    eps = np.where(inside, 4.0, 1.0)
    p = np.random.default_rng(3).integers(8, 25, size=E).astype(np.int32)
    thetas = np.random.default_rng(33).uniform(0.0, 2.0 * math.pi, size=n_rhs)
    name = "disk_hanging" if (base_n, n_rhs) == (32, 64) else f"disk_hanging_{base_n}_r{n_rhs}"
    return Workload(name, base_n, lv, p, eps, 150.0 * base_n / 32, thetas)


def random_eps_64() -> Workload:
    lv = uniform_leaves(64)
    E = lv.shape[0]
    eps = np.random.default_rng(4).uniform(1.0, 2.0, size=E)
    thetas = np.random.default_rng(44).uniform(0.0, 2.0 * math.pi, size=8)
    return Workload("random_eps_64", 64, lv, np.full(E, 20, np.int32), eps, 400.0, thetas)


def lens_48() -> Workload:
    lv = uniform_leaves(48)
    E = lv.shape[0]
    eps = np.random.default_rng(5).uniform(1.0, 4.0, size=E)
    pts = np.stack([np.full(32, 0.9), np.linspace(0.4, 0.6, 32)], axis=1)
    fd = np.random.default_rng(55).choice(E, size=16, replace=False)
    return Workload("lens_48", 48, lv, np.full(E, 16, np.int32), eps, 200.0,
                    np.array([0.0]), points=pts, fd_index=fd)


def corner_block(w: Workload, n: int, n_rhs: int = 1) -> Workload:
    """The n x n block of elements in the lower-left corner of a uniform workload, as a problem
    of its own on [0, n/base_n]^2 rescaled to the unit square by keeping the element size: the
    same degree, wavenumber and permittivity draws of those elements, and the first n_rhs angles.
    (A bounded sample of a large uniform workload for the CPU oracle.)"""
    assert int(w.leaves[:, 0].max()) == 0, "uniform workloads only"
    sel = (w.leaves[:, 1] < n) & (w.leaves[:, 2] < n)
    lv = w.leaves[sel]
    # same element size h = 1/base_n on a domain of n x n elements: wavenumber scaled by n/base_n
    scale = n / w.base_n
    return Workload(f"{w.name}_corner{n}", n, lv.copy(), w.p[sel].copy(), w.eps[sel].copy(), w.k * scale,
                    w.thetas[:n_rhs].copy())


@dataclass
class PoissonWorkload:
    """The Poisson test problem of Sec. 3.1 (Table 2): N = 4^n squares of degree p on the unit
    square, rho_ij = 10^((i - j)/4) on element (i, j), zero Dirichlet data, l primal moments per
    edge, and load vectors with entries ~ U(0, 1) (seeded) in the N basis."""
    name: str
    base_n: int
    leaves: np.ndarray
    p: np.ndarray
    rho: np.ndarray
    l: int
    loads: np.ndarray           # float64 [R, n_local]


def poisson_table2(p: int, N: int, l: int, n_rhs: int = 1, seed: int = 7) -> PoissonWorkload:
    m = int(round(math.sqrt(N)))
    leaves = uniform_leaves(m)
    rho = 10.0 ** ((leaves[:, 1] - leaves[:, 2]) / 4.0)
    n_local = m * m * (p + 1) ** 2
    loads = np.random.default_rng(seed).uniform(0.0, 1.0, size=(n_rhs, n_local))
    return PoissonWorkload(f"poisson_p{p}_N{N}_l{l}", m, leaves, np.full(m * m, p, np.int32), rho, l, loads)


WORKLOADS = {
    "plane_2x2": plane_2x2,
    "plane_16x16": plane_16x16,
    "disk_hanging": disk_hanging,
    "random_eps_64": random_eps_64,
    "lens_48": lens_48,
}


# ---------------------------------------------------------------- small test meshes

def small_uniform(n: int, p: int, k: float, seed: int | None = None, eps_range=(1.0, 1.0),
                  n_rhs: int = 1, p_range: tuple[int, int] | None = None) -> Workload:
    """n x n uniform mesh; eps ~ U[eps_range] and p ~ U{p_range} when given (seeded)."""
    lv = uniform_leaves(n)
    E = lv.shape[0]
    rng = np.random.default_rng(seed)
    lo, hi = eps_range
    eps = rng.uniform(lo, hi, size=E) if hi > lo else np.full(E, lo)
    if p_range is None:
        pp = np.full(E, p, np.int32)
    else:
        pp = rng.integers(p_range[0], p_range[1] + 1, size=E).astype(np.int32)
    thetas = (rng.uniform(0.0, 2.0 * math.pi, size=n_rhs) if n_rhs > 1
              else np.array([math.pi / 7]))
    return Workload(f"uniform{n}_p{p}", n, lv, pp, eps, k, thetas)


def small_hanging(base_n: int = 4, refine=((1, 1),), levels: int = 2, p: int = 8,
                  k: float = 6.0, seed: int | None = None, p_range=None, n_rhs: int = 1,
                  eps_in: float = 1.0) -> Workload:
    """base_n x base_n grid with the listed base cells refined ``levels`` times."""
    refine = set(tuple(r) for r in refine)
    m = 2 ** levels
    out = []
    for bj in range(base_n):
        for bi in range(base_n):
            if (bi, bj) in refine:
                for sj in range(m):
                    for si in range(m):
                        out.append((levels, bi * m + si, bj * m + sj))
            else:
                out.append((0, bi, bj))
    lv = np.asarray(out, np.int32)
    E = lv.shape[0]
    rng = np.random.default_rng(seed)
    if p_range is None:
        pp = np.full(E, p, np.int32)
    else:
        pp = rng.integers(p_range[0], p_range[1] + 1, size=E).astype(np.int32)
    eps = np.where(lv[:, 0] > 0, eps_in, 1.0)
    thetas = (rng.uniform(0.0, 2.0 * math.pi, size=n_rhs) if n_rhs > 1
              else np.array([math.pi / 7]))
    return Workload(f"hanging{base_n}", base_n, lv, pp, eps.astype(float), k, thetas)


def multilevel_hanging(p: int = 6, k: float = 4.0) -> Workload:
    """A 2x2 base grid where cell (0,0) is refined once and one of its children once more:
    leaves on levels 0, 1 and 2 (hanging nodes whose coarse side ends on level-1 corners)."""
    out = [(0, 1, 0), (0, 0, 1), (0, 1, 1)]
    # cell (0,0) -> level-1 children (0,0),(1,0),(0,1),(1,1); child (1,1) refined again
    for (si, sj) in [(0, 0), (1, 0), (0, 1)]:
        out.append((1, si, sj))
    for (si, sj) in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        out.append((2, 2 + si, 2 + sj))
    lv = np.asarray(out, np.int32)
    E = lv.shape[0]
    return Workload("multilevel", 2, lv, np.full(E, p, np.int32), np.ones(E), k,
                    np.array([math.pi / 7]))
