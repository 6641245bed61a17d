"""Quadtree mesh bookkeeping for the oracle (Sec. 2.2.3-2.2.4; plain Python, test infrastructure).

Leaves (level, i, j) over a base_n x base_n grid of [0,1]^2.  Sides are numbered as the
paper's Gamma_1..Gamma_4: 1 = left (x1=-1), 2 = right (x1=+1), 3 = bottom (x2=-1),
4 = top (x2=+1).  Along a side the edge coordinate t in [-1,1] runs with x2 (sides 1, 2)
or x1 (sides 3, 4).

A *master edge* is either a boundary side, a pair of equal-level sides (conforming), or a
coarse side together with the finer sides lying on it (hanging nodes).  For a fine side on
a coarse side, the coarse coordinate is u = a t + b with a = 2^-m and b from the sub-edge
position (eq. affine_parameters); here a and b are read off the integer coordinates.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class MasterEdge:
    kind: str                      # 'boundary' | 'conforming' | 'hanging'
    elem: int                      # boundary element, conforming 'c' element (left/bottom), or coarse element
    side: int
    others: list = field(default_factory=list)   # [(elem, side, a, b)] fine / neighbour sides
    degree: int = 0                # trace degree d = min of incident element degrees


@dataclass
class Mesh:
    base_n: int
    leaves: np.ndarray
    p: np.ndarray
    maxlev: int
    box: np.ndarray                # int64 [E,4]  X0, X1, Y0, Y1 in finest units
    h: np.ndarray                  # float [E] side length
    edges: list
    side_edge: dict                # (e, side) -> (edge index, role) role in {'b','c','f'}
    vertices: dict                 # (X, Y) -> vertex id for non-hanging vertices
    hanging: set                   # set of (X, Y) hanging vertex positions

    @property
    def n_elem(self) -> int:
        return int(self.leaves.shape[0])

    def corner_xy(self, e: int, a: int, b: int):
        X0, X1, Y0, Y1 = self.box[e]
        return (X1 if a == 0 else X0, Y1 if b == 0 else Y0)


SIDE_NEIGHBOUR = {1: (-1, 0), 2: (1, 0), 3: (0, -1), 4: (0, 1)}
OPPOSITE = {1: 2, 2: 1, 3: 4, 4: 3}


def build_mesh(base_n: int, leaves: np.ndarray, p: np.ndarray) -> Mesh:
    leaves = np.asarray(leaves, dtype=np.int64)
    p = np.asarray(p, dtype=np.int64)
    E = leaves.shape[0]
    maxlev = int(leaves[:, 0].max()) if E else 0
    lookup = {(int(l), int(i), int(j)): e for e, (l, i, j) in enumerate(leaves)}
    box = np.zeros((E, 4), np.int64)
    for e, (l, i, j) in enumerate(leaves):
        s = 2 ** (maxlev - l)
        box[e] = (i * s, (i + 1) * s, j * s, (j + 1) * s)
    h = 1.0 / (base_n * 2.0 ** leaves[:, 0])

    edges: list[MasterEdge] = []
    side_edge: dict = {}
    hang_map: dict = {}            # (coarse e, side) -> edge index

    def side_range(e, side):
        X0, X1, Y0, Y1 = box[e]
        return (Y0, Y1) if side in (1, 2) else (X0, X1)

    for e in range(E):
        l, i, j = (int(v) for v in leaves[e])
        nside = base_n * 2 ** l
        for side in (1, 2, 3, 4):
            if (e, side) in side_edge:
                continue
            di, dj = SIDE_NEIGHBOUR[side]
            ni, nj = i + di, j + dj
            if ni < 0 or nj < 0 or ni >= nside or nj >= nside:
                side_edge[(e, side)] = (len(edges), 'b')
                edges.append(MasterEdge('boundary', e, side, [], int(p[e])))
                continue
            if (l, ni, nj) in lookup:
                f = lookup[(l, ni, nj)]
                # conforming: 'c' role = left/bottom element
                if side in (2, 4):
                    c, cs, fe, fs = e, side, f, OPPOSITE[side]
                else:
                    c, cs, fe, fs = f, OPPOSITE[side], e, side
                idx = len(edges)
                edges.append(MasterEdge('conforming', c, cs, [(fe, fs, 1.0, 0.0)],
                                        int(min(p[c], p[fe]))))
                side_edge[(c, cs)] = (idx, 'c')
                side_edge[(fe, fs)] = (idx, 'f')
                continue
            # coarser neighbour?
            found = None
            for m in range(1, l + 1):
                key = (l - m, ni >> m, nj >> m)
                if key in lookup:
                    found = lookup[key]
                    break
            if found is not None:
                c, cs = found, OPPOSITE[side]
                C0, C1 = side_range(c, cs)
                F0, F1 = side_range(e, side)
                a = (F1 - F0) / (C1 - C0)
                b = (F0 + F1 - C0 - C1) / (C1 - C0)
                if (c, cs) not in hang_map:
                    hang_map[(c, cs)] = len(edges)
                    edges.append(MasterEdge('hanging', c, cs, [], int(p[c])))
                idx = hang_map[(c, cs)]
                edges[idx].others.append((e, side, a, b))
                edges[idx].degree = int(min(edges[idx].degree, p[e]))
                side_edge[(e, side)] = (idx, 'f')
                side_edge[(c, cs)] = (idx, 'c')
            # else: finer neighbours, registered when the fine elements are visited

    # vertices: hanging = strictly inside a hanging edge's coarse side
    hanging = set()
    for ed in edges:
        if ed.kind != 'hanging':
            continue
        C0, C1 = side_range(ed.elem, ed.side)
        for (f, fs, a, b) in ed.others:
            F0, F1 = side_range(f, fs)
            for t in (F0, F1):
                if C0 < t < C1:
                    X0, X1, Y0, Y1 = box[ed.elem]
                    if ed.side == 1:
                        hanging.add((X0, t))
                    elif ed.side == 2:
                        hanging.add((X1, t))
                    elif ed.side == 3:
                        hanging.add((t, Y0))
                    else:
                        hanging.add((t, Y1))
    vertices: dict = {}
    for e in range(E):
        X0, X1, Y0, Y1 = box[e]
        for xy in ((X1, Y1), (X0, Y1), (X1, Y0), (X0, Y0)):
            if xy not in hanging and xy not in vertices:
                vertices[xy] = len(vertices)
    return Mesh(base_n, leaves, p, maxlev, box, h, edges, side_edge, vertices, hanging)


def side_slot(p: int, side: int, m: int) -> int:
    """Flat tilde index (x1 index fastest) of trace coefficient m on a side.
    Along a side the trace is row a=1 (side 1), row a=0 (side 2), column b=1 (side 3)
    or column b=0 (side 4) of Phi~; m = 0 is the t=+1 end, m = 1 the t=-1 end."""
    n = p + 1
    if side == 1:
        return 1 + n * m
    if side == 2:
        return n * m
    if side == 3:
        return m + n
    return m


def side_corners(side: int):
    """(a, b) corner indices of trace entries m=0 (t=+1 end) and m=1 (t=-1 end)."""
    return {1: ((1, 0), (1, 1)), 2: ((0, 0), (0, 1)),
            3: ((0, 1), (1, 1)), 4: ((0, 0), (1, 0))}[side]


def element_neighbours(mesh: Mesh, e: int) -> list:
    """Elements sharing a side with e, side by side (1..4); across a coarse side of a hanging
    edge, every fine element on it in the edge's order; across a fine side, the coarse element."""
    out = []
    for side in (1, 2, 3, 4):
        ei, role = mesh.side_edge[(e, side)]
        ed = mesh.edges[ei]
        if ed.kind == 'boundary':
            continue
        if role == 'c':
            out.extend(f for (f, _fs, _a, _b) in ed.others)
        else:
            out.append(ed.elem)
    return out


def weak_two_colouring(mesh: Mesh) -> np.ndarray:
    """Signs +1 / -1 per element from a breadth-first spanning tree of the element adjacency
    graph started at element 0: even tree levels +1, odd levels -1 (Sec. 2.3.4, the weak
    2-colouring of the Robin-modified local problems).  Every element with a neighbour then has
    a neighbour of the opposite sign (its parent or a child in the tree)."""
    E = mesh.n_elem
    level = np.full(E, -1, np.int64)
    for root in range(E):
        if level[root] >= 0:
            continue
        level[root] = 0
        queue = [root]
        head = 0
        while head < len(queue):
            e = queue[head]
            head += 1
            for f in element_neighbours(mesh, e):
                if level[f] < 0:
                    level[f] = level[e] + 1
                    queue.append(f)
    return np.where(level % 2 == 0, 1, -1).astype(np.int64)
