"""Continuity constraints, unknown types and the nullspace basis (Sec. 2.2.4, 2.3.1-2.3.2).

* ``paper_constraints``: the global constraint matrix C of eq. final_constraint,
  (L_c^f)^T C_j^c phi_c - C_i^f phi_f = 0 with zero padding to degree max(p_c, p_f), one row
  per moment m = 0..max(p_c,p_f) on every conforming pair and every fine sub-edge,
  on the element-local N-basis coefficients.  Redundant rows are kept (the direct solve
  takes the null space numerically).
* ``classify``: the reading of Algorithm 1 used by the build.  On every master edge the
  trace degree d is the minimum of the incident element degrees; trace coefficients above d
  are zero (the padded rows with m > d are enforced directly, i.e. belong to C_p).  C_p
  holds moments m <= l (vertex continuity and the first l-1 bubble moments), C_d holds
  l < m <= d.  Type-2 (coarse) unknowns: one per non-hanging vertex, bubbles 2..min(l,d)
  of conforming and boundary edges, all bubbles 2..d of the coarse side of a hanging edge.
  Type-1: interior bubbles and edge bubbles l < m <= d not on a coarse hanging side.
  Fine-side vertex and low-bubble coefficients are slaved to the coarse trace through
  N~(ax+b) = L~ N~(x).  Z is the basis of null(C_p) dual to the kept unknowns
  (Z_1 = identity on type-1 slots).  With l = None every constraint is in C_p and Z is the
  conforming (globally assembled) basis.
* dual rows use unit weight on the interpolatory-basis bubble coefficients:
  sum_k L~_{k m} t_c[k] - t_f[m]  (a constant 1/sqrt(2) rescaling of the paper's rows).

Pins (tests/test_oracle_dd.py): C_p Z = 0 and rank(Z) = dim null(C_p) against an SVD of
the paper's C_p; the dual rows equal the paper's C_d rows / sqrt(2) on range(Z); the
conforming basis spans null(C).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import legendre as lg
from .element import side_vector
from .mesh import Mesh, side_slot, side_corners


def element_offsets(mesh: Mesh) -> np.ndarray:
    sizes = (mesh.p + 1) ** 2
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def paper_constraints(mesh: Mesh):
    """Rows of eq. final_constraint on the N-basis coefficients.
    Returns (C sparse [rows, n_local], tags list of (edge index, sub index, m))."""
    off = element_offsets(mesh)
    rows, cols, vals, tags = [], [], [], []
    r = 0
    for ei, ed in enumerate(mesh.edges):
        if ed.kind == 'boundary':
            continue
        c, cs = ed.elem, ed.side
        pc = int(mesh.p[c])
        for si, (f, fs, a, b) in enumerate(ed.others):
            pf = int(mesh.p[f])
            L = max(pc, pf)
            Lcf = lg.affine_L_N(L, a, b) if (a != 1.0 or b != 0.0) else np.eye(L + 1)
            wc = side_vector(pc, cs)
            wf = side_vector(pf, fs)
            for m in range(L + 1):
                # (L^T C_c phi_c)[m] = sum_k L[k,m] (C_c phi_c)[k]
                for k in range(min(pc, L) + 1):
                    coef = Lcf[k, m]
                    if coef == 0.0:
                        continue
                    for t in (0, 1):
                        if wc[t] == 0.0:
                            continue
                        # side 1,2: (C phi)[k] = sum_a w_a Phi[a,k]; side 3,4: sum_b w_b Phi[k,b]
                        idx = (t + (pc + 1) * k) if cs in (1, 2) else (k + (pc + 1) * t)
                        rows.append(r); cols.append(off[c] + idx); vals.append(coef * wc[t])
                if m <= pf:
                    for t in (0, 1):
                        idx = (t + (pf + 1) * m) if fs in (1, 2) else (m + (pf + 1) * t)
                        rows.append(r); cols.append(off[f] + idx); vals.append(-wf[t])
                tags.append((ei, si, m))
                r += 1
    C = sp.csr_matrix((vals, (rows, cols)), shape=(r, int(off[-1])))
    return C, tags


def dispersion_l(mesh: Mesh, k: float, eps: np.ndarray) -> int:
    """Eq. dispersion_criterion: l > (kh + (kh)^(1/3) - 1)/2 with kh = max_e k sqrt(eps_e) h_e;
    l is the smallest integer strictly above the bound, and at least 1."""
    kh = float(np.max(k * np.sqrt(eps) * mesh.h))
    rb = 0.5 * (kh + kh ** (1.0 / 3.0) - 1.0)
    l = int(np.floor(rb)) + 1
    return max(1, l)


@dataclass
class Split:
    l: int | None
    n1: int
    n2: int
    Z: sp.csr_matrix                 # [n_local_tilde, n1 + n2], columns: type-1 then type-2
    t1_of_elem: list                 # per element: array of tilde flat indices (type-1 slots)
    t1_edge_mask: list               # per element: bool array, True for edge (E1) slots
    t1_offset: np.ndarray            # [E+1] column offsets of type-1 unknowns per element
    Cd: sp.csr_matrix                # dual rows on the tilde slots (unit scaling)
    dual_tags: list                  # (edge index, sub index, m)
    off: np.ndarray                  # element offsets in the local vector


def classify(mesh: Mesh, l: int | None) -> Split:
    """Unknown types, Z and the dual rows for primal-constraint count l (None = all)."""
    LINF = 10 ** 9 if l is None else l
    off = element_offsets(mesh)
    E = mesh.n_elem
    # ---- coarse (type-2) dofs
    n_v = len(mesh.vertices)
    edge_dof = {}
    nxt = n_v
    for ei, ed in enumerate(mesh.edges):
        top = ed.degree if ed.kind == 'hanging' else min(LINF, ed.degree)
        for m in range(2, top + 1):
            edge_dof[(ei, m)] = nxt
            nxt += 1
    n2 = nxt

    Lt_cache = {}

    def Lt(n, a, b):
        key = (n, a, b)
        if key not in Lt_cache:
            Lt_cache[key] = lg.affine_L_tilde(n, a, b)
        return Lt_cache[key]

    def sub_entry(ei, e, side):
        for ent in mesh.edges[ei].others:
            if ent[0] == e and ent[1] == side:
                return ent
        raise KeyError((ei, e, side))

    memo = {}

    def corner_value(e, a, b):
        key = (e, a, b)
        if key in memo:
            return memo[key]
        xy = mesh.corner_xy(e, a, b)
        if xy in mesh.vertices:
            out = {mesh.vertices[xy]: 1.0}
        else:
            out = None
            for side in ((2 if a == 0 else 1), (4 if b == 0 else 3)):
                ei, role = mesh.side_edge[(e, side)]
                ed = mesh.edges[ei]
                if ed.kind == 'hanging' and role == 'f':
                    c0, c1 = side_corners(side)
                    m = 0 if c0 == (a, b) else 1
                    out = slaved(ei, e, side, m)
                    break
            assert out is not None, "hanging corner without a fine side"
        memo[key] = out
        return out

    def slaved(ei, f, fs, m):
        ed = mesh.edges[ei]
        _, _, a, b = sub_entry(ei, f, fs)
        c, cs = ed.elem, ed.side
        n = max(int(mesh.p[c]), int(mesh.p[f]), m)
        T = Lt(n, a, b)
        out: dict = {}
        cc = side_corners(cs)
        for k in (0, 1):
            w = T[k, m]
            if w != 0.0:
                for col, v in corner_value(c, *cc[k]).items():
                    out[col] = out.get(col, 0.0) + w * v
        for k in range(2, ed.degree + 1):
            w = T[k, m]
            if w != 0.0:
                col = edge_dof[(ei, k)]
                out[col] = out.get(col, 0.0) + w
        return out

    # ---- per-element slot classification
    zrows, zcols, zvals = [], [], []
    t1_of_elem, t1_edge_mask = [], []
    t1_offset = np.zeros(E + 1, np.int64)
    t2_entries = []                                  # (global row, {col2: w})
    n1 = 0
    for e in range(E):
        p = int(mesh.p[e])
        n = p + 1
        t1, mask = [], []
        # interior first, then edge slots in side order 1..4
        for bb in range(2, n):
            for aa in range(2, n):
                t1.append(aa + n * bb); mask.append(False)
        for side in (1, 2, 3, 4):
            ei, role = mesh.side_edge[(e, side)]
            ed = mesh.edges[ei]
            for m in range(2, n):
                slot = side_slot(p, side, m)
                if m > ed.degree:
                    continue                        # zero (trace degree)
                if ed.kind == 'hanging' and role == 'c':
                    t2_entries.append((off[e] + slot, {edge_dof[(ei, m)]: 1.0}))
                elif m <= LINF:
                    if ed.kind == 'hanging':
                        t2_entries.append((off[e] + slot, slaved(ei, e, side, m)))
                    else:
                        t2_entries.append((off[e] + slot, {edge_dof[(ei, m)]: 1.0}))
                else:
                    t1.append(slot); mask.append(True)
        for (aa, bb) in ((0, 0), (1, 0), (0, 1), (1, 1)):
            t2_entries.append((off[e] + aa + n * bb, corner_value(e, aa, bb)))
        t1 = np.asarray(t1, np.int64)
        for jj, s in enumerate(t1):
            zrows.append(off[e] + s); zcols.append(n1 + jj); zvals.append(1.0)
        t1_of_elem.append(t1)
        t1_edge_mask.append(np.asarray(mask, bool))
        n1 += len(t1)
        t1_offset[e + 1] = n1
    for row, expr in t2_entries:
        for col, w in expr.items():
            zrows.append(row); zcols.append(n1 + col); zvals.append(w)
    Z = sp.csr_matrix((zvals, (zrows, zcols)), shape=(int(off[-1]), n1 + n2))

    # ---- dual rows (tilde slots, unit scaling)
    drows, dcols, dvals, dtags = [], [], [], []
    r = 0
    if l is not None:
        for ei, ed in enumerate(mesh.edges):
            if ed.kind == 'boundary':
                continue
            c, cs = ed.elem, ed.side
            pc = int(mesh.p[c])
            for si, (f, fs, a, b) in enumerate(ed.others):
                pf = int(mesh.p[f])
                T = None if ed.kind == 'conforming' else Lt(max(pc, pf), a, b)
                for m in range(l + 1, ed.degree + 1):
                    if T is None:
                        drows.append(r); dcols.append(off[c] + side_slot(pc, cs, m)); dvals.append(1.0)
                    else:
                        for k in range(m, ed.degree + 1):
                            drows.append(r); dcols.append(off[c] + side_slot(pc, cs, k))
                            dvals.append(T[k, m])
                    drows.append(r); dcols.append(off[f] + side_slot(pf, fs, m)); dvals.append(-1.0)
                    dtags.append((ei, si, m))
                    r += 1
    Cd = sp.csr_matrix((dvals, (drows, dcols)), shape=(r, int(off[-1])))
    return Split(l, n1, n2, Z, t1_of_elem, t1_edge_mask, t1_offset, Cd, dtags, off)


def B_z(mesh: Mesh) -> sp.csr_matrix:
    """Block-diagonal B (x) B over all elements (phi~ = B_z phi)."""
    blocks = []
    for p in mesh.p:
        B = lg.B_matrix(int(p))
        blocks.append(sp.csr_matrix(np.kron(B, B)))
    return sp.block_diag(blocks, format="csr")


def split_rows(tags, mesh: Mesh, l: int):
    """Row masks of the paper's C: C_p (m <= l or m > d) and C_d (l < m <= d)."""
    isp = []
    for (ei, si, m) in tags:
        d = mesh.edges[ei].degree
        isp.append(m <= l or m > d)
    isp = np.asarray(isp, bool)
    return isp, ~isp
