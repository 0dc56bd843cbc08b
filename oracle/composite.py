"""Geometric assembly of the composite leaf-cell system -- TEST INFRASTRUCTURE ONLY.

This is the plain definition of what Afivo's FAS multigrid converges to
(arXiv:1701.04329, Sec. 3.2-3.3), written without any box connectivity: every
leaf cell is addressed by (level, global cell index), and for each of its 2D
faces the value across the face is found by dictionary lookups:

* a leaf cell of the same level: its value;
* a refined cell of the same level: the mean of the 2^D fine cells under it
  (restriction by averaging, Sec. 2.5 -- at an FAS fixed point the coarse
  value equals the restriction of the fine values);
* outside the domain: the Dirichlet ghost 2 b - u_i (b the value at the face
  centre), or the Neumann ghost u_i + h b (b the outward normal derivative);
  across a periodic side the lookup wraps around to the opposite side;
* a coarser leaf cell (refinement boundary): the default conservative
  two-point ghost of Sec. 3.3 (2D: u_H/2 + u_i - (u_t + u_n)/4; 3D:
  u_H/2 + 5/4 u_i - (u_n + u_t1 + u_t2)/4).

Each leaf equation is (sum_faces g_f - 2D u_i) / h_i^2 = rho_i.  Returns the
sparse K (leaf x leaf) and B (leaf x boundary face) with A(u) = K u + B b.
"""
import numpy as np
import scipy.sparse as sp


def assemble(dim, box_n, level, idx, children, bc_types=None, roots=None):
    """level/idx/children: canonical box arrays (export format); bc_types: per
    domain side (-x,+x,-y,+y[,-z,+z]) 0 = Dirichlet, 1 = Neumann, 2 = periodic
    (default all 0); roots: root boxes per axis (default one)."""
    D, N = dim, box_n
    nr = list(roots) if roots is not None else [1] * D
    bct = list(bc_types) if bc_types is not None else [0] * (2 * D)
    periodic = [bct[2 * a] == 2 for a in range(D)]
    nbox = len(level)
    is_leaf = children[:, 0] < 0
    leaf_ids = np.nonzero(is_leaf)[0]
    ncell = N ** D
    # cell offsets, lexicographic with x fastest
    offs = np.array([[(c // N ** a) % N for a in range(D)] for c in range(ncell)])
    leaf_cell = {}
    for li, b in enumerate(leaf_ids):
        base = (idx[b] - 1) * N
        for c in range(ncell):
            leaf_cell[(int(level[b]),) + tuple(int(v) for v in base + offs[c])] = li * ncell + c
    refined_cell = set()
    for b in range(nbox):
        if not is_leaf[b]:
            base = (idx[b] - 1) * N
            for c in range(ncell):
                refined_cell.add((int(level[b]),) + tuple(int(v) for v in base + offs[c]))

    rows, cols, vals = [], [], []
    brow, bcol, bval = [], [], []
    nface = 0
    for li, b in enumerate(leaf_ids):
        l = int(level[b])
        h = 1.0 / (N * 2 ** (l - 1))
        ih2 = 1.0 / (h * h)
        ncells = [nr[a] * N * 2 ** (l - 1) for a in range(D)]  # cells per axis at this level
        # boundary faces of this box, in side order
        face_base = {}
        for s in range(2 * D):
            a, hi = s // 2, s % 2
            if periodic[a]:
                continue
            if (hi == 0 and idx[b][a] == 1) or (hi == 1 and idx[b][a] == nr[a] * 2 ** (l - 1)):
                face_base[s] = nface
                nface += N ** (D - 1)
        base = (idx[b] - 1) * N
        for c in range(ncell):
            g = base + offs[c]
            me = li * ncell + c
            rows.append(me); cols.append(me); vals.append(-2.0 * D * ih2)
            for s in range(2 * D):
                a, sgn = s // 2, (1 if s % 2 else -1)
                q = g.copy()
                q[a] += sgn
                if periodic[a]:
                    q[a] %= ncells[a]
                if q[a] < 0 or q[a] >= ncells[a]:
                    neumann = bct[s] == 1
                    rows.append(me); cols.append(me); vals.append(ih2 if neumann else -ih2)
                    tang = [t for t in range(D) if t != a]
                    loc = offs[c]
                    f = loc[tang[0]] + (N * loc[tang[1]] if D == 3 else 0)
                    brow.append(me); bcol.append(face_base[s] + f); bval.append(h * ih2 if neumann else 2.0 * ih2)
                    continue
                key = (l,) + tuple(int(v) for v in q)
                if key in leaf_cell:
                    rows.append(me); cols.append(leaf_cell[key]); vals.append(ih2)
                    continue
                if key in refined_cell:
                    for bits in range(2 ** D):
                        fk = (l + 1,) + tuple(int(2 * q[e] + ((bits >> e) & 1)) for e in range(D))
                        rows.append(me); cols.append(leaf_cell[fk]); vals.append(ih2 / 2 ** D)
                    continue
                ck = (l - 1,) + tuple(int(v) // 2 for v in q)
                rows.append(me); cols.append(leaf_cell[ck]); vals.append(0.5 * ih2)
                rows.append(me); cols.append(me); vals.append((1.0 if D == 2 else 1.25) * ih2)
                n2 = g.copy()
                n2[a] -= sgn
                rows.append(me); cols.append(leaf_cell[(l,) + tuple(int(v) for v in n2)]); vals.append(-0.25 * ih2)
                for t in range(D):
                    if t == a:
                        continue
                    pt = g.copy()
                    pt[t] ^= 1
                    rows.append(me); cols.append(leaf_cell[(l,) + tuple(int(v) for v in pt)]); vals.append(-0.25 * ih2)
    n = len(leaf_ids) * ncell
    K = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    B = sp.csr_matrix((bval, (brow, bcol)), shape=(n, nface))
    return K, B


def cell_volumes(dim, box_n, level, children):
    leaf_ids = np.nonzero(children[:, 0] < 0)[0]
    h = 1.0 / (box_n * 2.0 ** (level[leaf_ids] - 1))
    return np.repeat(h ** dim, box_n ** dim)


def face_areas(dim, box_n, level, idx, children, bc_types=None, roots=None):
    """h^(D-1) for each boundary face, canonical face order."""
    bct = list(bc_types) if bc_types is not None else [0] * (2 * dim)
    nr = list(roots) if roots is not None else [1] * dim
    out = []
    for b in np.nonzero(children[:, 0] < 0)[0]:
        l = int(level[b])
        h = 1.0 / (box_n * 2 ** (l - 1))
        for s in range(2 * dim):
            a, hi = s // 2, s % 2
            if bct[2 * a] == 2:
                continue
            if (hi == 0 and idx[b][a] == 1) or (hi == 1 and idx[b][a] == nr[a] * 2 ** (l - 1)):
                out.extend([h ** (dim - 1)] * box_n ** (dim - 1))
    return np.array(out)


def assemble_var(dim, box_n, level, idx, children, eps, op=1, bc_types=None, roots=None):
    """The composite system of div(eps grad u) = rho (Sec. 3.4-3.5): as
    `assemble`, with every face term multiplied by the face coefficient c_f =
    2 e_i e_n / (e_i + e_n), e_i the cell's coefficient and e_n the one across
    the face: a same-level leaf's, the mean of the 2^D children of a refined
    cell, the coarse leaf cell's across a refinement boundary, the cell's own
    at the domain boundary.  op = 2 (2D, r = x): x-faces also carry r_face /
    r_cell, and the value (and coefficient) of a refined cell is the mean of
    its children weighted by their volumes (r at their centres).  Each leaf equation is sum_f c_f (g_f - u_i) / h_i^2 = rho_i.
    eps: one value per leaf cell, canonical order."""
    D, N = dim, box_n
    nr = list(roots) if roots is not None else [1] * D
    bct = list(bc_types) if bc_types is not None else [0] * (2 * D)
    periodic = [bct[2 * a] == 2 for a in range(D)]
    is_leaf = children[:, 0] < 0
    leaf_ids = np.nonzero(is_leaf)[0]
    ncell = N ** D
    offs = np.array([[(c // N ** a) % N for a in range(D)] for c in range(ncell)])
    leaf_cell = {}
    for li, b in enumerate(leaf_ids):
        base = (idx[b] - 1) * N
        for c in range(ncell):
            leaf_cell[(int(level[b]),) + tuple(int(v) for v in base + offs[c])] = li * ncell + c
    refined_cell = set()
    for b in range(len(level)):
        if not is_leaf[b]:
            base = (idx[b] - 1) * N
            for c in range(ncell):
                refined_cell.add((int(level[b]),) + tuple(int(v) for v in base + offs[c]))

    def hmean(a, b):
        return 2.0 * a * b / (a + b)

    rows, cols, vals = [], [], []
    brow, bcol, bval = [], [], []
    nface = 0
    for li, b in enumerate(leaf_ids):
        l = int(level[b])
        h = 1.0 / (N * 2 ** (l - 1))
        ih2 = 1.0 / (h * h)
        ncells = [nr[a] * N * 2 ** (l - 1) for a in range(D)]
        face_base = {}
        for s in range(2 * D):
            a, hi = s // 2, s % 2
            if periodic[a]:
                continue
            if (hi == 0 and idx[b][a] == 1) or (hi == 1 and idx[b][a] == nr[a] * 2 ** (l - 1)):
                face_base[s] = nface
                nface += N ** (D - 1)
        base = (idx[b] - 1) * N
        for c in range(ncell):
            g = base + offs[c]
            me = li * ncell + c
            ei = eps[me]
            for s in range(2 * D):
                a, sgn = s // 2, (1 if s % 2 else -1)
                geo = 1.0
                if op == 2 and a == 0:
                    geo = (g[0] + (1.0 if sgn > 0 else 0.0)) / (g[0] + 0.5)   # r_face / r_cell
                q = g.copy()
                q[a] += sgn
                if periodic[a]:
                    q[a] %= ncells[a]
                if q[a] < 0 or q[a] >= ncells[a]:
                    cf = hmean(ei, ei) * geo
                    neumann = bct[s] == 1
                    rows.append(me); cols.append(me); vals.append(0.0 if neumann else -2.0 * cf * ih2)
                    tang = [t for t in range(D) if t != a]
                    loc = offs[c]
                    f = loc[tang[0]] + (N * loc[tang[1]] if D == 3 else 0)
                    brow.append(me); bcol.append(face_base[s] + f)
                    bval.append(cf * h * ih2 if neumann else 2.0 * cf * ih2)
                    continue
                key = (l,) + tuple(int(v) for v in q)
                if key in leaf_cell:
                    cf = hmean(ei, eps[leaf_cell[key]]) * geo
                    rows.append(me); cols.append(leaf_cell[key]); vals.append(cf * ih2)
                    rows.append(me); cols.append(me); vals.append(-cf * ih2)
                    continue
                if key in refined_cell:
                    kids = [leaf_cell[(l + 1,) + tuple(int(2 * q[e] + ((bits >> e) & 1)) for e in range(D))]
                            for bits in range(2 ** D)]
                    # the refined cell's value: the mean of its children, weighted by their
                    # volumes in (r,z) (r at the child centres), plain otherwise
                    if op == 2:
                        wk = [2 * q[0] + (bits & 1) + 0.5 for bits in range(2 ** D)]
                    else:
                        wk = [1.0] * 2 ** D
                    wk = [w / sum(wk) for w in wk]
                    cf = hmean(ei, sum(w * eps[k] for w, k in zip(wk, kids))) * geo
                    for w, k in zip(wk, kids):
                        rows.append(me); cols.append(k); vals.append(cf * ih2 * w)
                    rows.append(me); cols.append(me); vals.append(-cf * ih2)
                    continue
                ck = leaf_cell[(l - 1,) + tuple(int(v) // 2 for v in q)]
                cf = hmean(ei, eps[ck]) * geo
                # ghost u_H/2 + w u_i - (u_n + u_t...)/4, w = 1 (2D) or 5/4 (3D), then g - u_i
                rows.append(me); cols.append(ck); vals.append(0.5 * cf * ih2)
                rows.append(me); cols.append(me); vals.append(((1.0 if D == 2 else 1.25) - 1.0) * cf * ih2)
                n2 = g.copy()
                n2[a] -= sgn
                rows.append(me); cols.append(leaf_cell[(l,) + tuple(int(v) for v in n2)]); vals.append(-0.25 * cf * ih2)
                for t in range(D):
                    if t == a:
                        continue
                    pt = g.copy()
                    pt[t] ^= 1
                    rows.append(me); cols.append(leaf_cell[(l,) + tuple(int(v) for v in pt)])
                    vals.append(-0.25 * cf * ih2)
    n = len(leaf_ids) * ncell
    K = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    B = sp.csr_matrix((bval, (brow, bcol)), shape=(n, nface))
    return K, B
