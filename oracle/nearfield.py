"""Near-element correction of Eq. 14c: exact element integrals minus their point charges.

Test infrastructure (see ``oracle/__init__``).

Sources are the tetrahedra (uniform volume charge rho_e = -div M = -sum_j M_j.grad(phi_j))
and the true boundary triangles (linear surface charge sigma = M.n).  Their nodal
moments, the point charges of Eq. 14b, are
    tet:      q_k^e = rho_e V_e / 4                       (int_e phi_k rho_e)
    triangle: q_k^f = (A_f / 12) (2 sigma_k + sum_{j != k} sigma_j)   (int_f phi_k sigma)
and they add up to q = W^q M exactly.

A placement (s, l) is source element s translated by lattice vector l.  It is near
observer n when
  (a) one of its vertices lands on the observer (every element touching the node,
      including those reached through a periodic image), or
  (b) its centroid lies within r_E of the observer (periodic images included, as in
      Eq. 17 for the box search).
Reading of Sec. 3.2, which ties the element radius to the tetrahedron size (the mean
edge length): r_E = near_elem_factor * mean edge; factor 0 keeps only (a).

For every near placement, 4 pi u_n gains  int_{s+l} G0(r_n - r') dens_s - sum_k q_k^s G0'(r_n - r_k - l)
where G0'(0) = 0 (the self point is carried by R(0) in the lattice sum).  This is
linear in M; E_nk (a 3-vector per (n, k)) collects it so that 4 pi u += E M.

Pinned by tests: on a small free-space mesh with every element near, O1 equals an
independent quadrature of the full continuous potential; moments add up to W^q M.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

from .integrals import tet_uniform, triangle_linear
from .topology import lattice_round, periodic_axes


def boundary_geometry(xyz, tri):
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nn = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(nn, axis=1)
    return nn / (2 * area[:, None]), area


def node_moments(M, xyz, tets, tri, lca, vol, grad, n_unknowns):
    """Sum of element moments per unknown (equals W^q M)."""
    kt = lca[tets]
    rho = -np.einsum("tjd,tjd->t", grad, M[kt])
    q = np.bincount(kt.ravel(), weights=np.repeat(rho * vol / 4.0, 4), minlength=n_unknowns)
    if tri.shape[0]:
        n, area = boundary_geometry(xyz, tri)
        kf = lca[tri]
        sig = np.einsum("fjd,fd->fj", M[kf], n)
        for j in range(3):
            qj = area / 12.0 * (sig[:, j] + sig.sum(axis=1))
            q += np.bincount(kf[:, j], weights=qj, minlength=n_unknowns)
    return q


def _incident(elem_nodes, pos_f, xyz, lca, periods):
    """(n, s, l) for every element s and every vertex landing on its unknown."""
    ne, nv = elem_nodes.shape
    s = np.repeat(np.arange(ne), nv)
    node = elem_nodes.ravel()
    n = lca[node]
    shift = lattice_round(pos_f[n] - xyz[node], periods)
    return n, s, shift


def _geometric(centroids, pos_f, periods, r_E, span):
    if r_E <= 0:
        return np.zeros(0, int), np.zeros(0, int), np.zeros((0, 3))
    per = periodic_axes(periods)
    tree = cKDTree(centroids)
    out_n, out_s, out_l = [], [], []
    for offs in itertools.product(*[range(-span[a], span[a] + 1) if a in per else (0,) for a in range(3)]):
        l = np.array([offs[a] * periods[a] if a in per else 0.0 for a in range(3)])
        hits = tree.query_ball_point(pos_f - l, r_E)
        for n, hs in enumerate(hits):
            if hs:
                out_n.append(np.full(len(hs), n))
                out_s.append(np.asarray(hs))
                out_l.append(np.tile(l, (len(hs), 1)))
    if not out_n:
        return np.zeros(0, int), np.zeros(0, int), np.zeros((0, 3))
    return np.concatenate(out_n), np.concatenate(out_s), np.concatenate(out_l)


def _unique_triples(n, s, l, periods):
    key_l = np.zeros((l.shape[0], 3), dtype=np.int64)
    for a in periodic_axes(periods):
        key_l[:, a] = np.round(l[:, a] / periods[a]).astype(np.int64)
    keys = np.concatenate([n[:, None], s[:, None], key_l], axis=1)
    _, idx = np.unique(keys, axis=0, return_index=True)
    idx = np.sort(idx)
    return n[idx], s[idx], l[idx]


def near_sets(pos_f, xyz, tets, tri, lca, periods, r_E):
    """Near placements for tetrahedra and boundary triangles: two (n, s, l) triples."""
    per = periodic_axes(periods)
    ext = np.ptp(xyz, axis=0)
    span = [int(np.ceil(ext[a] / periods[a])) + 2 if a in per else 0 for a in range(3)]
    res = []
    for elem in (tets, tri):
        if elem.shape[0] == 0:
            res.append((np.zeros(0, int), np.zeros(0, int), np.zeros((0, 3))))
            continue
        n1, s1, l1 = _incident(elem, pos_f, xyz, lca, periods)
        n2, s2, l2 = _geometric(xyz[elem].mean(axis=1), pos_f, periods, r_E, span)
        n = np.concatenate([n1, n2]); s = np.concatenate([s1, s2]); l = np.concatenate([l1, l2])
        res.append(_unique_triples(n, s, l, periods))
    return res


def near_matrix(pos_f, xyz, tets, tri, lca, vol, grad, periods, n_unknowns, r_E, self_tol, observers=None):
    """E as three csr matrices (x, y, z components): 4 pi u += sum_d E[d] @ M[:, d].

    observers (optional): only these rows are built (the others stay empty), for problems
    too large to integrate every near placement; the kept rows are unchanged."""
    (nt, st, lt), (nf, sf, lf) = near_sets(pos_f, xyz, tets, tri, lca, periods, r_E)
    if observers is not None:
        keep_row = np.zeros(n_unknowns, bool)
        keep_row[np.asarray(observers)] = True
        kt, kf = keep_row[nt], keep_row[nf]
        nt, st, lt = nt[kt], st[kt], lt[kt]
        nf, sf, lf = nf[kf], sf[kf], lf[kf]
    rows, cols, vals = [], [], []
    # tetrahedra
    if nt.size:
        obs = pos_f[nt] - lt
        X = xyz[tets[st]]
        I = tet_uniform(obs, X)
        P = np.zeros_like(I)
        for i in range(4):
            node = tets[st, i]
            dist = np.linalg.norm(obs - xyz[node], axis=1)
            is_self = (lca[node] == nt) & (dist < self_tol)
            P += np.where(is_self, 0.0, vol[st] / 4.0 / np.where(is_self, 1.0, dist))
        coef = I - P
        for j in range(4):
            rows.append(nt)
            cols.append(lca[tets[st, j]])
            vals.append(-grad[st, j, :] * coef[:, None])
    # boundary triangles
    if nf.size:
        normal, area = boundary_geometry(xyz, tri)
        obs = pos_f[nf] - lf
        Ij = triangle_linear(obs, xyz[tri[sf]])
        G = np.zeros((nf.size, 3))
        for i in range(3):
            node = tri[sf, i]
            dist = np.linalg.norm(obs - xyz[node], axis=1)
            is_self = (lca[node] == nf) & (dist < self_tol)
            G[:, i] = np.where(is_self, 0.0, 1.0 / np.where(is_self, 1.0, dist))
        A = area[sf]
        for j in range(3):
            Pj = A / 12.0 * (G.sum(axis=1) + G[:, j])
            rows.append(nf)
            cols.append(lca[tri[sf, j]])
            vals.append(normal[sf] * (Ij[:, j] - Pj)[:, None])
    if not rows:
        z = sp.csr_matrix((n_unknowns, n_unknowns))
        return (z, z.copy(), z.copy()), {"tets": 0, "tris": 0}
    r = np.concatenate(rows); c = np.concatenate(cols); v = np.concatenate(vals)
    E = []
    for d in range(3):
        m = sp.coo_matrix((v[:, d], (r, c)), shape=(n_unknowns, n_unknowns)).tocsr()
        m.sum_duplicates()
        E.append(m)
    return tuple(E), {"tets": int(nt.size), "tris": int(nf.size)}
