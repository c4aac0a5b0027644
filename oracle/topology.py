"""Periodic pairing, lowest common ancestors, boundary faces and the protruding fold.

Test infrastructure (see ``oracle/__init__``).

* Pairing and LCA follow Sec. 2.2: nodes i, j form a PBC pair when r_j - r_i is a
  lattice vector sum_i n_i L_i e_i with n_i in {-1, 0, 1}, not all zero (Eq. 5,
  touching cells of Sec. 2.1).  Chains are merged with union-find so every node
  maps to one ancestor; the ancestors are the N' unknowns.
  Reading (the paper does not fix the ancestor of a group): the ancestor is the
  member with the lexicographically smallest coordinates along the periodic axes
  (the low-face copy), and unknowns are numbered by increasing original node index.
* The fold follows Eq. 18: each unknown is shifted by whole periods to lie in the
  half-open window [r0 - L/2, r0 + L/2) along each periodic axis, with r0 the mean
  of the unknowns' positions.  Reading: Eq. 18 minimises a Manhattan distance to r0
  while the text says the result lies in [0, L); the window above does the former.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.spatial import cKDTree


def periodic_axes(periods) -> list[int]:
    return [a for a in range(3) if periods[a] > 0]


def pair_nodes(xyz: np.ndarray, periods, rel_tol: float = 1e-9):
    """Return (lca, roots): lca[i] = unknown index of node i, roots[u] = node index.

    Pinned by tests: film/cube/prism pair counts (closed form for the structured
    meshes), the L = 2, D = 3 parallelogram fold, and invariance of every field
    under translation of the mesh.
    """
    N = xyz.shape[0]
    per = periodic_axes(periods)
    parent = np.arange(N)

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    if per:
        L = np.asarray(periods, dtype=np.float64)
        tol = rel_tol * min(L[a] for a in per)
        tree = cKDTree(xyz)
        for offs in itertools.product((-1, 0, 1), repeat=len(per)):
            if not any(offs):
                continue
            o = np.zeros(3)
            for a, n in zip(per, offs):
                o[a] = n * L[a]
            d, j = tree.query(xyz + o, distance_upper_bound=tol)
            hit = np.nonzero(np.isfinite(d))[0]
            for i, jj in zip(hit.tolist(), j[hit].tolist()):
                ri, rj = find(i), find(jj)
                if ri != rj:
                    parent[max(ri, rj)] = min(ri, rj)
    comp = np.array([find(i) for i in range(N)])
    # ancestor = member with lexicographically smallest periodic coordinates
    groups: dict[int, list[int]] = {}
    for i, c in enumerate(comp.tolist()):
        groups.setdefault(c, []).append(i)
    root_of_comp = {}
    for c, mem in groups.items():
        if len(mem) == 1 or not per:
            root_of_comp[c] = mem[0]
        else:
            root_of_comp[c] = min(mem, key=lambda i: tuple(xyz[i, a] for a in per))
    root = np.array([root_of_comp[c] for c in comp.tolist()])
    roots = np.unique(root)           # sorted by original index
    uid = -np.ones(N, dtype=np.int64)
    uid[roots] = np.arange(roots.size)
    lca = uid[root]
    return lca, roots


def fold_positions(pos: np.ndarray, periods) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 18: shift positions by whole periods into [r0 - L/2, r0 + L/2).

    pos: (N', 3) positions of the unknowns.  Returns (folded, r0).
    The shift count per axis is floor((x - r0 + L/2) / L).
    """
    out = pos.copy()
    r0 = pos.mean(axis=0)
    for a in periodic_axes(periods):
        L = float(periods[a])
        k = np.floor((pos[:, a] - r0[a] + 0.5 * L) / L)
        out[:, a] = pos[:, a] - k * L
    return out, r0


def lattice_round(d: np.ndarray, periods) -> np.ndarray:
    """Nearest lattice vector to each row of d (zero along non-periodic axes)."""
    out = np.zeros_like(d)
    for a in periodic_axes(periods):
        L = float(periods[a])
        out[..., a] = np.round(d[..., a] / L) * L
    return out


def boundary_faces(xyz: np.ndarray, tets: np.ndarray, lca: np.ndarray):
    """True (non-periodic) boundary faces.

    A face is interior when its three vertices, mapped to unknowns, occur in two
    tetrahedra; a face on a periodic boundary meets its image on the opposite face
    this way, so only faces of the true boundary remain (Sec. 3.2: surface charges
    live on the boundary of the magnetised domain).
    Returns (tri (F, 3) original node indices ordered so that the normal
    (b - a) x (c - a) points out of the tetrahedron, owner tet index (F,)).
    """
    opp = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
    faces = np.concatenate([tets[:, list(o)] for o in opp], axis=0)
    owner = np.tile(np.arange(tets.shape[0]), 4)
    keys = np.sort(lca[faces], axis=1)
    _, inv, cnt = np.unique(keys, axis=0, return_inverse=True, return_counts=True)
    once = cnt[inv.ravel()] == 1
    tri, own = faces[once], owner[once]
    # make the orientation outward with respect to the owner tetrahedron
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    n = np.cross(b - a, c - a)
    cen = xyz[tets[own]].mean(axis=1)
    flip = np.einsum("ij,ij->i", n, a - cen) < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    return tri, own
