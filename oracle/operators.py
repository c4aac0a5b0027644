"""Local sparse operators on the periodized P1 basis.

Test infrastructure (see ``oracle/__init__``).

Every operator is assembled tetrahedron by tetrahedron with the original
(unfolded) vertex coordinates and the vertex indices mapped to their unknowns
(LCA).  Assembling each element once with mapped indices gives the extended
neighbourhoods of cases 1-3 of Sec. 3.1 (Eqs. 9-12) with every edge counted once,
which is what the de-duplication of Eq. 11 asks for.

Reading of the weights (the paper cites its parent code for omega): standard P1
with lumped nodal volumes V_n = sum_e V_e / 4,
  exchange (Eq. 7-8):   H_ex = -(2A / (mu0 Ms)) V^-1 K m,  K_nk = sum_e V_e grad(phi_n).grad(phi_k)
  charges  (Eq. 14a):   q_n = sum_e int_e M . grad(phi_n) dV  ->  (W^q)_nk = sum_e (V_e/4) grad(phi_n)
  gradient (Eq. 14d):   H_ms = -V^-1 (W^q)^T u.
The charge form equals the volume charge -div M plus the surface charge M.n on
true boundary faces (integration by parts); on periodic faces the two surface
terms cancel.

Pinned by tests: K 1 = 0, K symmetric, sum_n q_n = 0, (W^q)^T 1 = 0 rows of the
gradient, the plane-wave Laplacian on a periodic cube, and the closed-form
demagnetising factors of the film, prism and filled 3D cell.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MU0 = 4e-7 * np.pi


def tet_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Volumes (T,) and barycentric gradients (T, 4, 3) of each tetrahedron."""
    v = xyz[tets]                                     # (T, 4, 3)
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)  # columns
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                            # rows = grad(lambda_1..3)
    g = np.empty((tets.shape[0], 4, 3))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    return det / 6.0, g


def assemble(xyz: np.ndarray, tets: np.ndarray, lca: np.ndarray, n_unknowns: int):
    """Return dict with K (csr), Wq (tuple of 3 csr, x/y/z), V (N',)."""
    vol, g = tet_geometry(xyz, tets)
    ids = lca[tets]                                    # (T, 4)
    rows = np.repeat(ids, 4, axis=1).ravel()           # (T*16,) row = i
    cols = np.tile(ids, (1, 4)).ravel()                # col = j
    gi = np.repeat(g, 4, axis=1)                       # (T, 16, 3) grad_i
    gj = np.tile(g, (1, 4, 1))                         # (T, 16, 3) grad_j
    kval = (vol[:, None] * np.einsum("tkd,tkd->tk", gi, gj)).ravel()
    K = sp.coo_matrix((kval, (rows, cols)), shape=(n_unknowns, n_unknowns)).tocsr()
    K.sum_duplicates()
    Wq = []
    for d in range(3):
        w = (0.25 * vol[:, None] * gi[:, :, d]).ravel()
        M = sp.coo_matrix((w, (rows, cols)), shape=(n_unknowns, n_unknowns)).tocsr()
        M.sum_duplicates()
        Wq.append(M)
    V = np.bincount(ids.ravel(), weights=np.repeat(0.25 * vol, 4), minlength=n_unknowns)
    return {"K": K, "Wq": tuple(Wq), "V": V, "vol": vol, "grad": g}


def mean_edge(xyz: np.ndarray, tets: np.ndarray) -> float:
    """Mean length of the unique edges of the (original, unmapped) mesh."""
    e = np.concatenate([tets[:, [a, b]] for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(xyz[e[:, 1]] - xyz[e[:, 0]], axis=1).mean())


def charges(Wq, M: np.ndarray) -> np.ndarray:
    """Eq. 14a: q = W^q M (M = Ms m, (N', 3))."""
    return Wq[0] @ M[:, 0] + Wq[1] @ M[:, 1] + Wq[2] @ M[:, 2]


def gradient_field(Wq, V: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Eq. 14d: H_ms = -V^-1 (W^q)^T u, returns (N', 3)."""
    return -np.stack([Wq[d].T @ u for d in range(3)], axis=1) / V[:, None]


def exchange_field(K, V: np.ndarray, m: np.ndarray, A: float, Ms: float) -> np.ndarray:
    """Eqs. 7-12: H_ex = -(2A / (mu0 Ms)) V^-1 K m."""
    return -(2.0 * A / (MU0 * Ms)) * (K @ m) / V[:, None]
