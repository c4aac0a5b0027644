"""Local field terms beyond exchange: crystalline anisotropy per grain and exchange stiffness per
tetrahedron (Eq. 3's local terms; the granular example of Sec. 4.4 has grains with their own
easy axes and a reduced exchange across grain boundaries).

Test infrastructure (see ``oracle/__init__``).

Energy densities of a grain g with orthonormal axes a1, a2, a3 (rows of its 3x3 axis matrix),
cubic constant K1 [J/m^3], uniaxial constant Ku [J/m^3] and axis u, with ai = m . a_i:
  cubic     e_c = K1 (a1^2 a2^2 + a2^2 a3^2 + a3^2 a1^2)
  uniaxial  e_u = -Ku (m . u)^2
Their fields h_g(m) = -(1/(mu0 Ms)) de/dm:
  cubic     h_c = -(2 K1 / (mu0 Ms)) sum_i ai (aj^2 + ak^2) a_i   ({i, j, k} = {1, 2, 3})
  uniaxial  h_u = (2 Ku / (mu0 Ms)) (m . u) u
Discretisation (reading; the paper gives no formula): the energy of tetrahedron e is its volume
times e_{g(e)} at the nodal values, lumped to the nodes, E = sum_e (V_e / 4) sum_{n in e}
e_{g(e)}(m_n), so the nodal field is the volume-weighted mean of the grains meeting at the node,
  H_an,n = sum_g w_ng h_g(m_n),  w_ng = sum_{e ni n, g(e) = g} (V_e / 4) / V_n.

Exchange with a stiffness per tetrahedron (reading of the inter-grain exchange A_iex: the
tetrahedra that touch a grain boundary carry A_iex, the others the grain's A):
  H_ex = -(2 / (mu0 Ms)) V^-1 K_A m,   (K_A)_nk = sum_e A_e V_e grad(phi_n) . grad(phi_k),
which is Eq. 8 with A moved inside the element sum.

Pinned by tests: Euler's identity for the quartic cubic energy (m . de/dm = 4 e) against the
closed-form energies K1/3 along [111], K1/4 along [110] and 0 along [100]; the closed-form
field along [110]; a finite difference of the lumped total energy; the uniaxial closed form;
and K_A = A K for a uniform stiffness.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .operators import MU0, tet_geometry


def grain_weights(tets, lca, vol, tet_grain, n_unknowns, n_grains):
    """w (N', G) dense: the volume share of each grain at each unknown (rows sum to 1)."""
    ids = lca[tets]
    rows = ids.ravel()
    cols = np.repeat(np.asarray(tet_grain), 4)
    vals = np.repeat(0.25 * vol, 4)
    W = sp.coo_matrix((vals, (rows, cols)), shape=(n_unknowns, n_grains)).toarray()
    return W / W.sum(axis=1, keepdims=True)


def cubic_field(m, axes, K1, Ms):
    """h_c of one grain for unit vectors m (N, 3); axes (3, 3) rows a1, a2, a3."""
    a = m @ axes.T                                     # (N, 3) direction cosines
    s = a * a
    f = np.stack([a[:, 0] * (s[:, 1] + s[:, 2]), a[:, 1] * (s[:, 0] + s[:, 2]), a[:, 2] * (s[:, 0] + s[:, 1])], 1)
    return -(2.0 * K1 / (MU0 * Ms)) * (f @ axes)


def uniaxial_field(m, u, Ku, Ms):
    u = np.asarray(u, dtype=np.float64)
    return (2.0 * Ku / (MU0 * Ms)) * (m @ u)[:, None] * u[None, :]


def cubic_energy_density(m, axes, K1):
    a = m @ axes.T
    s = a * a
    return K1 * (s[:, 0] * s[:, 1] + s[:, 1] * s[:, 2] + s[:, 2] * s[:, 0])


def anisotropy_field(m, weights, axes, K1, Ku, u, Ms):
    """H_an at every unknown: sum over grains of w_ng (h_c + h_u)(m_n)."""
    H = np.zeros_like(m)
    for g in range(weights.shape[1]):
        sel = weights[:, g] > 0
        if not np.any(sel):
            continue
        h = cubic_field(m[sel], axes[g], K1[g], Ms) + uniaxial_field(m[sel], u[g], Ku[g], Ms)
        H[sel] += weights[sel, g][:, None] * h
    return H


def lumped_energy(m, tets, lca, vol, tet_grain, axes, K1, Ku, u):
    """E = sum_e (V_e/4) sum_{n in e} e_g(e)(m_n) [J] (cubic + uniaxial)."""
    E = 0.0
    ids = lca[tets]
    for g in np.unique(tet_grain):
        sel = np.asarray(tet_grain) == g
        mm = m[ids[sel].ravel()]
        e = cubic_energy_density(mm, axes[g], K1[g]) - Ku[g] * (mm @ np.asarray(u[g])) ** 2
        E += float(np.sum(np.repeat(0.25 * vol[sel], 4) * e))
    return E


def exchange_matrix_per_tet(xyz, tets, lca, n_unknowns, A_tet):
    """K_A = sum_e A_e V_e grad(phi_n) . grad(phi_k) (csr)."""
    vol, g = tet_geometry(xyz, tets)
    ids = lca[tets]
    rows = np.repeat(ids, 4, axis=1).ravel()
    cols = np.tile(ids, (1, 4)).ravel()
    gi = np.repeat(g, 4, axis=1)
    gj = np.tile(g, (1, 4, 1))
    kval = ((np.asarray(A_tet) * vol)[:, None] * np.einsum("tkd,tkd->tk", gi, gj)).ravel()
    K = sp.coo_matrix((kval, (rows, cols)), shape=(n_unknowns, n_unknowns)).tocsr()
    K.sum_duplicates()
    return K


def exchange_field_per_tet(KA, V, m, Ms):
    """H_ex = -(2 / (mu0 Ms)) V^-1 K_A m."""
    return -(2.0 / (MU0 * Ms)) * (KA @ m) / V[:, None]
