"""Pins of the periodic near-element correction of Eq. 14c (``oracle/nearfield.py``).

The oracle finds near placements (element s translated by lattice vector l) with a k-d tree
over element centroids, queried at every observer shifted by every image vector.  These tests
enumerate the same placements by brute force (every observer x every element x every lattice
vector in a generous range, plain distance tests), and rebuild the correction
    4 pi u_n += sum over near (s, l) [ int_{s+l} G0(r_n - r') dens_s  -  sum_k q_k^s G0'(r_n - r_k - l) ]
directly from the source densities (uniform rho on tetrahedra, linear sigma on boundary
triangles, Sec. 3.2), without the matrix E.  The exact integrals are the library step (pinned
against quadrature in test_oracle_core).  A wrong sign or image vector in the search, a range
of images too small, a lost self-point skip or a transposed 3-vector in E fails one of these.
"""
import itertools

import numpy as np
import pytest

import meshgen
from oracle.integrals import tet_uniform, triangle_linear
from oracle.nearfield import boundary_geometry, near_sets
from oracle.problem import OracleProblem


def _protruding_prism():
    p = meshgen.prism_cell(3, 3, 4, jitter=0.15, seed=5)
    xyz = p.xyz.copy()
    xyz[:, 2] += 0.37 * p.periods[2] + 0.2 * xyz[:, 0]       # straddles the cell boundary along z
    return meshgen.Mesh(xyz, p.tets, p.periods)


def _shifted_film():
    f = meshgen.film_cell(4, 3, 2, jitter=0.15, seed=4)
    xyz = f.xyz.copy()
    xyz[:, 0] += 0.41 * f.periods[0] + 0.1 * xyz[:, 2]
    xyz[:, 1] -= 0.23 * f.periods[1]
    return meshgen.Mesh(xyz, f.tets, f.periods)


MESHES = {
    "prism_1d": (_protruding_prism, 1.5),
    "film_2d": (_shifted_film, 1.2),
    "cube_3d": (lambda: meshgen.cube_cell(3, jitter=0.2, seed=6), 1.1),
}


def _brute_placements(ob, elems, r_E, S=4):
    """{(n, s, l-integers)} of every near placement, by exhaustive enumeration."""
    per = [a for a in range(3) if ob.periods[a] > 0]
    tol = 1e-6 * ob.mean_edge
    cent = ob.xyz[elems].mean(axis=1)
    found = set()
    for img in itertools.product(*[range(-S, S + 1) if a in per else (0,) for a in range(3)]):
        lvec = np.array([img[a] * ob.periods[a] for a in range(3)])
        for n in range(ob.Np):
            r = ob.pos_f[n]
            d_cent = np.linalg.norm(r - cent - lvec, axis=1)
            lands = np.zeros(elems.shape[0], bool)
            for j in range(elems.shape[1]):
                v = elems[:, j]
                lands |= (ob.lca[v] == n) & (np.linalg.norm(ob.xyz[v] + lvec - r, axis=1) < tol)
            near = lands | ((d_cent <= r_E) if r_E > 0 else False)
            for s in np.nonzero(near)[0]:
                found.add((n, int(s), img))
    return found


def _oracle_placements(ob, n, s, l):
    out = set()
    for nn, ss, ll in zip(n.tolist(), s.tolist(), l):
        out.add((nn, ss, tuple(int(round(ll[a] / ob.periods[a])) if ob.periods[a] > 0 else 0 for a in range(3))))
    return out


@pytest.fixture(scope="module", params=sorted(MESHES))
def case(request):
    mk, factor = MESHES[request.param]
    mesh = mk()
    ob = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, near_elem_factor=factor)
    return request.param, ob


def test_near_search_matches_exhaustive_enumeration(case):
    name, ob = case
    (nt, st, lt), (nf, sf, lf) = near_sets(ob.pos_f, ob.xyz, ob.tets, ob.tri, ob.lca, ob.periods, ob.r_E)
    got_t = _oracle_placements(ob, nt, st, lt)
    got_f = _oracle_placements(ob, nf, sf, lf)
    want_t = _brute_placements(ob, ob.tets, ob.r_E)
    want_f = _brute_placements(ob, ob.tri, ob.r_E)
    assert len(got_t) == nt.size and len(got_f) == nf.size          # no placement twice
    assert got_t == want_t, (name, len(got_t ^ want_t))
    assert got_f == want_f, (name, len(got_f ^ want_f))
    # the radius reaches past the touching elements, also through periodic images
    assert any(any(k[2]) for k in want_t)
    touching = _brute_placements(ob, ob.tets, 0.0)
    assert len(want_t) > len(touching)


def test_near_correction_matches_direct_sum_over_placements(case):
    name, ob = case
    m = meshgen.m_random(ob.Np, seed=21)
    M = ob.Ms * m
    tol = 1e-6 * ob.mean_edge
    u = np.zeros(ob.Np)
    # tetrahedra: uniform rho_e = -div M on the element, point charges rho_e V_e / 4 at its vertices
    rho = -np.einsum("tjd,tjd->t", ob.grad, M[ob.lca[ob.tets]])
    for (n, s, img) in sorted(_brute_placements(ob, ob.tets, ob.r_E)):
        lvec = np.array([img[a] * ob.periods[a] for a in range(3)])
        X = ob.xyz[ob.tets[s]] + lvec
        r = ob.pos_f[n]
        exact = rho[s] * tet_uniform(r[None], X[None])[0]
        point = sum(rho[s] * ob.vol[s] / 4 / np.linalg.norm(r - X[j]) for j in range(4)
                    if np.linalg.norm(r - X[j]) >= tol)
        u[n] += exact - point
    # boundary triangles: linear sigma = M.n, point charges (A/12)(2 sigma_k + sum_{j != k} sigma_j)
    nrm, area = boundary_geometry(ob.xyz, ob.tri)
    for (n, s, img) in sorted(_brute_placements(ob, ob.tri, ob.r_E)):
        lvec = np.array([img[a] * ob.periods[a] for a in range(3)])
        X = ob.xyz[ob.tri[s]] + lvec
        sig = M[ob.lca[ob.tri[s]]] @ nrm[s]
        r = ob.pos_f[n]
        exact = float(sig @ triangle_linear(r[None], X[None])[0])
        point = sum(area[s] / 12 * (sig[k] + sig.sum()) / np.linalg.norm(r - X[k]) for k in range(3)
                    if np.linalg.norm(r - X[k]) >= tol)
        u[n] += exact - point
    em = ob.EM(m)
    assert np.abs(em - u).max() <= 1e-12 * np.abs(u).max(), name
