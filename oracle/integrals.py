"""Exact potential integrals of uniform and linear sources on triangles and tetrahedra.

Test infrastructure (see ``oracle/__init__``).

These are the exact element integrals of Sec. 3.2 that
replace the point-charge contributions of nearby sources (Eq. 14c).

Triangle T with unit normal n, observer r, projection p = r - d n onto the plane.
For each edge i (counter-clockwise about n) from P- to P+ with unit direction l_i
and in-plane outward normal u_i = l_i x n:
    t_i = (P- - p).u_i,  l+- = (P+- - p).l_i,  R0_i^2 = t_i^2 + d^2,  R+- = |P+- - r|,
    f_i = ln((R+ + l+) / (R- + l-)).
Then (integration of 1/R in polar form about p, edge by edge):
    I0   = int_T dS/R       = sum_i [ t_i f_i - |d| (atan(t_i l+ / (R0^2 + |d| R+)) - atan(t_i l- / (R0^2 + |d| R-))) ]
    Ivec = int_T (r'-p)/R dS = 1/2 sum_i u_i [ R0_i^2 f_i + l+ R+ - l- R- ]
and a linear density phi(r') = phi(p) + grad(phi).(r' - p) integrates to
phi(p) I0 + grad(phi).Ivec.

Tetrahedron with uniform density: div'((r'-r)/|r'-r|) = 2/|r'-r| gives
    int_V dV/|r - r'| = 1/2 sum_faces h_f I0_f,  h_f = (P_f - r).n_f (outward n_f).

Pinned by tests against Duffy-transformed Gauss-Legendre quadrature for observers
far away, inside, on a face, on an edge and at a vertex, and against the far-field
limit (total charge / distance).
"""
from __future__ import annotations

import numpy as np

_EPS = 1e-13


def _dot(a, b):
    return np.einsum("...i,...i->...", a, b)


def triangle_integrals(r: np.ndarray, P: np.ndarray):
    """r: (M, 3) observers, P: (M, 3, 3) triangle vertices (one triangle per observer).

    Returns (I0 (M,), Ivec (M, 3), p (M, 3), n (M, 3)).
    """
    a, b, c = P[:, 0], P[:, 1], P[:, 2]
    nn = np.cross(b - a, c - a)
    area2 = np.linalg.norm(nn, axis=1)
    n = nn / area2[:, None]
    d = _dot(r - a, n)
    p = r - d[:, None] * n
    ad = np.abs(d)
    scale = np.sqrt(area2)
    I0 = np.zeros(r.shape[0])
    Iv = np.zeros_like(r)
    for (Pm, Pp) in ((a, b), (b, c), (c, a)):
        e = Pp - Pm
        le = np.linalg.norm(e, axis=1)
        l = e / le[:, None]
        u = np.cross(l, n)
        t = _dot(Pm - p, u)
        lm = _dot(Pm - p, l)
        lp = _dot(Pp - p, l)
        R02 = t * t + d * d
        Rm = np.linalg.norm(Pm - r, axis=1)
        Rp = np.linalg.norm(Pp - r, axis=1)
        ok = R02 > (_EPS * scale) ** 2
        R02s = np.where(ok, R02, 1.0)
        # R + l without cancellation: for l < 0 use R0^2 / (R - l)
        with np.errstate(divide="ignore", invalid="ignore"):
            Ap = np.where(lp >= 0, Rp + lp, R02s / (Rp - lp))
            Am = np.where(lm >= 0, Rm + lm, R02s / (Rm - lm))
            f = np.where(ok, np.log(Ap / Am), 0.0)
            at = (np.arctan(t * lp / (R02s + ad * Rp)) - np.arctan(t * lm / (R02s + ad * Rm)))
        I0 += np.where(ok, t * f - ad * at, 0.0)
        Iv += 0.5 * u * np.where(ok, R02 * f, 0.0)[:, None] + 0.5 * u * (lp * Rp - lm * Rm)[:, None]
    return I0, Iv, p, n


def triangle_linear(r: np.ndarray, P: np.ndarray) -> np.ndarray:
    """int_T phi_j(r') / |r - r'| dS' for the three P1 hat functions: (M, 3)."""
    I0, Iv, p, n = triangle_integrals(r, P)
    a, b, c = P[:, 0], P[:, 1], P[:, 2]
    nn = np.cross(b - a, c - a)
    A2 = _dot(nn, n)                      # twice the area
    out = np.empty((r.shape[0], 3))
    verts = (a, b, c)
    for j in range(3):
        q1, q2 = verts[(j + 1) % 3], verts[(j + 2) % 3]
        # barycentric of vertex j: area(p, q1, q2) / area(T); gradient n x (q2 - q1) / (2 area)
        lam_p = _dot(np.cross(q1 - p, q2 - p), n) / A2
        grad = np.cross(n, q2 - q1) / A2[:, None]
        out[:, j] = lam_p * I0 + _dot(grad, Iv)
    return out


def tet_uniform(r: np.ndarray, X: np.ndarray) -> np.ndarray:
    """int_tet dV' / |r - r'| for (M, 3) observers and (M, 4, 3) vertices."""
    out = np.zeros(r.shape[0])
    cen = X.mean(axis=1)
    for f in ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)):
        P = X[:, list(f)].copy()
        nn = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        flip = _dot(nn, P[:, 0] - cen) < 0
        P[flip, 1], P[flip, 2] = P[flip, 2].copy(), P[flip, 1].copy()
        I0, _, _, n = triangle_integrals(r, P)
        h = _dot(P[:, 0] - r, n)
        out += 0.5 * h * I0
    return out
