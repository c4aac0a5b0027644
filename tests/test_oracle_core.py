"""Pins of the oracle's exact integrals, pairing/fold, local operators and LLG."""
import math

import numpy as np
import pytest

import meshgen
from oracle import operators as ops
from oracle.integrals import tet_uniform, triangle_linear
from oracle.llg import rk4_step, llg_rhs
from oracle.paim import lagrange_weights
from oracle.topology import fold_positions, pair_nodes
from oracle.problem import GAMMA0

# ---------------------------------------------------------------- exact integrals
_X, _W = np.polynomial.legendre.leggauss(40)
_X = 0.5 * (_X + 1)
_W = 0.5 * _W


def quad_tet(o, X):
    """Signed cone decomposition about o + Duffy map: smooth integrand, tensor Gauss-Legendre."""
    cen = X.mean(0)
    tot = 0.0
    U, V, Wt = np.meshgrid(_X, _X, _X, indexing="ij")
    WW = _W[:, None, None] * _W[None, :, None] * _W[None, None, :]
    for f in ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)):
        A, B, C = X[list(f)]
        if np.dot(np.cross(B - A, C - A), A - cen) < 0:
            B, C = C, B
        det = np.dot(A - o, np.cross(B - o, C - o))
        if abs(det) < 1e-30:
            continue
        P = (A - o)[None, None, None] + V[..., None] * ((B - A)[None, None, None] + Wt[..., None] * (C - B)[None, None, None])
        tot += np.sum(WW * U * V * det / np.linalg.norm(P, axis=-1))
    return tot


def quad_tri(o, T):
    """Sub-triangles about the projection of o, Duffy map, Gauss-Legendre; returns int phi_j / R."""
    a_, b_, c_ = T
    n = np.cross(b_ - a_, c_ - a_)
    A2 = np.linalg.norm(n)
    n = n / A2
    p = o - np.dot(o - a_, n) * n
    U, V = np.meshgrid(_X, _X, indexing="ij")
    WW = _W[:, None] * _W[None, :]
    tot = np.zeros(3)
    for (A, B) in ((a_, b_), (b_, c_), (c_, a_)):
        sa = np.dot(np.cross(A - p, B - p), n)
        if abs(sa) < 1e-40:
            continue
        R = p + U[..., None] * ((A - p) + V[..., None] * (B - A))
        dist = np.linalg.norm(R - o, axis=-1)
        for j in range(3):
            q1, q2 = T[(j + 1) % 3], T[(j + 2) % 3]
            lam = np.einsum("...i,i->...", np.cross(q1 - R, q2 - R), n) / A2
            tot[j] += np.sum(WW * U * sa * lam / dist)
    return tot


TET = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 1.1, 0], [0.3, 0.2, 0.9]], float)


@pytest.mark.parametrize("obs", [TET.mean(0), TET[0], 0.5 * (TET[0] + TET[1]), (TET[1] + TET[2] + TET[3]) / 3,
                                 np.array([3.0, 2.0, 1.0]), np.array([0.5, 0.5, -0.3])])
def test_tet_integral_vs_quadrature(obs):
    e = tet_uniform(obs[None], TET[None])[0]
    q = quad_tet(obs, TET)
    assert abs(e - q) < 1e-12 * abs(q)


@pytest.mark.parametrize("obs", [TET[:3].mean(0), TET[0], 0.5 * (TET[0] + TET[1]), np.array([0.3, 0.3, 0.5]),
                                 np.array([2.0, -1.0, 0.0]), np.array([2.0, -1.0, 0.7]), np.array([0.3, 0.3, -0.05])])
def test_triangle_integral_vs_quadrature(obs):
    e = triangle_linear(obs[None], TET[:3][None])[0]
    q = quad_tri(obs, TET[:3])
    assert np.abs(e - q).max() < 1e-12 * np.abs(q).max()


def test_far_field_limits():
    far = np.array([[400.0, -300.0, 1200.0]])
    d = np.linalg.norm(far[0] - TET.mean(0))
    vol = abs(np.linalg.det(TET[1:] - TET[0])) / 6
    assert abs(tet_uniform(far, TET[None])[0] * d / vol - 1) < 1e-6
    area = 0.5 * np.linalg.norm(np.cross(TET[1] - TET[0], TET[2] - TET[0]))
    s = triangle_linear(far, TET[:3][None])[0]
    for j in range(3):
        cj = (TET[:3].sum(0) + TET[j]) / 4.0           # first moment of the hat function phi_j
        assert abs(s[j] * np.linalg.norm(far[0] - cj) / (area / 3) - 1.0) < 1e-6


# ---------------------------------------------------------------- pairing and fold
def test_pair_counts():
    f = meshgen.film_cell(10, 10, 2)
    lca, roots = pair_nodes(f.xyz, f.periods)
    assert f.n_nodes == 11 * 11 * 3 and roots.size == 10 * 10 * 3
    c = meshgen.cube_cell(4)
    lca, roots = pair_nodes(c.xyz, c.periods)
    assert roots.size == 4 ** 3
    # a corner has 7 images that all map to one unknown
    corner = np.nonzero(np.all(np.isclose(c.xyz, 0.0), axis=1))[0][0]
    assert np.sum(lca == lca[corner]) == 8
    # ancestors sit on the low faces
    assert np.all(c.xyz[roots] < 4e-9 - 1e-15)
    p = meshgen.prism_cell(3, 3, 4)
    lca, roots = pair_nodes(p.xyz, p.periods)
    assert roots.size == 4 * 4 * 4


def test_nt_mesh_has_no_pairs():
    s = meshgen.sphere_lattice(target_nodes=1500, seed=3)
    lca, roots = pair_nodes(s.xyz, s.periods)
    assert roots.size == s.n_nodes and np.array_equal(lca, np.arange(s.n_nodes))


def test_fold_parallelogram():
    # Sec. 4.1 example: a parallelogram with period L_x = 2 spanning D_x = 3
    ys = np.linspace(0, 1, 5)
    xs = np.linspace(0, 2, 9)
    P = np.array([(x + y, y, 0.0) for y in ys for x in xs])
    assert np.ptp(P[:, 0]) == pytest.approx(3.0)
    folded, r0 = fold_positions(P, (2.0, 0.0, 0.0))
    assert np.ptp(folded[:, 0]) < 2.0
    assert np.all(folded[:, 0] >= r0[0] - 1.0) and np.all(folded[:, 0] < r0[0] + 1.0)
    d = (folded[:, 0] - P[:, 0]) / 2.0
    assert np.allclose(d, np.round(d))       # shifted by whole periods only
    assert np.array_equal(folded[:, 1:], P[:, 1:])


# ---------------------------------------------------------------- local operators
@pytest.fixture(scope="module")
def cube_ops():
    c = meshgen.cube_cell(5, jitter=0.2, seed=4)
    lca, roots = pair_nodes(c.xyz, c.periods)
    return c, lca, roots, ops.assemble(c.xyz, c.tets.astype(np.int64), lca, roots.size)


def test_laplacian_invariants(cube_ops):
    c, lca, roots, op = cube_ops
    K = op["K"]
    assert abs(K - K.T).max() < 1e-12 * abs(K).max()
    assert np.abs(K @ np.ones(roots.size)).max() < 1e-12 * abs(K).max()
    assert np.isclose(op["V"].sum(), 125e-27, rtol=1e-12)   # lumped volumes fill the cell


def test_charge_and_gradient_invariants(cube_ops):
    c, lca, roots, op = cube_ops
    Wq = op["Wq"]
    rng = np.random.default_rng(0)
    M = rng.normal(size=(roots.size, 3))
    q = ops.charges(Wq, M)
    assert abs(q.sum()) < 1e-13 * np.abs(q).sum()
    # rows of the gradient annihilate constants
    H = ops.gradient_field(Wq, op["V"], np.ones(roots.size))
    assert np.abs(H).max() < 1e-12 * np.abs(ops.gradient_field(Wq, op["V"], rng.normal(size=roots.size))).max()


def test_gradient_exact_for_linear_potential():
    # on a non-periodic mesh the P1 gradient of a linear function is exact at every node
    xyz, tets = meshgen.kuhn_box(4, 3, 3, 1e-9, jitter=0.2, seed=5)
    lca, roots = pair_nodes(xyz, (0, 0, 0))
    op = ops.assemble(xyz, tets.astype(np.int64), lca, roots.size)
    g = np.array([1.5e9, -0.7e9, 0.2e9])
    u = xyz @ g
    H = ops.gradient_field(op["Wq"], op["V"], u)
    assert np.allclose(H, -g[None, :], rtol=1e-11, atol=0)


def test_plane_wave_laplacian():
    errs = []
    for n in (8, 16):
        xyz, tets = meshgen.kuhn_box(n, n, 2, 1.0 / n, jitter=0.0)
        per = (1.0, 1.0, 2.0 / n)
        lca, roots = pair_nodes(xyz, per)
        op = ops.assemble(xyz, tets.astype(np.int64), lca, roots.size)
        k = 2 * math.pi
        x = xyz[roots, 0]
        m = np.stack([np.cos(k * x), np.sin(k * x), np.zeros_like(x)], axis=1)
        lap = -(op["K"] @ m) / op["V"][:, None]
        errs.append(np.abs(lap + k * k * m).max() / (k * k))
    assert errs[1] < 0.3 * errs[0] and errs[1] < 0.02    # second order in h


# ---------------------------------------------------------------- stencils
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_lagrange_reproduces_polynomials(p):
    s = np.linspace(0.37, 2.61, 13)
    w = lagrange_weights(s, p)
    for deg in range(p + 1):
        vals = (np.arange(p + 1, dtype=float) ** deg)
        assert np.allclose(w @ vals, s ** deg, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- LLG
def test_single_spin_precession():
    # constant field along z, no damping: m precesses at gamma0 H about z
    H0 = 1e5
    m0 = np.array([[math.sin(0.3), 0.0, math.cos(0.3)]])
    field = lambda m: np.array([[0.0, 0.0, H0]])
    dt, n = 1e-13, 200
    m = m0.copy()
    for _ in range(n):
        m = rk4_step(m, dt, field, alpha=0.0)
    ang = GAMMA0 * H0 * dt * n          # -gamma m x H turns m right-handedly about H
    ref = np.array([math.sin(0.3) * math.cos(ang), math.sin(0.3) * math.sin(ang), math.cos(0.3)])
    assert np.abs(m[0] - ref).max() < 1e-9


def test_damped_spin_angle():
    # damped LLG in a constant field: tan(theta/2) = tan(theta0/2) exp(-alpha gamma0 H t / (1 + alpha^2))
    H0, alpha = 2e5, 0.1
    th0 = 1.0
    m = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    field = lambda m: np.array([[0.0, 0.0, H0]])
    dt, n = 5e-14, 400
    for _ in range(n):
        m = rk4_step(m, dt, field, alpha=alpha)
    th = math.acos(m[0, 2])
    ref = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * GAMMA0 * H0 * dt * n / (1 + alpha * alpha)))
    assert abs(th - ref) < 1e-9


def test_rhs_orthogonal_to_m():
    rng = np.random.default_rng(2)
    m = meshgen.m_random(50, 3)
    H = rng.normal(size=(50, 3))
    assert np.abs(np.einsum("ij,ij->i", llg_rhs(m, H, 0.3), m)).max() < 1e-12 * np.abs(H).max() * GAMMA0
