"""Pins of the anisotropy and per-tetrahedron exchange oracle (oracle/local_terms.py)."""
import math

import numpy as np
import pytest

import meshgen
from oracle import local_terms as LT
from oracle import operators as ops
from oracle.topology import pair_nodes

MS = 8e5


@pytest.fixture(scope="module")
def cell():
    mesh, gr = meshgen.granular_cell(n=5, grains=4, seed=2)
    lca, roots = pair_nodes(mesh.xyz, mesh.periods)
    op = ops.assemble(mesh.xyz, mesh.tets.astype(np.int64), lca, roots.size)
    return mesh, gr, lca, roots.size, op


def test_cubic_energy_closed_forms_and_euler_identity(cell):
    """Uniform m in one grain: e = K1/3 along [111], K1/4 along [110], 0 along [100] (with zero
    field); and for this quartic energy m . de/dm = 4 e, i.e. -(mu0 Ms / 4) sum V_n m . H_n = E."""
    mesh, gr, lca, n, op = cell
    one = np.zeros(mesh.tets.shape[0], np.int32)
    w = LT.grain_weights(mesh.tets, lca, op["vol"], one, n, 1)
    ax = gr.axes[:1]
    K1 = np.array([-4.5e3])
    Vt = op["vol"].sum()
    for comb, e_closed in (((1, 1, 1), K1[0] / 3), ((1, 1, 0), K1[0] / 4), ((1, 0, 0), 0.0)):
        d = np.asarray(comb, float) @ ax[0]
        m = np.tile(d / np.linalg.norm(d), (n, 1))
        H = LT.anisotropy_field(m, w, ax, K1, np.zeros(1), np.zeros((1, 3)), MS)
        E = LT.lumped_energy(m, mesh.tets, lca, op["vol"], one, ax, K1, np.zeros(1), np.zeros((1, 3)))
        assert abs(E - e_closed * Vt) <= 1e-12 * abs(K1[0]) * Vt
        assert abs(-(ops.MU0 * MS / 4) * np.sum(op["V"][:, None] * m * H) - E) <= 1e-12 * abs(K1[0]) * Vt
        if comb == (1, 0, 0):
            assert np.abs(H).max() <= 1e-9
        if comb == (1, 1, 0):
            want = -(2 * K1[0] / (ops.MU0 * MS)) / (2 * math.sqrt(2)) * (ax[0][0] + ax[0][1])
            assert np.abs(H - want[None]).max() <= 1e-12 * np.abs(want).max()


def test_anisotropy_field_is_minus_the_energy_gradient(cell):
    """H_an,n = -(1 / (mu0 Ms V_n)) dE/dm_n for the lumped energy of several grains (finite
    differences on a few unknowns, m not normalised in the perturbation)."""
    mesh, gr, lca, n, op = cell
    w = LT.grain_weights(mesh.tets, lca, op["vol"], gr.tet_grain, n, gr.axes.shape[0])
    Ku = np.linspace(1e3, 3e3, gr.axes.shape[0])
    m = meshgen.m_random(n, seed=3)
    H = LT.anisotropy_field(m, w, gr.axes, gr.K1, Ku, gr.u, MS)
    E = lambda x: LT.lumped_energy(x, mesh.tets, lca, op["vol"], gr.tet_grain, gr.axes, gr.K1, Ku, gr.u)
    mixed = np.nonzero((w > 0).sum(axis=1) > 1)[0]
    assert mixed.size > 0                         # some unknowns sit where grains meet
    for node in list(mixed[:3]) + [int(np.argmax(w.max(axis=1)))]:
        for d in range(3):
            eps = 1e-6
            mp, mm = m.copy(), m.copy()
            mp[node, d] += eps
            mm[node, d] -= eps
            g = (E(mp) - E(mm)) / (2 * eps)
            assert abs(-g / (ops.MU0 * MS * op["V"][node]) - H[node, d]) <= 1e-6 * np.abs(H[node]).max() + 1e-9


def test_uniaxial_closed_form():
    m = meshgen.m_random(50, seed=4)
    u = np.array([0.6, 0.0, 0.8])
    H = LT.uniaxial_field(m, u, 2e4, MS)
    want = 2 * 2e4 / (ops.MU0 * MS) * (m @ u)[:, None] * u[None]
    assert np.abs(H - want).max() <= 1e-12 * np.abs(want).max()


def test_exchange_per_tet(cell):
    mesh, gr, lca, n, op = cell
    A = 1.3e-11
    KA = LT.exchange_matrix_per_tet(mesh.xyz, mesh.tets, lca, n, np.full(mesh.tets.shape[0], A))
    assert abs(KA - A * op["K"]).max() <= 1e-14 * abs(A * op["K"]).max()
    KB = LT.exchange_matrix_per_tet(mesh.xyz, mesh.tets, lca, n, gr.A_tet)
    assert np.abs(KB @ np.ones(n)).max() <= 1e-12 * abs(KB).max()
    assert abs(KB - KB.T).max() <= 1e-14 * abs(KB).max()
    assert 0 < (gr.A_tet < A).mean() < 1          # a boundary layer, not all of the cell
    m = meshgen.m_random(n, seed=5)
    H = LT.exchange_field_per_tet(KA, op["V"], m, MS)
    assert np.abs(H - ops.exchange_field(op["K"], op["V"], m, A, MS)).max() <= 1e-12 * np.abs(H).max()
