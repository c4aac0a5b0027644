"""Pins of the implicit midpoint Newton-Krylov oracle (oracle/implicit.py)."""
import math

import numpy as np
import pytest

import meshgen
from oracle.implicit import MidpointStepper, block_preconditioner, llg_jvp
from oracle.llg import llg_rhs, rk4_step
from oracle.operators import MU0
from oracle.problem import GAMMA0, OracleProblem


def _spin_stepper(H, alpha):
    H = np.asarray(H, dtype=float)
    return MidpointStepper(lambda m: np.broadcast_to(H, m.shape).copy(), lambda v: np.zeros_like(v),
                           np.zeros(1), alpha)


def test_single_spin_turns_by_the_cayley_angle():
    """alpha = 0, uniform H along z: the midpoint rule is the Cayley transform of the rotation
    about z at rate gamma0 H, i.e. exactly 2 atan(gamma0 H dt / 2) per step."""
    Hz, dt, steps = 8e4, 3e-11, 7
    st = _spin_stepper((0.0, 0.0, Hz), 0.0)
    m = np.array([[math.cos(0.3), math.sin(0.3), 0.0]])
    for _ in range(steps):
        m = st.step(m, dt)
    theta = 2 * math.atan(GAMMA0 * Hz * dt / 2)
    want = np.array([[math.cos(0.3 + steps * theta), math.sin(0.3 + steps * theta), 0.0]])
    assert np.abs(m - want).max() < 1e-12
    assert abs(theta - GAMMA0 * Hz * dt) > 5e-3            # a large step: far from the exact rate


def test_damped_spin_converges_at_second_order():
    """Closed form of a damped spin in a uniform field: tan(theta/2) = tan(theta0/2) e^{-alpha g H t},
    phi = phi0 + g H t, g = gamma0 / (1 + alpha^2)."""
    Hz, alpha, T = 5e4, 0.1, 2e-10
    g = GAMMA0 / (1 + alpha * alpha)
    th0, ph0 = 1.0, 0.2

    def exact(t):
        th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * g * Hz * t))
        ph = ph0 + g * Hz * t
        return np.array([[math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)]])

    errs = []
    for n in (40, 80, 160):
        st = _spin_stepper((0.0, 0.0, Hz), alpha)
        m = exact(0.0)
        for _ in range(n):
            m = st.step(m, T / n)
        errs.append(np.abs(m - exact(T)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, (errs, r1, r2)


@pytest.fixture(scope="module")
def film():
    mesh = meshgen.film_cell(8, 8, 2, seed=3)
    pb = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, grid=(16, 16, 8), near_boxes=3, H_ap=(1e4, 0, 2e4))
    K = pb.K.tocsr()
    c = -(2 * pb.A / (MU0 * pb.Ms)) * K.diagonal() / pb.V
    return pb, c


def _stepper(pb, c, **kw):
    return MidpointStepper(lambda m: pb.h_eff(m, "paim"), lambda v: pb.h_eff(v, "paim", ap=False), c, pb.alpha, **kw)


def test_jacobian_product_matches_finite_differences(film):
    pb, c = film
    m = meshgen.m_random(pb.Np, seed=4)
    v = meshgen.m_random(pb.Np, seed=5)
    eps = 1e-6
    f = lambda x: llg_rhs(x, pb.h_eff(x, "paim"), pb.alpha)
    fd = (f(m + eps * v) - f(m - eps * v)) / (2 * eps)
    jv = llg_jvp(m, pb.h_eff(m, "paim"), pb.h_eff(v, "paim", ap=False), v, pb.alpha)
    assert np.linalg.norm(jv - fd) <= 1e-8 * np.linalg.norm(fd)


def test_block_preconditioner_is_the_local_jacobian(film):
    """With the linear field replaced by its diagonal, the 3x3 blocks reproduce J v exactly."""
    pb, c = film
    m = meshgen.m_random(pb.Np, seed=6)
    H = pb.h_eff(m, "paim")
    v = meshgen.m_random(pb.Np, seed=7)
    dt = 1e-13
    P = block_preconditioner(m, H, c, dt, pb.alpha)
    Jv = v - 0.5 * dt * llg_jvp(m, H, c[:, None] * v, v, pb.alpha)
    assert np.abs(np.einsum("nij,nj->ni", P, v) - Jv).max() <= 1e-13 * np.abs(Jv).max()


def test_midpoint_keeps_the_norm_and_matches_rk4_for_small_steps(film):
    pb, c = film
    m0 = meshgen.m_random(pb.Np, seed=8)
    st = _stepper(pb, c)
    m = m0
    for _ in range(3):
        m = st.step(m, 1e-13)            # about 4 / (gamma0 |exchange diagonal|): beyond RK4's stable step
    assert np.abs(np.linalg.norm(m, axis=1) - 1).max() < 1e-11
    assert st.newton_its >= 3 and st.krylov_its > 0
    rel = []
    for dt in (4e-15, 2e-15):           # one step each: midpoint and RK4 differ by O(dt^3)
        a = _stepper(pb, c).step(m0, dt)
        b = rk4_step(m0, dt, lambda x: pb.h_eff(x, "paim"), pb.alpha)
        rel.append(np.linalg.norm(a - b) / np.linalg.norm(b - m0))
    assert rel[0] < 1e-3 and 3.5 < rel[0] / rel[1] < 4.5, rel
