"""Pins of the oracle's periodic Green's function (Eq. 15) against textbook facts."""
import itertools
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.pgf import default_eta, pgf, pgf_reg0, spectral_1d, ein


A = 1.3  # lattice spacing (arbitrary units)


def site_potential(periods, charges):
    """Potential at charges[0] from all charges and all their images."""
    r0, q0 = charges[0]
    phi = pgf_reg0(periods) * q0
    for r, q in charges[1:]:
        phi += q * pgf(np.array([np.subtract(r0, r)]), periods)[0]
    return phi


def test_madelung_1d_chain():
    # alternating +-1 chain, spacing a: site potential -2 ln 2 / a
    phi = site_potential((0.0, 0.0, 2 * A), [((0, 0, 0), 1.0), ((0, 0, A), -1.0)])
    assert abs(phi * A + 2 * math.log(2)) < 1e-12


def test_madelung_2d_square():
    # checkerboard square lattice: site potential -1.6155426267128 / a
    ch = [((0, 0, 0), 1.0), ((A, A, 0), 1.0), ((A, 0, 0), -1.0), ((0, A, 0), -1.0)]
    phi = site_potential((2 * A, 2 * A, 0.0), ch)
    assert abs(phi * A + 1.6155426267128) < 1e-11


def test_madelung_3d_rocksalt():
    # NaCl: site potential -1.747564594633182 / a
    ch = [((i * A, j * A, k * A), (-1.0) ** (i + j + k)) for i in range(2) for j in range(2) for k in range(2)]
    phi = site_potential((2 * A,) * 3, ch)
    assert abs(phi * A + 1.747564594633182) < 1e-11


@pytest.mark.parametrize("periods", [(0, 0, 2.6), (0, 3.0, 0), (2.6, 2.6, 0), (2.0, 3.0, 0), (0, 2.0, 2.5),
                                     (2.6, 2.6, 2.6), (1.5, 2.0, 2.5)])
def test_eta_independence(periods):
    rng = np.random.default_rng(0)
    r = rng.uniform(-2, 2, size=(100, 3))
    e0 = default_eta(periods)
    g = [pgf(r, periods, eta=e0 * f) for f in (0.5, 1.0, 2.0)]
    scale = np.abs(g[1]).max()
    assert np.abs(g[0] - g[1]).max() / scale < 1e-12
    assert np.abs(g[2] - g[1]).max() / scale < 1e-12
    r0 = [pgf_reg0(periods, eta=e0 * f) for f in (0.5, 1.0, 2.0)]
    assert abs(r0[0] - r0[1]) < 1e-12 * (1 + abs(r0[1])) and abs(r0[2] - r0[1]) < 1e-12 * (1 + abs(r0[1]))


@pytest.mark.parametrize("periods", [(0, 0, 2.6), (2.6, 2.0, 0), (2.6, 2.6, 2.6), (1.5, 2.0, 2.5)])
def test_symmetry_and_periodicity(periods):
    rng = np.random.default_rng(1)
    r = rng.uniform(-1.2, 1.2, size=(50, 3))
    g = pgf(r, periods)
    assert np.allclose(pgf(-r, periods), g, rtol=1e-13, atol=1e-14)
    for a in range(3):
        if periods[a] > 0:
            s = r.copy()
            s[:, a] += periods[a]
            assert np.allclose(pgf(s, periods), g, rtol=1e-13, atol=1e-14)
        # reflection in one axis (orthogonal lattice)
        s = r.copy()
        s[:, a] = -s[:, a]
        assert np.allclose(pgf(s, periods), g, rtol=1e-13, atol=1e-14)


def _richardson(vals, Ms, order):
    # vals(M) = S + c / M^order: eliminate from the last two
    (m1, v1), (m2, v2) = (Ms[-2], vals[-2]), (Ms[-1], vals[-1])
    f = (m2 / m1) ** order
    return (f * v2 - v1) / (f - 1)


def test_brute_force_1d():
    L = 2.0
    cl = [((0.1, 0.2, 0.3), 1.0), ((-0.3, 0.1, -0.4), -2.0), ((0.2, -0.2, 0.7), 1.0)]
    obs = np.array([[0.5, -0.4, 0.1], [-0.2, 0.6, -0.8]])
    exact = sum(q * pgf(obs - np.array(r), (0, 0, L)) for r, q in cl)
    Ms = [2000, 4000]
    vals = []
    for Mx in Ms:
        l = np.arange(-Mx, Mx + 1) * L
        s = 0.0
        for r, q in cl:
            d = obs[:, None, :] - np.array(r)[None, None, :]
            d = d + np.stack([np.zeros_like(l), np.zeros_like(l), -l], axis=1)[None]
            s = s + q * (1.0 / np.linalg.norm(d, axis=2)).sum(axis=1)
        vals.append(s)
    bf = _richardson(vals, Ms, 2)
    assert np.abs(bf - exact).max() < 1e-8


def test_brute_force_2d_differences():
    L = (2.0, 2.5, 0.0)
    # neutral, dipole-free cluster
    cl = [((0.3, 0.0, 0.1), 1.0), ((-0.3, 0.0, 0.1), 1.0), ((0.0, 0.2, -0.2), -1.0), ((0.0, -0.2, -0.2), -1.0)]
    obs = np.array([[0.7, 0.4, 0.5], [-0.5, -0.9, -0.3]])
    exact = sum(q * pgf(obs - np.array(r), L) for r, q in cl)
    Rs = [200.0, 400.0]
    vals = []
    for R in Rs:
        nx, ny = int(R / L[0]) + 1, int(R / L[1]) + 1
        I, J = np.meshgrid(np.arange(-nx, nx + 1), np.arange(-ny, ny + 1), indexing="ij")
        lv = np.stack([I.ravel() * L[0], J.ravel() * L[1], np.zeros(I.size)], axis=1)
        lv = lv[np.linalg.norm(lv, axis=1) <= R]
        s = 0.0
        for r, q in cl:
            d = obs[:, None, :] - np.array(r)[None, None, :] - lv[None]
            s = s + q * (1.0 / np.linalg.norm(d, axis=2)).sum(axis=1)
        vals.append(s)
    bf = _richardson(vals, Rs, 1)
    assert abs((bf[0] - bf[1]) - (exact[0] - exact[1])) < 1e-6


def test_brute_force_3d_differences():
    L = (2.0, 2.0, 2.0)
    cl = [((0.3, 0.0, 0.1), 1.0), ((-0.3, 0.0, 0.1), 1.0), ((0.0, 0.2, -0.2), -1.0), ((0.0, -0.2, -0.2), -1.0)]
    obs = np.array([[0.7, 0.4, 0.5], [-0.5, -0.9, -0.3]])
    exact = sum(q * pgf(obs - np.array(r), L) for r, q in cl)
    Rs = [24.0, 48.0]
    vals = []
    for R in Rs:
        n = int(R / 2.0) + 1
        g = np.arange(-n, n + 1) * 2.0
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        lv = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        lv = lv[np.linalg.norm(lv, axis=1) <= R]
        s = 0.0
        for r, q in cl:
            d = obs[:, None, :] - np.array(r)[None, None, :] - lv[None]
            s = s + q * (1.0 / np.linalg.norm(d, axis=2)).sum(axis=1)
        vals.append(s)
    bf = _richardson(vals, Rs, 2)
    # spherical summation order adds the surface term (4 pi / 3V) p . r to the tin-foil
    # (Ewald, k = 0 dropped) potential of a neutral cluster with dipole p
    p = sum(q * np.array(r) for r, q in cl)
    surf = 4 * math.pi / (3 * 8.0) * float(p @ (obs[0] - obs[1]))
    assert abs(p[2]) > 0.1
    assert abs((bf[0] - bf[1]) - (exact[0] - exact[1]) - surf) < 1e-5


def test_spectral_1d_quadrature():
    eta = math.sqrt(math.pi) / 2.0
    for rho in (0.0, 0.1, 1.0, 3.0):
        for k in (math.pi, 2 * math.pi, 3 * math.pi):
            ref = quad(lambda s: math.exp(-rho * rho * s - k * k / (4 * s)) / s, 0, eta * eta,
                       epsabs=0, epsrel=1e-13, limit=200)[0]
            val = spectral_1d(np.array([rho]), k, eta)[0]
            assert abs(val - ref) <= 1e-13 * ref + 1e-300


def test_ein_matches_integral():
    for x in (1e-6, 0.3, 0.99, 1.0, 2.5, 17.0):
        ref = quad(lambda t: -math.expm1(-t) / t, 0, x, epsabs=0, epsrel=1e-13)[0]
        assert abs(ein(np.array([x]))[0] - ref) < 1e-13 * max(1.0, ref)
