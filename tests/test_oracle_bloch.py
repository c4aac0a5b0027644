"""Pins of the Bloch-phase periodic Green's function (oracle/bloch.py, Eq. 15 with k0 != 0)."""
import math

import numpy as np
import pytest

from oracle.bloch import (convolve_bloch, convolve_bloch_direct, pgf_bloch, reg0_bloch,
                          twisted_kernel_table)
from oracle.paim import AimGrid

L = 2.0
CASES = {
    "1d": ((0.0, 0.0, L), np.array([0.0, 0.0, 0.9])),
    "2d": ((L, 1.5, 0.0), np.array([0.7, -1.3, 0.0])),
    "3d": ((L, 1.5, 1.8), np.array([0.4, 1.1, -0.8])),
}


def _pts(seed, n=12, spread=1.0):
    return np.random.default_rng(seed).uniform(-spread, spread, size=(n, 3))


@pytest.mark.parametrize("name", sorted(CASES))
def test_quasi_periodicity(name):
    periods, k0 = CASES[name]
    r = _pts(1)
    g = pgf_bloch(r, periods, k0)
    for a in range(3):
        if periods[a] == 0:
            continue
        for n in (1, -2):
            l = np.zeros(3)
            l[a] = n * periods[a]
            g2 = pgf_bloch(r + l, periods, k0)
            assert np.abs(g2 - np.exp(-1j * k0 @ l) * g).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("name", sorted(CASES))
def test_independent_of_eta(name):
    periods, k0 = CASES[name]
    r = _pts(2)
    per = [p for p in periods if p > 0]
    base = math.sqrt(math.pi) / np.prod(per) ** (1 / len(per))
    ref = pgf_bloch(r, periods, k0, eta=base)
    for s in (0.6, 1.7):
        assert np.abs(pgf_bloch(r, periods, k0, eta=s * base) - ref).max() <= 1e-12 * np.abs(ref).max()
    r0 = reg0_bloch(periods, k0, eta=base)
    assert abs(reg0_bloch(periods, k0, eta=1.7 * base) - r0) <= 1e-12 * abs(r0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_symmetries(name):
    periods, k0 = CASES[name]
    r = _pts(3)
    g = pgf_bloch(r, periods, k0)
    assert np.abs(pgf_bloch(-r, periods, k0) - pgf_bloch(r, periods, -k0)).max() <= 1e-12 * np.abs(g).max()
    assert np.abs(pgf_bloch(r, periods, -k0) - np.conj(g)).max() <= 1e-12 * np.abs(g).max()


def test_1d_against_direct_image_sum():
    """sum_{|i|<=M} e^{-j t i}/|r - i L z| plus the tail of its far images, sum_{|i|>M} e^{-j t i}/(|i| L)
    = (2/L)[-ln(2 sin(t/2)) - sum_{i<=M} cos(t i)/i]; what is left decays as 1/M^2."""
    periods, k0 = CASES["1d"]
    t = k0[2] * L
    r = _pts(4, n=6, spread=0.8)
    M = 4000
    i = np.arange(-M, M + 1)
    img = np.zeros((i.size, 3))
    img[:, 2] = i * L
    d = np.linalg.norm(r[:, None, :] - img[None, :, :], axis=2)
    direct = (np.exp(-1j * t * i)[None, :] / d).sum(axis=1)
    tail = (2 / L) * (-math.log(2 * math.sin(t / 2)) - np.sum(np.cos(t * np.arange(1, M + 1)) / np.arange(1, M + 1)))
    want = direct + tail
    got = pgf_bloch(r, periods, k0)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()


@pytest.mark.parametrize("name", sorted(CASES))
def test_grid_convolution_reproduces_point_sums_at_grid_nodes(name):
    """Charges sitting on grid nodes: u(r_g) = sum_k G_k(r_g - r_k) q_k equals e^{-j k0.r_g} times
    the circular convolution of q~ = q e^{j k0.r_k} with the twisted kernel, by FFT or plain sum."""
    periods, k0 = CASES[name]
    dims = tuple(8 if p > 0 else 6 for p in periods)
    rng = np.random.default_rng(5)
    pos = rng.uniform(0.1, 1.4, size=(20, 3))
    g = AimGrid(pos, periods, dims, 3)
    Kt = twisted_kernel_table(g, k0)
    cells = [(1, 2, 3), (5, 0, 2), (3, 4, 1), (0, 3, 4)]
    q = np.array([1.0, -0.4, 0.7, 0.25])
    Q = np.zeros(dims, dtype=np.complex128)
    node = lambda c: g.origin + np.array(c) * g.delta
    for c, qq in zip(cells, q):
        Q[c] = qq * np.exp(1j * k0 @ node(c))
    U1 = convolve_bloch(g, Q, Kt)
    U2 = convolve_bloch_direct(g, Q, Kt)
    assert np.abs(U1 - U2).max() <= 1e-12 * np.abs(U2).max()
    R0 = reg0_bloch(periods, k0)
    for obs in ((2, 2, 2), (1, 2, 3), (7 if periods[0] else 5, 1, 0)):
        ro = node(obs)
        want = 0
        for c, qq in zip(cells, q):
            want += qq * (R0 if tuple(c) == obs else pgf_bloch((ro - node(c))[None], periods, k0)[0])
        got = np.exp(-1j * k0 @ ro) * U1[obs]
        assert abs(got - want) <= 1e-11 * abs(want)


def test_twisted_kernel_is_hermitian_so_its_spectrum_is_real():
    periods, k0 = CASES["3d"]
    g = AimGrid(np.random.default_rng(6).uniform(0, 1.4, (10, 3)), periods, (8, 8, 8), 3)
    S = np.fft.fftn(twisted_kernel_table(g, k0))
    assert np.abs(S.imag).max() <= 1e-12 * np.abs(S.real).max()
