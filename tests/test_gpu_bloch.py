"""Bloch-phase PGF on the GPU (pmfem_bloch_spectrum, pmfem_bloch_convolve) against the oracle
(oracle/bloch.py): the FP64 spectrum of the twisted grid kernel, and the grid convolution of
quasi-periodic sources in FP64 (1e-11) and FP32 (1e-5), on 1D-, 2D- and 3D-periodic cells, with
FFT lengths from 8 to 256."""
import math

import numpy as np
import pytest

import meshgen
from oracle.bloch import convolve_bloch, twisted_kernel_table
from oracle.paim import AimGrid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _prism():
    p = meshgen.prism_cell(4, 4, 6, jitter=0.15, seed=5)
    return p, (8, 8, 16), np.array([0.0, 0.0, 0.37 * 2 * math.pi / p.periods[2]])


def _film():
    f = meshgen.film_cell(6, 5, 2, seed=4)
    return f, (16, 16, 8), np.array([0.21 * 2 * math.pi / f.periods[0], -0.33 * 2 * math.pi / f.periods[1], 0.0])


def _cube():
    c = meshgen.cube_cell(4, jitter=0.2, seed=3)
    L = c.periods[0]
    return c, (8, 8, 8), np.array([0.1, 0.25, -0.4]) * 2 * math.pi / L


def _prism_long():
    p = meshgen.prism_cell(4, 4, 32, jitter=0.15, seed=6)
    return p, (8, 8, 256), np.array([0.0, 0.0, -0.29 * 2 * math.pi / p.periods[2]])


def _prism_wide():
    p = meshgen.prism_cell(8, 8, 16, jitter=0.15, seed=5)
    return p, (32, 32, 64), np.array([0.0, 0.0, 0.37 * 2 * math.pi / p.periods[2]])


def _film_wide():
    f = meshgen.film_cell(12, 10, 3, seed=4)
    return f, (64, 64, 16), np.array([0.21 * 2 * math.pi / f.periods[0], -0.33 * 2 * math.pi / f.periods[1], 0.0])


# the small cells, and grids of 16-256 points per axis (FFT lengths 16 to 256: every two-factor
# shape of the line transform from 4 x 4 to 16 x 16, several blocks per pass)
CASES = {"prism_1d": _prism, "film_2d": _film, "cube_3d": _cube, "prism_1d_long": _prism_long,
         "prism_1d_wide": _prism_wide, "film_2d_wide": _film_wide}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _setup(name, prec):
    from paper_2409_13958_gb300 import Pmfem
    mesh, grid, k0 = CASES[name]()
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(*grid, 3, 2, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(prec)
    g = AimGrid(h.folded_positions(), mesh.periods, grid, 3)
    dims, fft, origin, delta = h.grid_info()
    assert tuple(dims) == g.dims and tuple(fft) == tuple(g.fft)
    assert np.allclose(origin, g.origin, rtol=0, atol=1e-20) and np.allclose(delta, g.delta, rtol=1e-14)
    return h, g, k0


@pytest.mark.parametrize("name", sorted(CASES))
def test_bloch_spectrum_matches_the_oracle(name):
    h, g, k0 = _setup(name, 0)
    got, max_imag = h.bloch_spectrum(k0)
    want = np.fft.fftn(twisted_kernel_table(g, k0))
    scale = np.abs(want.real).max()
    assert np.abs(want.imag).max() <= 1e-12 * scale          # the kernel is Hermitian
    assert max_imag <= 1e-12 * scale
    assert np.abs(got - want.real.transpose(2, 1, 0)).max() <= 1e-12 * scale
    h.destroy()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bloch_convolution_matches_the_oracle(name, prec, tol):
    h, g, k0 = _setup(name, prec)
    rng = np.random.default_rng(3)
    Q = rng.normal(size=g.dims) + 1j * rng.normal(size=g.dims)
    if prec:
        Q = Q.astype(np.complex64).astype(np.complex128)
    want = convolve_bloch(g, Q, twisted_kernel_table(g, k0))
    ct = torch.complex128 if prec == 0 else torch.complex64
    Qd = torch.tensor(Q.transpose(2, 1, 0).copy(), dtype=ct, device="cuda")       # x fastest
    Ud = torch.empty_like(Qd)
    for _ in range(2):                                                          # the second call reuses the spectrum
        Ud.fill_(float("nan"))
        h.bloch_convolve(k0, Qd, Ud)
        h.sync()
        got = Ud.cpu().numpy().astype(np.complex128).transpose(2, 1, 0)
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= tol, (name, prec, err)
    h.destroy()


def test_bloch_rejects_k0_off_the_periodic_axes_or_on_the_lattice():
    from paper_2409_13958_gb300 import PmfemError
    h, g, k0 = _setup("film_2d", 0)
    for bad in ([0.0, 0.0, 1e8], [2 * math.pi / g.periods[0], 0.0, 0.0]):
        with pytest.raises(PmfemError) as e:
            h.bloch_spectrum(np.array(bad))
        assert e.value.code == -1
    h.destroy()
