"""Bloch-phase periodic Green's function (Eq. 15 with k0 != 0) and its grid convolution.

Test infrastructure (see ``oracle/__init__``).

Eq. 15 with a phase per image: G_k(r) = sum_l e^{-j k0 . l} / |r - l| over the lattice vectors
l of the periodic axes (k0 has components only along them).  It is quasi-periodic,
G_k(r + l) = e^{-j k0 . l} G_k(r), and is the potential kernel of sources that repeat with the
same phase (phase-shifted excitation, spin-wave band problems, Sec. 4.3).  For k0 off the
reciprocal lattice no neutralisation is needed.  Ewald splitting with parameter eta, Poisson
summation of the smooth part (the phase shifts every reciprocal vector G to G + k0):
  3D (volume V):   sum_l e^{-jk0.l} erfc(eta|r-l|)/|r-l|
                   + (4 pi / V) sum_G e^{-j(G+k0).r} e^{-|G+k0|^2/4eta^2} / |G+k0|^2
  2D (area A, z open):  sum_l ... + (pi / A) sum_G e^{-j(G+k0).rho} / k [e^{kz} erfc(k/2eta + eta z)
                   + e^{-kz} erfc(k/2eta - eta z)],  k = |G + k0|
  1D (period L along the axis, rho = distance to it):  sum_l ... + (1/L) sum_m e^{-j(k_m+k0) z}
                   int_0^{eta^2} exp(-rho^2 s - (k_m+k0)^2 / 4s) ds / s,  k_m = 2 pi m / L
with the same truncations as the k0 = 0 sums (``pgf``).  R_k(0) = lim (G_k - 1/r) is the self
term.

Grid form (reading; the paper adapts its periodic method to this case without details): with
q~_k = q_k e^{j k0 . r_k} and the periodic kernel K~(d) = G_k(d) e^{j k0 . d}, the potential
u(r) = sum_k G_k(r - r_k) q_k equals e^{-j k0 . r} sum_k K~(r - r_k) q~_k, a circular
convolution on the grid of Eq. 16 (periodic axes; open axes zero-padded as for k0 = 0).  K~ is
Hermitian, K~(-d) = conj(K~(d)), so its discrete Fourier transform is real.

Pinned by tests: quasi-periodicity, independence of eta, the symmetry G_k(-r) = G_{-k}(r) =
conj(G_k(r)), in 1D a direct image sum whose slowly decaying tail is summed in closed form,
sum_{i>=1} cos(i t)/i = -ln(2 sin(t/2)); the grid form reproduces the point sums exactly for
charges on grid nodes, and the twisted kernel's spectrum is real.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.special import erfc

from .pgf import _CUT_REAL, _CUT_SPEC, _per_axes, default_eta

_GL16 = np.polynomial.legendre.leggauss(16)


def spectral_1d_any(rho, k, eta):
    """int_0^{eta^2} exp(-rho^2 s - k^2/(4 s)) ds / s for any k > 0.  With s = eta^2 e^{-t} it is
    int_0^inf exp(-b e^{-t} - a e^{t}) dt, a = k^2/(4 eta^2), b = (rho eta)^2: a smooth bell in t
    that has fallen below e^{-45} once a e^t > 45; summed by 16-point Gauss-Legendre on unit
    panels of t (the k0 = 0 sums use one Gauss-Legendre rule in s, which loses accuracy when
    a is small, as it is for the phase-shifted wavenumber nearest zero)."""
    a = k * k / (4.0 * eta * eta)
    b = (np.asarray(rho, dtype=np.float64) * eta) ** 2
    T = max(1.0, math.log(45.0 / a) + 1.0) if a < 45.0 else 1.0
    npan = int(math.ceil(T))
    x, w = _GL16
    out = np.zeros(b.shape)
    for p in range(npan):
        t = p + 0.5 * (x + 1.0)
        val = np.exp(-b[..., None] * np.exp(-t) - a * np.exp(t))
        out += 0.5 * (val @ w)
    return out


def _phase_images(periods, eta, r):
    per = _per_axes(periods)
    ranges = []
    for a in range(3):
        if a in per:
            # images far enough that erfc(eta |r - l|) is negligible for any r within the images
            ext = float(np.max(np.abs(r[..., a]))) if r.size else 0.0
            n = int(math.ceil((_CUT_REAL / eta + ext) / periods[a])) + 1
            ranges.append(range(-n, n + 1))
        else:
            ranges.append(range(0, 1))
    return itertools.product(*ranges)


def _real_space_bloch(r, periods, k0, eta, exclude_origin):
    out = np.zeros(r.shape[:-1], dtype=np.complex128)
    for i, j, k in _phase_images(periods, eta, r):
        l = np.array([i * periods[0], j * periods[1], k * periods[2]])
        if exclude_origin and not (i or j or k):
            continue
        d = np.linalg.norm(r - l, axis=-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = erfc(eta * d) / d
        out += np.exp(-1j * float(np.dot(k0, l))) * t
    return out


def _kvecs(periods, k0, eta, dims):
    """Shifted reciprocal vectors G + k0 (rows) within the Gaussian cut."""
    per = _per_axes(periods)
    kmax = 2.0 * eta * math.sqrt(_CUT_SPEC)
    rng = []
    for a in range(3):
        if a in per:
            n = int(math.ceil((kmax + abs(k0[a])) * periods[a] / (2 * math.pi))) + 1
            rng.append(range(-n, n + 1))
        else:
            rng.append(range(0, 1))
    out = []
    for idx in itertools.product(*rng):
        g = np.array([2 * math.pi * idx[a] / periods[a] if a in per else 0.0 for a in range(3)]) + k0
        if float(g @ g) / (4 * eta * eta) <= _CUT_SPEC and dims >= 1:
            out.append(g)
    return np.array(out) if out else np.zeros((0, 3))


def pgf_bloch(r, periods, k0, eta=None, exclude_origin=False):
    """G_k(r) (complex) for displacement rows r; exclude_origin drops the l = 0 image of the
    real-space sum (then r = 0 is allowed and the sum is G_k - 1/r's regular part minus the
    Gaussian self term, see reg0_bloch)."""
    periods = tuple(float(L) for L in periods)
    k0 = np.asarray(k0, dtype=np.float64)
    per = _per_axes(periods)
    assert all(k0[a] == 0 for a in range(3) if a not in per), "k0 must lie along the periodic axes"
    eta = default_eta(periods) if eta is None else eta
    r = np.asarray(r, dtype=np.float64)
    out = _real_space_bloch(r, periods, k0, eta, exclude_origin)
    d = len(per)
    kv = _kvecs(periods, k0, eta, d)
    if d == 3:
        V = periods[0] * periods[1] * periods[2]
        for g in kv:
            k2 = float(g @ g)
            out += (4 * math.pi / V) * math.exp(-k2 / (4 * eta * eta)) / k2 * np.exp(-1j * (r @ g))
    elif d == 2:
        nz = [a for a in range(3) if a not in per][0]
        A = periods[per[0]] * periods[per[1]]
        z = r[..., nz]
        for g in kv:
            k = math.sqrt(float(g @ g))
            slab = np.zeros(z.shape)
            for s in (1.0, -1.0):
                e = erfc(k / (2 * eta) + s * eta * z)
                with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
                    slab += np.where(e > 0, np.exp(s * k * z + np.log(np.where(e > 0, e, 1.0))), 0.0)
            out += (math.pi / A) / k * np.exp(-1j * (r @ g)) * slab
    else:
        ax = per[0]
        L = periods[ax]
        z = r[..., ax]
        rho = np.sqrt(np.maximum(np.sum(r * r, axis=-1) - z * z, 0.0))
        for g in kv:
            k = abs(float(g[ax]))
            out += (1.0 / L) * np.exp(-1j * g[ax] * z) * spectral_1d_any(rho, k, eta)
    return out


def reg0_bloch(periods, k0, eta=None):
    """R_k(0) = lim_{r -> 0} G_k(r) - 1/r."""
    eta = default_eta(periods) if eta is None else eta
    v = pgf_bloch(np.zeros((1, 3)), periods, k0, eta, exclude_origin=True)[0]
    return v - 2 * eta / math.sqrt(math.pi)


def twisted_kernel_table(grid, k0, eta=None):
    """K~ on the grid's FFT index space: K~(d) = G_k(d Delta) e^{j k0 . d Delta}, K~(0) = R_k(0);
    open axes laid out as for k0 = 0 (zero beyond the node grid, zero at index N)."""
    F = grid.fft
    idx = [np.arange(F[a]) for a in range(3)]
    offs, valid = [], []
    for a in range(3):
        N = grid.dims[a]
        j = idx[a]
        if grid.periodic[a]:
            d = np.where(j <= N // 2, j, j - N)           # signed offset (circular)
            valid.append(np.ones(F[a], bool))
        else:
            d = np.where(j < N, j, j - 2 * N)
            valid.append(j != N)
        offs.append(d)
    D = np.stack(np.meshgrid(*[offs[a] * grid.delta[a] for a in range(3)], indexing="ij"), -1).reshape(-1, 3)
    zero = np.all(D == 0.0, axis=1)
    K = np.zeros(D.shape[0], dtype=np.complex128)
    if np.any(~zero):
        K[~zero] = pgf_bloch(D[~zero], grid.periods, k0, eta) * np.exp(1j * (D[~zero] @ np.asarray(k0, float)))
    K[zero] = reg0_bloch(grid.periods, k0, eta)
    K = K.reshape(F)
    return K * valid[0][:, None, None] * valid[1][None, :, None] * valid[2][None, None, :]


def convolve_bloch(grid, Qt, Kt):
    """U~ = IFFT(FFT(K~) FFT(Q~)) on the node grid (complex Q~)."""
    Nx, Ny, Nz = grid.dims
    Qp = np.zeros(grid.fft, dtype=np.complex128)
    Qp[:Nx, :Ny, :Nz] = Qt
    return np.fft.ifftn(np.fft.fftn(Kt) * np.fft.fftn(Qp))[:Nx, :Ny, :Nz]


def convolve_bloch_direct(grid, Qt, Kt):
    """Plain grid sum U~_g = sum_g' K~(g - g') Q~_g' (small grids only)."""
    Nx, Ny, Nz = grid.dims
    U = np.zeros(grid.dims, dtype=np.complex128)
    for (i, j, k) in np.argwhere(Qt != 0):
        ix = (np.arange(Nx) - i) % grid.fft[0]
        iy = (np.arange(Ny) - j) % grid.fft[1]
        iz = (np.arange(Nz) - k) % grid.fft[2]
        U += Qt[i, j, k] * Kt[np.ix_(ix, iy, iz)]
    return U
