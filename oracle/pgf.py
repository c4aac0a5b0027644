"""Periodic Green's function G^p of Eq. 15 (static case k0 = 0, G0 = 1/r).

Test infrastructure (see ``oracle/__init__``).

The lattice sums of Eq. 15 are evaluated by Ewald splitting of 1/r with the
Gaussian parameter eta (the paper names only a family of exponentially convergent
sums, without details).
Readings, since the paper fixes no neutralisation convention: the sums diverge (1D,
2D) or are conditionally convergent (3D) for a non-neutral charge set, so the
constant / k = 0 part is the one that makes the result independent of eta:

  3D (volume V):  G3 = sum_l erfc(eta|r+l|)/|r+l| + (4 pi / V) sum_{k!=0} exp(-k^2/4eta^2) cos(k.r)/k^2
                       - pi / (eta^2 V)                                   ("tin-foil")
  2D (area A, z normal to the lattice plane, rho in-plane):
                  G2 = sum_l erfc(eta|r+l|)/|r+l|
                       + (pi/A) sum_{k!=0} cos(k.rho)/k [e^{kz} erfc(k/2eta + eta z) + e^{-kz} erfc(k/2eta - eta z)]
                       - (2 pi / A) [z erf(eta z) + exp(-eta^2 z^2) / (eta sqrt(pi))]
  1D (period L along the axis, rho = distance to the axis, z along it):
                  G1 = sum_l erfc(eta r_l)/r_l + (1/L) [2 ln eta - Ein(eta^2 rho^2)]
                       + (2/L) sum_{j>=1} cos(k_j z) int_0^{eta^2} exp(-rho^2 s - k_j^2 / 4s) ds / s
with Ein(x) = int_0^x (1 - e^-t)/t dt.  Every charge set the method sums over is
neutral (sum_n q_n = 0 exactly), so the constants do not reach the field.

R(0) = lim_{r->0} (G^p(r) - 1/r) is the regular part used for the self term and at
zero grid offset.

Pinned by tests: independence of eta, the 1D / 2D / 3D Madelung constants,
brute-force image sums of neutral clusters, symmetry and periodicity.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.special import erfc, erf, exp1

_CUT_REAL = 6.3      # erfc(6.3) ~ 1e-19
_CUT_SPEC = 43.0     # exp(-43) ~ 2e-19

_GL_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def _gauss_legendre_01(n: int):
    if n not in _GL_CACHE:
        x, w = np.polynomial.legendre.leggauss(n)
        _GL_CACHE[n] = (0.5 * (x + 1.0), 0.5 * w)
    return _GL_CACHE[n]


def ein(x: np.ndarray) -> np.ndarray:
    """Ein(x) = int_0^x (1 - e^-t)/t dt = E1(x) + ln x + gamma (series for small x)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = x < 1.0
    xs = x[small]
    term = xs.copy()
    acc = xs.copy()
    for k in range(2, 40):
        term = -term * xs / k
        acc = acc + term / k
    out[small] = acc
    xl = x[~small]
    out[~small] = exp1(xl) + np.log(xl) + np.euler_gamma
    return out


def spectral_1d(rho: np.ndarray, k: float, eta: float, n: int = 48) -> np.ndarray:
    """int_0^{eta^2} exp(-rho^2 s - k^2/(4 s)) ds / s by Gauss-Legendre in u = s / eta^2."""
    u, w = _gauss_legendre_01(n)
    a = k * k / (4.0 * eta * eta)
    b = (rho * eta) ** 2
    val = np.exp(-b[..., None] * u - a / u) / u
    return val @ w


def default_eta(periods) -> float:
    per = [float(L) for L in periods if L > 0]
    if not per:
        return 0.0
    return math.sqrt(math.pi) / float(np.prod(per)) ** (1.0 / len(per))


def _per_axes(periods):
    return [a for a in range(3) if periods[a] > 0]


def _min_image(r: np.ndarray, periods) -> np.ndarray:
    r = np.array(r, dtype=np.float64, copy=True)
    for a in _per_axes(periods):
        L = float(periods[a])
        r[..., a] -= np.round(r[..., a] / L) * L
    return r


def _real_space(r: np.ndarray, periods, eta: float, exclude_origin: bool) -> np.ndarray:
    """sum over lattice vectors l of erfc(eta |r + l|) / |r + l| (r min-imaged)."""
    per = _per_axes(periods)
    ranges = []
    for a in range(3):
        if a in per:
            n = int(math.ceil(_CUT_REAL / (eta * periods[a]) + 0.5)) + 1
            ranges.append(range(-n, n + 1))
        else:
            ranges.append(range(0, 1))
    out = np.zeros(r.shape[:-1])
    for i, j, k in itertools.product(*ranges):
        l = np.array([i * (periods[0] if 0 in per else 0.0),
                      j * (periods[1] if 1 in per else 0.0),
                      k * (periods[2] if 2 in per else 0.0)])
        if exclude_origin and i == 0 and j == 0 and k == 0:
            continue
        d = np.linalg.norm(r + l, axis=-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = erfc(eta * d) / d
        out += t
    return out


def G3(r: np.ndarray, periods, eta: float | None = None) -> np.ndarray:
    eta = default_eta(periods) if eta is None else eta
    r = _min_image(r, periods)
    V = float(periods[0] * periods[1] * periods[2])
    out = _real_space(r, periods, eta, False)
    kmax = 2.0 * eta * math.sqrt(_CUT_SPEC)
    n = [int(math.ceil(kmax * periods[a] / (2 * math.pi))) for a in range(3)]
    for i, j, k in itertools.product(range(-n[0], n[0] + 1), range(-n[1], n[1] + 1), range(-n[2], n[2] + 1)):
        if i == 0 and j == 0 and k == 0:
            continue
        kv = 2 * math.pi * np.array([i / periods[0], j / periods[1], k / periods[2]])
        k2 = float(kv @ kv)
        out += (4 * math.pi / V) * math.exp(-k2 / (4 * eta * eta)) / k2 * np.cos(r @ kv)
    return out - math.pi / (eta * eta * V)


def G3_reg0(periods, eta: float | None = None) -> float:
    eta = default_eta(periods) if eta is None else eta
    V = float(periods[0] * periods[1] * periods[2])
    out = float(_real_space(np.zeros((1, 3)), periods, eta, True)[0])
    kmax = 2.0 * eta * math.sqrt(_CUT_SPEC)
    n = [int(math.ceil(kmax * periods[a] / (2 * math.pi))) for a in range(3)]
    for i, j, k in itertools.product(range(-n[0], n[0] + 1), range(-n[1], n[1] + 1), range(-n[2], n[2] + 1)):
        if i == 0 and j == 0 and k == 0:
            continue
        kv = 2 * math.pi * np.array([i / periods[0], j / periods[1], k / periods[2]])
        k2 = float(kv @ kv)
        out += (4 * math.pi / V) * math.exp(-k2 / (4 * eta * eta)) / k2
    return out - math.pi / (eta * eta * V) - 2 * eta / math.sqrt(math.pi)


def _split_2d(periods):
    per = _per_axes(periods)
    nrm = [a for a in range(3) if a not in per][0]
    return per, nrm


def _slab_term(k: float, z: np.ndarray, eta: float) -> np.ndarray:
    """e^{kz} erfc(k/2eta + eta z) + e^{-kz} erfc(k/2eta - eta z), overflow-safe."""
    out = np.zeros_like(z)
    for s in (1.0, -1.0):
        a = k / (2 * eta) + s * eta * z
        kz = s * k * z
        # when kz is large the erfc factor is tiny; combine in the log domain
        with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
            e = erfc(a)
            t = np.where(e > 0, np.exp(kz + np.log(np.where(e > 0, e, 1.0))), 0.0)
        out += t
    return out


def G2(r: np.ndarray, periods, eta: float | None = None) -> np.ndarray:
    eta = default_eta(periods) if eta is None else eta
    r = _min_image(r, periods)
    (pa, pb), nz = _split_2d(periods)
    La, Lb = float(periods[pa]), float(periods[pb])
    A = La * Lb
    out = _real_space(r, periods, eta, False)
    z = r[..., nz]
    # for k beyond the Gaussian cut both slab terms are below exp(-_CUT_SPEC) for every z
    kmax = 2.0 * eta * math.sqrt(_CUT_SPEC)
    na = int(math.ceil(kmax * La / (2 * math.pi)))
    nb = int(math.ceil(kmax * Lb / (2 * math.pi)))
    for i, j in itertools.product(range(-na, na + 1), range(-nb, nb + 1)):
        if i == 0 and j == 0:
            continue
        ka, kb = 2 * math.pi * i / La, 2 * math.pi * j / Lb
        k = math.hypot(ka, kb)
        out += (math.pi / A) * np.cos(ka * r[..., pa] + kb * r[..., pb]) / k * _slab_term(k, z, eta)
    out -= (2 * math.pi / A) * (z * erf(eta * z) + np.exp(-(eta * z) ** 2) / (eta * math.sqrt(math.pi)))
    return out


def G2_reg0(periods, eta: float | None = None) -> float:
    eta = default_eta(periods) if eta is None else eta
    (pa, pb), nz = _split_2d(periods)
    La, Lb = float(periods[pa]), float(periods[pb])
    A = La * Lb
    out = float(_real_space(np.zeros((1, 3)), periods, eta, True)[0])
    kmax = 2.0 * eta * math.sqrt(_CUT_SPEC)
    na = int(math.ceil(kmax * La / (2 * math.pi)))
    nb = int(math.ceil(kmax * Lb / (2 * math.pi)))
    for i, j in itertools.product(range(-na, na + 1), range(-nb, nb + 1)):
        if i == 0 and j == 0:
            continue
        k = math.hypot(2 * math.pi * i / La, 2 * math.pi * j / Lb)
        out += (math.pi / A) * 2.0 * math.erfc(k / (2 * eta)) / k
    return out - 2 * math.pi / (A * eta * math.sqrt(math.pi)) - 2 * eta / math.sqrt(math.pi)


def G1(r: np.ndarray, periods, eta: float | None = None) -> np.ndarray:
    eta = default_eta(periods) if eta is None else eta
    r = _min_image(r, periods)
    ax = _per_axes(periods)[0]
    L = float(periods[ax])
    out = _real_space(r, periods, eta, False)
    z = r[..., ax]
    rho = np.sqrt(np.maximum(np.sum(r * r, axis=-1) - z * z, 0.0))
    out += (2.0 * math.log(eta) - ein((eta * rho) ** 2)) / L
    j = 1
    while True:
        k = 2 * math.pi * j / L
        if k * k / (4 * eta * eta) > _CUT_SPEC:
            break
        out += (2.0 / L) * np.cos(k * z) * spectral_1d(rho, k, eta)
        j += 1
    return out


def G1_reg0(periods, eta: float | None = None) -> float:
    eta = default_eta(periods) if eta is None else eta
    ax = _per_axes(periods)[0]
    L = float(periods[ax])
    out = float(_real_space(np.zeros((1, 3)), periods, eta, True)[0])
    out += 2.0 * math.log(eta) / L
    j = 1
    while True:
        k = 2 * math.pi * j / L
        a = k * k / (4 * eta * eta)
        if a > _CUT_SPEC:
            break
        out += (2.0 / L) * float(exp1(a))
        j += 1
    return out - 2 * eta / math.sqrt(math.pi)


def pgf(r: np.ndarray, periods, eta: float | None = None) -> np.ndarray:
    """G^p(r) for displacement rows r (r not on the lattice)."""
    d = len(_per_axes(periods))
    r = np.asarray(r, dtype=np.float64)
    if d == 0:
        return 1.0 / np.linalg.norm(r, axis=-1)
    return {1: G1, 2: G2, 3: G3}[d](r, periods, eta)


def pgf_reg0(periods, eta: float | None = None) -> float:
    """R(0) = lim_{r -> 0} G^p(r) - 1/r (0 for free space)."""
    d = len(_per_axes(periods))
    if d == 0:
        return 0.0
    return {1: G1_reg0, 2: G2_reg0, 3: G3_reg0}[d](periods, eta)
