"""O2: the periodic adaptive-integral method (BAIM steps 1-4 of Sec. 3.2).

Test infrastructure (see ``oracle/__init__``).

Grid (Eq. 16, read per axis; the printed formula reuses Delta_x for y and z and
ignores periodicity):
  periodic axis:      Delta = L / N, origin = smallest folded coordinate, indices wrap mod N;
  non-periodic axis:  margin m = ceil((p+1)/2) cells each side, Delta = D / (N - 1 - 2m),
                      origin = smallest coordinate - m Delta, FFT length 2N (linear
                      convolution by zero padding; periodic axes need none, Sec. 4.5).
Stencil of order p: t = (x - origin) / Delta; base = floor(t) - (p-1)/2 for odd p,
round-half-down(t) - p/2 for even p; points base..base+p with 1D Lagrange weights,
tensor product in 3D.  Projection (step 1) is the transpose of interpolation (step 3).
Grid kernel (step 2, Sec. 3.2: the periodic G^p takes the place of G0): K(d) = G^p(d Delta), K(0) = R(0).
Precorrection (step 4, only G0 is corrected, Sec. 3.2): for every source image
(k, l) whose box lies within Chebyshev distance near_boxes of the observer's box
(periodic wrap gives the expanded regions of Eq. 17),
  C_nk += G0(r_n - r_k - l) [skipped for the self pair]
          - sum_{a in S(n)} sum_{b in S(k)} w_na w_kb G0'(r_a - r_b - l),   G0'(0) = 0.
Potential: 4 pi u = interp(IFFT(FFT(K) FFT(project(q)))) + C q + E M.

Pinned by tests: the FFT convolution equals the plain grid sum on small grids;
Lagrange weights reproduce polynomials of degree p; O2 converges to O1 as the grid
is refined (method error <= 1e-3).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

from .pgf import pgf, pgf_reg0


def lagrange_weights(s: np.ndarray, p: int) -> np.ndarray:
    """w_i(s) = prod_{j != i} (s - j) / (i - j) for i = 0..p; s shape (...,) -> (..., p+1)."""
    out = np.ones(s.shape + (p + 1,))
    for i in range(p + 1):
        for j in range(p + 1):
            if j != i:
                out[..., i] *= (s - j) / (i - j)
    return out


class AimGrid:
    def __init__(self, pos_f: np.ndarray, periods, dims, p: int = 3):
        self.p = int(p)
        self.dims = tuple(int(n) for n in dims)
        self.periods = tuple(float(L) for L in periods)
        self.periodic = [L > 0 for L in self.periods]
        self.delta = np.zeros(3)
        self.origin = np.zeros(3)
        self.fft = []
        m = int(math.ceil((self.p + 1) / 2))
        for a in range(3):
            N = self.dims[a]
            lo, hi = float(pos_f[:, a].min()), float(pos_f[:, a].max())
            if self.periodic[a]:
                self.delta[a] = self.periods[a] / N
                self.origin[a] = lo
                self.fft.append(N)
            else:
                self.delta[a] = (hi - lo) / (N - 1 - 2 * m)
                self.origin[a] = lo - m * self.delta[a]
                self.fft.append(2 * N)

    def stencil(self, pos: np.ndarray):
        """base (M, 3) int64 unwrapped, local coordinate s (M, 3), weights (M, 3, p+1)."""
        t = (pos - self.origin) / self.delta
        if self.p % 2 == 1:
            base = np.floor(t).astype(np.int64) - (self.p - 1) // 2
        else:
            base = np.ceil(t - 0.5).astype(np.int64) - self.p // 2
        s = t - base
        return base, s, lagrange_weights(s, self.p)

    def boxes(self, pos: np.ndarray) -> np.ndarray:
        return np.floor((pos - self.origin) / self.delta).astype(np.int64)

    def flat(self, pos: np.ndarray):
        """Wrapped linear indices (M, (p+1)^3) into an (Nx, Ny, Nz) array and weights."""
        base, _, w = self.stencil(pos)
        P = self.p + 1
        idx = np.zeros((pos.shape[0], P, P, P), dtype=np.int64)
        wt = np.ones((pos.shape[0], P, P, P))
        Nx, Ny, Nz = self.dims
        ii = [(base[:, a][:, None] + np.arange(P)[None, :]) for a in range(3)]
        for a in range(3):
            if self.periodic[a]:
                ii[a] = np.mod(ii[a], self.dims[a])
            assert ii[a].min() >= 0 and ii[a].max() < self.dims[a], "stencil leaves the grid"
        idx = (ii[0][:, :, None, None] * Ny + ii[1][:, None, :, None]) * Nz + ii[2][:, None, None, :]
        wt = w[:, 0, :, None, None] * w[:, 1, None, :, None] * w[:, 2, None, None, :]
        return idx.reshape(pos.shape[0], -1), wt.reshape(pos.shape[0], -1)

    # -------------------------------------------------------------- step 2 kernel
    def kernel_table(self, eta=None) -> np.ndarray:
        """K on the FFT index space (Fx, Fy, Fz): K(d) = G^p(d Delta), K(0) = R(0).

        Uses the reflection symmetry of G^p in each axis (orthogonal lattice): values are
        computed on non-negative offsets and mirrored.
        """
        uniq = []
        for a in range(3):
            N = self.dims[a]
            uniq.append(np.arange(N // 2 + 1) if self.periodic[a] else np.arange(N))
        D = np.stack(np.meshgrid(*[u * self.delta[a] for a, u in enumerate(uniq)], indexing="ij"), axis=-1)
        flatD = D.reshape(-1, 3)
        vals = np.empty(flatD.shape[0])
        zero = np.all(flatD == 0.0, axis=1)
        if np.any(~zero):
            vals[~zero] = pgf(flatD[~zero], self.periods, eta)
        vals[zero] = pgf_reg0(self.periods, eta)
        Ku = vals.reshape(D.shape[:3])
        maps = []
        valid = []
        for a in range(3):
            F = self.fft[a]
            j = np.arange(F)
            N = self.dims[a]
            if self.periodic[a]:
                d = np.minimum(j, N - j)
                maps.append(d)
                valid.append(np.ones(F, bool))
            else:
                d = np.where(j < N, j, 2 * N - j)
                valid.append(j != N)
                maps.append(np.where(j == N, 0, d))
        K = Ku[np.ix_(maps[0], maps[1], maps[2])]
        K = K * valid[0][:, None, None] * valid[1][None, :, None] * valid[2][None, None, :]
        return K

    def convolve(self, Q: np.ndarray, Khat: np.ndarray) -> np.ndarray:
        """U = IFFT(Khat FFT(Q)) restricted to the node grid."""
        Nx, Ny, Nz = self.dims
        Qp = np.zeros(self.fft)
        Qp[:Nx, :Ny, :Nz] = Q
        U = np.fft.irfftn(np.fft.rfftn(Qp) * Khat, s=self.fft, axes=(0, 1, 2))
        return U[:Nx, :Ny, :Nz]

    def convolve_direct(self, Q: np.ndarray, K: np.ndarray) -> np.ndarray:
        """Plain grid sum U_g = sum_g' K(g - g') Q_g' (small grids only)."""
        Nx, Ny, Nz = self.dims
        U = np.zeros(self.dims)
        src = np.argwhere(Q != 0)
        for (i, j, k) in src:
            ix = (np.arange(Nx) - i) % self.fft[0]
            iy = (np.arange(Ny) - j) % self.fft[1]
            iz = (np.arange(Nz) - k) % self.fft[2]
            U += Q[i, j, k] * K[np.ix_(ix, iy, iz)]
        return U


def box_near_pairs(grid: AimGrid, pos_f: np.ndarray, near_boxes: int, observers=None):
    """(n, k, lvec (P,3), limg (P,3) integer image counts) for box-near source images."""
    N = np.array(grid.dims)
    b = grid.boxes(pos_f)
    buckets: dict[tuple, list[int]] = {}
    for k, bb in enumerate(map(tuple, b.tolist())):
        buckets.setdefault(bb, []).append(k)
    obs = range(pos_f.shape[0]) if observers is None else observers
    rn, rk, rl = [], [], []
    rng = range(-near_boxes, near_boxes + 1)
    for n in obs:
        bn = b[n]
        for off in itertools.product(rng, rng, rng):
            t = bn + np.array(off)
            img = np.zeros(3, dtype=np.int64)
            ok = True
            for a in range(3):
                if grid.periodic[a]:
                    img[a] = t[a] // N[a]
                    t[a] = t[a] - img[a] * N[a]
                elif t[a] < 0 or t[a] >= N[a]:
                    ok = False
            if not ok:
                continue
            for k in buckets.get(tuple(t.tolist()), ()):
                rn.append(n); rk.append(k); rl.append(img.copy())
    if not rn:
        return np.zeros(0, int), np.zeros(0, int), np.zeros((0, 3)), np.zeros((0, 3), int)
    limg = np.array(rl, dtype=np.int64)
    lvec = limg * np.array([grid.periods[a] if grid.periodic[a] else 0.0 for a in range(3)])
    return np.array(rn), np.array(rk), lvec, limg


def precorrection_matrix(grid: AimGrid, pos_f: np.ndarray, near_boxes: int, observers=None, chunk=256):
    """C (csr, N' x N') of step 4: exact point G0 minus the grid's G0 for box-near pairs."""
    n, k, lvec, limg = box_near_pairs(grid, pos_f, near_boxes, observers)
    Np = pos_f.shape[0]
    vals = np.zeros(n.size)
    if n.size == 0:
        return sp.csr_matrix((Np, Np))
    d = pos_f[n] - pos_f[k] - lvec
    dist = np.linalg.norm(d, axis=1)
    is_self = (n == k) & np.all(limg == 0, axis=1)
    vals += np.where(is_self, 0.0, 1.0 / np.where(is_self, 1.0, dist))
    base, _, w = grid.stencil(pos_f)
    P = grid.p + 1
    ar = np.arange(P)
    Nv = np.array(grid.dims)
    for s in range(0, n.size, chunk):
        nn, kk, li = n[s:s + chunk], k[s:s + chunk], limg[s:s + chunk]
        # unwrapped grid offsets a - b - l N along each axis: (B, P, P)
        off = []
        for a in range(3):
            ia = base[nn, a][:, None] + ar[None, :]                     # observer stencil
            ib = base[kk, a][:, None] + ar[None, :] + li[:, a][:, None] * Nv[a]  # source image stencil
            off.append((ia[:, :, None] - ib[:, None, :]) * grid.delta[a])
        ox = off[0][:, :, None, None, :, None, None]
        oy = off[1][:, None, :, None, None, :, None]
        oz = off[2][:, None, None, :, None, None, :]
        r = np.sqrt(ox * ox + oy * oy + oz * oz)
        g0 = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
        wn = (w[nn, 0][:, :, None, None] * w[nn, 1][:, None, :, None] * w[nn, 2][:, None, None, :])
        wk = (w[kk, 0][:, :, None, None] * w[kk, 1][:, None, :, None] * w[kk, 2][:, None, None, :])
        grid_part = np.einsum("bijk,blmn,bijklmn->b", wn, wk, g0)
        vals[s:s + chunk] -= grid_part
    C = sp.coo_matrix((vals, (n, k)), shape=(Np, Np)).tocsr()
    C.sum_duplicates()
    return C
