"""O1: the periodic scalar potential by direct lattice sums (Eq. 14b) plus Eq. 14c.

Test infrastructure (see ``oracle/__init__``).

    4 pi u_n = sum_{k != n} G^p(r_n - r_k) q_k + R(0) q_n + (E M)_n

with G^p from ``pgf`` (Eq. 15), folded positions r (any lattice translate gives the
same value since G^p is periodic) and E from ``nearfield``.  O(N'^2); observers may
be a subset.  This is the quantity the FFT-based method approximates.

Pinned by tests: closed-form demagnetising factors (film N_zz = 1, prism
N_xx = 1/2, filled 3D cell H = 0), the free-space exact-integral check, and the
sphere-lattice mean field.
"""
from __future__ import annotations

import numpy as np

from .pgf import pgf, pgf_reg0


def potential_direct(pos_f, q, periods, EM=None, observers=None, max_pairs=1_000_000, eta=None):
    """4 pi u at the observers (all unknowns by default).

    q may be (N,) or (N, k): k charge sets share every evaluation of G^p (EM then (N,) or
    (N, k) alike)."""
    N = pos_f.shape[0]
    obs = np.arange(N) if observers is None else np.asarray(observers)
    q = np.asarray(q, dtype=np.float64)
    u = np.zeros((obs.size,) + q.shape[1:])
    R0 = pgf_reg0(periods, eta)
    B = max(1, max_pairs // N)
    for s in range(0, obs.size, B):
        o = obs[s:s + B]
        d = pos_f[o][:, None, :] - pos_f[None, :, :]
        self_mask = o[:, None] == np.arange(N)[None, :]
        G = np.empty((o.size, N))
        G[~self_mask] = pgf(d[~self_mask], periods, eta)
        G[self_mask] = R0                      # the self term is the regular part R(0)
        u[s:s + o.size] = G @ q
    if EM is not None:
        u += EM[obs]
    return u
