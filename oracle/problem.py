"""Oracle set-up and field evaluation for one periodic unit cell.

Test infrastructure (see ``oracle/__init__``).

H_eff = H_ex + H_ms + H_ap (Eq. 3 without anisotropy), SI units, m = unit
magnetisation, M = Ms m.  Readings of the paper's sign conventions: Eq. 13a prints
rho = div M and rho_s = -n.M, which with H = -grad u would give a field along M in a
film; the standard convention rho = -div M, sigma = +M.n is used (pinned by the
film factor N_zz = +1).  The potential is u = (1/4 pi)(sum G q + corrections) in SI.
"""
from __future__ import annotations

import math

import numpy as np

from . import operators as ops
from .direct import potential_direct
from .nearfield import near_matrix, node_moments
from .paim import AimGrid, precorrection_matrix
from .topology import boundary_faces, fold_positions, pair_nodes

GAMMA_E = 1.76085963023e11          # electron gyromagnetic ratio, rad/(s T)
GAMMA0 = ops.MU0 * GAMMA_E          # m/(A s)


class OracleProblem:
    def __init__(self, xyz, tets, periods, Ms=8e5, A=1.3e-11, alpha=0.02, H_ap=(0.0, 0.0, 0.0),
                 grid=None, p=3, near_boxes=1, near_elem_factor=0.0, eta=None, build_paim=True,
                 observers=None):
        """observers (optional): the unknowns at which the potential is needed.  The
        precorrection C and the near-element matrix E are then built for those rows only,
        and both potentials (O1 and O2) are valid at those rows only; H_ms is valid at an
        unknown whose adjacency neighbours are all observers."""
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.periods = tuple(float(L) for L in periods)
        self.Ms, self.A, self.alpha = float(Ms), float(A), float(alpha)
        self.H_ap = np.asarray(H_ap, dtype=np.float64)
        self.eta = eta
        self.lca, self.roots = pair_nodes(self.xyz, self.periods)
        self.Np = int(self.roots.size)
        self.pos = self.xyz[self.roots]
        self.pos_f, self.r0 = fold_positions(self.pos, self.periods)
        op = ops.assemble(self.xyz, self.tets, self.lca, self.Np)
        self.K, self.Wq, self.V, self.vol, self.grad = op["K"], op["Wq"], op["V"], op["vol"], op["grad"]
        self.tri, _ = boundary_faces(self.xyz, self.tets, self.lca)
        self.mean_edge = ops.mean_edge(self.xyz, self.tets)
        self.r_E = near_elem_factor * self.mean_edge
        self.E, self.near_counts = near_matrix(self.pos_f, self.xyz, self.tets, self.tri, self.lca, self.vol,
                                               self.grad, self.periods, self.Np, self.r_E,
                                               1e-6 * self.mean_edge, observers)
        self.grid = None
        if grid is not None and build_paim:
            self.grid = AimGrid(self.pos_f, self.periods, grid, p)
            self.Ktab = self.grid.kernel_table(eta)
            self.Khat = np.fft.rfftn(self.Ktab).real
            self.C = precorrection_matrix(self.grid, self.pos_f, near_boxes, observers)
            self.stencil_idx, self.stencil_w = self.grid.flat(self.pos_f)

    # ------------------------------------------------------------------ pieces
    def M(self, m):
        return self.Ms * np.asarray(m, dtype=np.float64)

    def charges(self, m):
        return ops.charges(self.Wq, self.M(m))

    def EM(self, m):
        M = self.M(m)
        return self.E[0] @ M[:, 0] + self.E[1] @ M[:, 1] + self.E[2] @ M[:, 2]

    def moments(self, m):
        return node_moments(self.M(m), self.xyz, self.tets, self.tri, self.lca, self.vol, self.grad, self.Np)

    def project(self, q):
        Q = np.zeros(int(np.prod(self.grid.dims)))
        np.add.at(Q, self.stencil_idx.ravel(), (self.stencil_w * q[:, None]).ravel())
        return Q.reshape(self.grid.dims)

    def interpolate(self, U):
        return np.einsum("nk,nk->n", U.ravel()[self.stencil_idx], self.stencil_w)

    def potential_paim(self, m):
        """4 pi u by O2."""
        q = self.charges(m)
        U = self.grid.convolve(self.project(q), self.Khat)
        return self.interpolate(U) + self.C @ q + self.EM(m)

    def potential_direct(self, m, observers=None):
        """4 pi u by O1."""
        return potential_direct(self.pos_f, self.charges(m), self.periods, self.EM(m), observers, eta=self.eta)

    def h_ms_from_potential(self, u4pi):
        return ops.gradient_field(self.Wq, self.V, u4pi / (4 * math.pi))

    def h_ms(self, m, method="paim"):
        u = self.potential_paim(m) if method == "paim" else self.potential_direct(m)
        return self.h_ms_from_potential(u)

    def h_ex(self, m):
        return ops.exchange_field(self.K, self.V, np.asarray(m, dtype=np.float64), self.A, self.Ms)

    def h_eff(self, m, method="paim", ex=True, ms=True, ap=True):
        H = np.zeros((self.Np, 3))
        if ex:
            H += self.h_ex(m)
        if ms:
            H += self.h_ms(m, method)
        if ap:
            H += self.H_ap[None, :]
        return H
