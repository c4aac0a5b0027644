"""Implicit midpoint time stepping of the LLG equation with Newton-Krylov (Sec. 2.2 and Sec. 4).

Test infrastructure (see ``oracle/__init__``).

The paper integrates the discrete LLG system (Eq. 6) with implicit schemes, solving each
step by Newton iterations whose linear systems go to a preconditioned Krylov solver; the
only field operation this needs is the product of the field's linear part with a vector.
This module states one such scheme plainly, in FP64:

  dm/dt = f(m) = -g [ m x H(m) + alpha m x (m x H(m)) ],   g = gamma0 / (1 + alpha^2),
  H(m)  = A m + H_ap  (A: exchange + magnetostatic, linear; H_ap uniform).

Implicit midpoint rule, y = m_{n+1}, mb = (m_n + y) / 2:
  R(y) = y - m_n - dt f(mb) = 0.
Its Jacobian acts on v as
  J v = v - (dt/2) Df(mb) v,
  Df(m) v = -g [ v x H + m x (A v) + alpha ( v x (m x H) + m x (v x H) + m x (m x (A v)) ) ],
with H = H(mb).  The rule keeps |m| of every node exactly (m . f(m) = 0, and mb . (y - m_n)
= (|y|^2 - |m_n|^2) / 2), so no renormalisation is applied.

Newton: y_0 = m_n; then J(y_k) d = -R(y_k), solved by
GMRES to a relative residual gmres_tol, y_{k+1} = y_k + d, until |d| <= newton_tol |y|.
Preconditioner (right): block-Jacobi, one 3x3 block per node, J with A replaced by its
diagonal c_n (the exchange operator's own coefficient, -(2A/(mu0 Ms)) K_nn / V_n):
  P_n v = v - (dt/2) ( -g [ v x H_n + c_n m_n x v + alpha ( v x (m_n x H_n) + m_n x (v x H_n)
                                                           + c_n m_n x (m_n x v) ) ] ).
The Krylov solver is scipy's GMRES (a library step) on the preconditioned operator.

Pinned by tests: a single spin in a uniform field (alpha = 0) turns by exactly
2 atan(gamma0 H dt / 2) per step (the midpoint rule is the Cayley transform of the rotation);
|m| is kept to the Newton tolerance; the damped single spin converges to its closed form at
second order; small steps agree with RK4.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, gmres

from .llg import llg_rhs
from .problem import GAMMA0


def llg_jvp(m, H, Av, v, alpha, gamma0=GAMMA0):
    """Df(m) v for f(m) = llg_rhs(m, H(m)) with H(m + eps v) = H + eps A v."""
    g = gamma0 / (1.0 + alpha * alpha)
    mxH = np.cross(m, H)
    t = np.cross(v, H) + np.cross(m, Av)
    t = t + alpha * (np.cross(v, mxH) + np.cross(m, np.cross(v, H)) + np.cross(m, np.cross(m, Av)))
    return -g * t


def _cross_matrix(a):
    """[a]_x with [a]_x v = a x v, shape (..., 3, 3)."""
    z = np.zeros(a.shape[:-1])
    return np.stack([np.stack([z, -a[..., 2], a[..., 1]], -1),
                     np.stack([a[..., 2], z, -a[..., 0]], -1),
                     np.stack([-a[..., 1], a[..., 0], z], -1)], -2)


def block_preconditioner(m, H, c, dt, alpha, gamma0=GAMMA0):
    """3x3 blocks P_n of the block-Jacobi preconditioner (A replaced by diag(c))."""
    g = gamma0 / (1.0 + alpha * alpha)
    I = np.eye(3)[None]
    Hx = _cross_matrix(H)                      # v -> H x v
    mx = _cross_matrix(m)                      # v -> m x v
    mxHx = _cross_matrix(np.cross(m, H))       # v -> (m x H) x v
    # v x H = -[H]_x v;  v x (m x H) = -[m x H]_x v;  m x (v x H) = -[m]_x [H]_x v
    D = -Hx + c[:, None, None] * mx + alpha * (-mxHx - mx @ Hx + c[:, None, None] * (mx @ mx))
    return I - 0.5 * dt * (-g) * D


class MidpointStepper:
    """Implicit midpoint steps for an OracleProblem-like field: field(m) = A m + H_ap and
    lin(v) = A v (the problem's h_eff without / with the applied field)."""

    def __init__(self, field, lin, diag, alpha, newton_tol=1e-12, gmres_tol=1e-10, restart=30, max_newton=20,
                 gamma0=GAMMA0):
        self.field, self.lin, self.diag = field, lin, np.asarray(diag, dtype=np.float64)
        self.alpha, self.gamma0 = float(alpha), float(gamma0)
        self.newton_tol, self.gmres_tol, self.restart, self.max_newton = newton_tol, gmres_tol, restart, max_newton
        self.newton_its = 0
        self.krylov_its = 0

    def step(self, m, dt):
        a, g0 = self.alpha, self.gamma0
        n = m.shape[0]
        y = m.copy()
        for _ in range(self.max_newton):
            mb = 0.5 * (m + y)
            H = self.field(mb)
            R = y - m - dt * llg_rhs(mb, H, a, g0)
            P = block_preconditioner(mb, H, self.diag, dt, a, g0)
            Pinv = np.linalg.inv(P)

            def J(v):
                v = v.reshape(n, 3)
                return (v - 0.5 * dt * llg_jvp(mb, H, self.lin(v), v, a, g0)).ravel()

            def Minv(v):
                return np.einsum("nij,nj->ni", Pinv, v.reshape(n, 3)).ravel()

            its = [0]

            def count(_):
                its[0] += 1

            d, info = gmres(LinearOperator((3 * n, 3 * n), matvec=J), -R.ravel(),
                            M=LinearOperator((3 * n, 3 * n), matvec=Minv), rtol=self.gmres_tol, atol=0.0,
                            restart=self.restart, maxiter=50, callback=count, callback_type="pr_norm")
            self.krylov_its += its[0]
            self.newton_its += 1
            d = d.reshape(n, 3)
            y = y + d
            if np.linalg.norm(d) <= self.newton_tol * np.linalg.norm(y):
                break
        return y
