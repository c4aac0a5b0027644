"""Landau-Lifshitz-Gilbert right-hand side (Eq. 2 / Eq. 6) and classical RK4.

Test infrastructure (see ``oracle/__init__``).

For unit m:  dm/dt = -gamma0/(1+alpha^2) [ m x H + alpha m x (m x H) ].
Reading of Eq. 6, which prints M x M_n x H: the double product is M_n x (M_n x H).
gamma0 = mu0 * 1.76085963023e11 m/(A s) (the paper gives no value).
Time stepping: classical 4-stage Runge-Kutta with the field re-evaluated at every
stage, then m <- m / |m| (the paper uses implicit schemes; this integrator is the
one the GPU path implements).

Pinned by tests: |m| is conserved by the continuous flow (the RHS is orthogonal to
m), energy decreases for alpha > 0 on the exchange-only problem, and a single spin
in a constant field precesses at gamma0 H / (1 + alpha^2) with the closed-form
damped angle.
"""
from __future__ import annotations

import numpy as np

from .problem import GAMMA0


def llg_rhs(m, H, alpha, gamma0=GAMMA0):
    mxH = np.cross(m, H)
    return -gamma0 / (1.0 + alpha * alpha) * (mxH + alpha * np.cross(m, mxH))


def rk4_step(m, dt, field, alpha, gamma0=GAMMA0):
    k1 = llg_rhs(m, field(m), alpha, gamma0)
    k2 = llg_rhs(m + 0.5 * dt * k1, field(m + 0.5 * dt * k1), alpha, gamma0)
    k3 = llg_rhs(m + 0.5 * dt * k2, field(m + 0.5 * dt * k2), alpha, gamma0)
    k4 = llg_rhs(m + dt * k3, field(m + dt * k3), alpha, gamma0)
    out = m + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return out / np.linalg.norm(out, axis=1, keepdims=True)
