"""Oracle of the learned surrogate of the FFT convolution (BAIM step 2) -- test
infrastructure only (imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs).

The surrogate is a small 3D convolutional network on the AIM grid: it maps the grid
charges Q (the anterpolated charges of BAIM step 1) to the grid potential U that the FFT
convolution with the periodic Green's function would give (Sec. 3.2, Eq. 15).  The paper
has no such network; its definition here is the plain textbook one, in FP64 numpy:

  h1 = act(conv(Q / sq, W1) + b1)     1 -> C channels
  h2 = act(conv(h1, W2) + b2)         C -> C
  h3 = act(conv(h2, W3) + b3)         C -> C
  U  = su * (conv(h3, W4) + b4)       C -> 1

conv is a 3x3x3 cross-correlation, y[o](x) = sum_i sum_t W[o, i, t] x_pad[i](x + t - 1),
with circular padding along periodic axes and zero padding along the others; act is the
leaky rectifier act(z) = z (z > 0), 0.1 z (z <= 0); sq and su are fixed input/output
scales.  Training minimises the mean squared error in units of su, by backpropagation and
the Adam update (Kingma and Ba, 2015).
"""
from __future__ import annotations

import numpy as np

SLOPE = 0.1


def pad(x: np.ndarray, periodic) -> np.ndarray:
    """x [C, Z, Y, X] -> [C, Z+2, Y+2, X+2]; periodic is (px, py, pz) for the X, Y, Z axes."""
    out = x
    for axis, per in ((3, periodic[0]), (2, periodic[1]), (1, periodic[2])):
        out = np.pad(out, [(1, 1) if a == axis else (0, 0) for a in range(4)], mode="wrap" if per else "constant")
    return out


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray, periodic) -> np.ndarray:
    """3x3x3 cross-correlation: x [Ci, Z, Y, X], W [Co, Ci, 3, 3, 3], b [Co] -> [Co, Z, Y, X]."""
    Ci, Z, Y, X = x.shape
    xp = pad(x, periodic)
    y = np.empty((W.shape[0], Z, Y, X))
    for o in range(W.shape[0]):
        acc = np.full((Z, Y, X), float(b[o]))
        for i in range(Ci):
            for dz in range(3):
                for dy in range(3):
                    for dx in range(3):
                        acc += W[o, i, dz, dy, dx] * xp[i, dz:dz + Z, dy:dy + Y, dx:dx + X]
        y[o] = acc
    return y


def conv_adjoint(gy: np.ndarray, W: np.ndarray, periodic) -> np.ndarray:
    """Adjoint of conv in its input: gx[i](x) = sum_o sum_t W[o, i, t] gy[o](x - t + 1),
    accumulated by scattering each output's contribution back (no kernel flip trick)."""
    Co, Z, Y, X = gy.shape
    Ci = W.shape[1]
    gxp = np.zeros((Ci, Z + 2, Y + 2, X + 2))
    for o in range(Co):
        for i in range(Ci):
            for dz in range(3):
                for dy in range(3):
                    for dx in range(3):
                        gxp[i, dz:dz + Z, dy:dy + Y, dx:dx + X] += W[o, i, dz, dy, dx] * gy[o]
    return unpad_adjoint(gxp, periodic)


def unpad_adjoint(gxp: np.ndarray, periodic) -> np.ndarray:
    """Adjoint of pad: fold the halo back onto the interior (periodic) or drop it (zero)."""
    g = gxp
    for axis, per in ((3, periodic[0]), (2, periodic[1]), (1, periodic[2])):
        n = g.shape[axis] - 2
        core = np.take(g, range(1, n + 1), axis=axis).copy()
        if per:
            lo = np.take(g, [0], axis=axis)
            hi = np.take(g, [n + 1], axis=axis)
            idx_last = [slice(None)] * 4
            idx_last[axis] = slice(n - 1, n)
            idx_first = [slice(None)] * 4
            idx_first[axis] = slice(0, 1)
            core[tuple(idx_last)] += lo
            core[tuple(idx_first)] += hi
        g = core
    return g


def conv_weight_grad(x: np.ndarray, gy: np.ndarray, periodic) -> tuple[np.ndarray, np.ndarray]:
    """dL/dW[o, i, t] = sum_x gy[o](x) x_pad[i](x + t - 1) and dL/db[o] = sum_x gy[o](x)."""
    Ci, Z, Y, X = x.shape
    Co = gy.shape[0]
    xp = pad(x, periodic)
    gW = np.empty((Co, Ci, 3, 3, 3))
    for o in range(Co):
        for i in range(Ci):
            for dz in range(3):
                for dy in range(3):
                    for dx in range(3):
                        gW[o, i, dz, dy, dx] = np.sum(gy[o] * xp[i, dz:dz + Z, dy:dy + Y, dx:dx + X])
    return gW, gy.sum(axis=(1, 2, 3))


def act(z: np.ndarray) -> np.ndarray:
    return np.where(z > 0, z, SLOPE * z)


def act_grad(h: np.ndarray) -> np.ndarray:
    """Derivative of act, read from its output (act keeps the sign of its argument)."""
    return np.where(h > 0, 1.0, SLOPE)


def init_params(C: int = 32, seed: int = 0) -> list:
    """He-style initialisation: W ~ N(0, 2 / fan_in), b = 0 (the GPU path takes these as inputs)."""
    rng = np.random.default_rng(seed)
    shapes = [(C, 1), (C, C), (C, C), (1, C)]
    params = []
    for co, ci in shapes:
        params.append(rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), size=(co, ci, 3, 3, 3)))
        params.append(np.zeros(co))
    return params


def forward(params: list, Q: np.ndarray, sq: float, su: float, periodic) -> tuple[np.ndarray, list]:
    """Q [Z, Y, X] -> U [Z, Y, X]; also the layer inputs kept for the backward pass."""
    x = (Q / sq)[None]
    keep = []
    for k in range(4):
        keep.append(x)
        z = conv(x, params[2 * k], params[2 * k + 1], periodic)
        x = act(z) if k < 3 else z
    return su * x[0], keep


def loss_and_grad(params: list, Q: np.ndarray, U: np.ndarray, sq: float, su: float, periodic):
    """Mean squared error in units of su, and its gradient with respect to every parameter."""
    pred, keep = forward(params, Q, sq, su, periodic)
    r = (pred - U) / su
    loss = float(np.mean(r * r))
    gy = (2.0 / r.size) * r[None]           # d loss / d (last conv output)
    grads = [None] * 8
    for k in (3, 2, 1, 0):
        gW, gb = conv_weight_grad(keep[k], gy, periodic)
        grads[2 * k], grads[2 * k + 1] = gW, gb
        if k > 0:
            gx = conv_adjoint(gy, params[2 * k], periodic)
            gy = gx * act_grad(keep[k])       # keep[k] = act(z of layer k - 1)
    return loss, grads


def adam_step(params: list, grads: list, m: list, v: list, t: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update (in place); t counts from 1."""
    for k in range(len(params)):
        m[k] = beta1 * m[k] + (1.0 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * grads[k] ** 2
        mh = m[k] / (1.0 - beta1 ** t)
        vh = v[k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
