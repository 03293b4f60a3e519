"""FP64 CPU reference of the learned p2r path-length seed.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py use this module.  It shares no code with the GPU library
(paper_2409_09228_gb300/csrc/mlp.cu, mlp.cuh), which it checks.

The paper's p2r (Sec. 3.2, "propagation to r") finds the path length to the
cylinder iteratively; the GPU library adds a small network that predicts
where that iteration should start.  This module writes out what that network
computes, plainly and in float64, so that its kernels can be compared with it:

  inputs   (features)  eight numbers per sample, in the frame whose x axis
           points along the track's transverse position (definitions below);
  target   g = (h - h_line) / (kappa h_line^2 / 2), h the exact transverse path
           length, h_line the straight-line distance along the momentum;
  network  8 -> 64 -> 64 -> 1, ReLU, y = W3 relu(W2 relu(W1 x + b1) + b2) + b3;
  loss     L = (1/n) sum over samples with a finite target of (y - g)^2, and its
           gradient by the chain rule (backpropagation) written out per layer;
  Adam     Kingma and Ba (2015), Algorithm 1.

With emulate=True every number the GPU rounds to BF16 is rounded here too, at
the same place: the weights, each input split into hi = bf16(x) and
lo = bf16(x - hi), the hidden activations, and (backward) the two hidden
layers' error signals before they enter a matrix product.  Rounding passes
gradients through unchanged (the gradient of the rounded value is used for
the unrounded one).  With emulate=False nothing is rounded: the exact FP64
network and its exact gradient.

Parameter vector (4801): W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
from __future__ import annotations

import numpy as np

KA = 0.00299792458  # GeV / (T cm)
N_IN, N_HID = 8, 64
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 512, 576, 4672, 4736, 4800
N_PARAMS = 4801


def unpack(params):
    """(W1, b1, W2, b2, W3, b3) views of the parameter vector."""
    p = np.asarray(params)
    return (p[OFF_W1:OFF_B1].reshape(N_HID, N_IN), p[OFF_B1:OFF_W2],
            p[OFF_W2:OFF_B2].reshape(N_HID, N_HID), p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3],
            p[OFF_B3])


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2),
                           np.ravel(W3), np.atleast_1d(b3)])


def bf16(x):
    """x rounded to the nearest bfloat16 (1 sign, 8 exponent, 7 fraction bits),
    ties to even, returned as float64.  x is first rounded to float32 (the GPU
    holds every such value in float32 before it rounds it to BF16).  Finite
    inputs only."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


# ---- inputs and target -----------------------------------------------------------


def features(B, par, q, R):
    """The eight inputs (n, 8) of states par (6, n) with charges q (n,) towards
    radii R (n,), field B [T]:
      x0 = r0 / R, x1 = z / R, x2 = kA B w R / 2, x3 = cos psi, x4 = sin psi,
      x5 = cos theta, x6 = q, x7 = R / 100 cm,
    r0 = sqrt(x^2 + y^2), psi = phi - atan2(y, x) (0 when r0 = 0)."""
    p = np.asarray(par, np.float64)
    R = np.asarray(R, np.float64)
    x, y, z, w, phi, th = p
    r0 = np.hypot(x, y)
    psi = np.where(r0 > 0, phi - np.arctan2(y, x), 0.0)
    return np.stack([r0 / R, z / R, 0.5 * KA * B * w * R, np.cos(psi), np.sin(psi), np.cos(th),
                     np.asarray(q, np.float64), R / 100.0], axis=1)


def line_distance(par, R):
    """Distance along the momentum direction from (x, y), inside the circle of
    radius R, to the circle: the positive root of |P + h u|^2 = R^2; NaN from
    outside."""
    p = np.asarray(par, np.float64)
    R = np.asarray(R, np.float64)
    x, y, phi = p[0], p[1], p[4]
    b = x * np.cos(phi) + y * np.sin(phi)
    c = x * x + y * y - R * R
    with np.errstate(invalid="ignore"):
        return np.where(c <= 0, -b + np.sqrt(b * b - c), np.nan)


def curvature(B, par, q):
    return -np.asarray(q, np.float64) * KA * B * np.asarray(par, np.float64)[3]


def target(B, par, q, R, h):
    """g = (h - h_line) / (kappa h_line^2 / 2); NaN where h_line is undefined or
    kappa = 0."""
    hl = line_distance(par, R)
    k = curvature(B, par, q)
    with np.errstate(invalid="ignore", divide="ignore"):
        g = (np.asarray(h, np.float64) - hl) / (0.5 * k * hl * hl)
    return np.where(np.isfinite(g) & (k != 0), g, np.nan)


def seed(B, par, q, R, g):
    """The path length the network's output g stands for."""
    hl = line_distance(par, R)
    return hl + np.asarray(g, np.float64) * 0.5 * curvature(B, par, q) * hl * hl


# ---- network -----------------------------------------------------------------------


def _split(X, emulate):
    X = np.asarray(X)
    if not emulate:
        return np.asarray(X, np.float64)
    hi = bf16(X)
    lo = bf16(np.asarray(X, np.float32) - hi.astype(np.float32))
    return hi + lo


def forward(params, X, emulate=True):
    """y (n,) for inputs X (n, 8); also the intermediates for backward."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(params, np.float64))
    rw = bf16 if emulate else (lambda v: np.asarray(v, np.float64))
    W1r, W2r, W3r = rw(W1), rw(W2), rw(W3)
    xin = _split(X, emulate)
    z1 = xin @ W1r.T + b1
    a1 = rw(np.maximum(z1, 0.0))
    z2 = a1 @ W2r.T + b2
    a2 = rw(np.maximum(z2, 0.0))
    y = a2 @ W3r + b3
    cache = dict(xin=xin, z1=z1, a1=a1, z2=z2, a2=a2, W2r=W2r, W3r=W3r)
    return y, cache


def loss_grad(params, X, t, emulate=True):
    """(L, dL/dparams) for L = (1/n) sum_{i: t_i finite} (y_i - t_i)^2."""
    n = len(t)
    y, c = forward(params, X, emulate)
    t = np.asarray(t, np.float64)
    ok = np.isfinite(t)
    e = np.where(ok, y - np.where(ok, t, 0.0), 0.0)
    L = float(np.sum(e * e) / n)
    rw = bf16 if emulate else (lambda v: np.asarray(v, np.float64))
    dy = 2.0 * e / n
    dW3 = c["a2"].T @ dy
    db3 = np.sum(dy)
    dz2 = np.outer(dy, c["W3r"]) * (c["z2"] > 0)
    db2 = dz2.sum(axis=0)
    dz2r = rw(dz2)
    dW2 = dz2r.T @ c["a1"]
    da1 = dz2r @ c["W2r"]
    dz1 = da1 * (c["z1"] > 0)
    db1 = dz1.sum(axis=0)
    dW1 = rw(dz1).T @ c["xin"]
    return L, pack(dW1, db1, dW2, db2, dW3, db3)


def adam(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015, Algorithm 1), step number t >= 1:
    returns the new (params, m, v)."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(params, np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v
