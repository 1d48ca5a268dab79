"""Oracle of the per-element MLP initial guess (TEST INFRASTRUCTURE ONLY).

Plain numpy, FP64.  Shares no code with the CUDA path.  The network (not in the paper;
the paper's Newton guess is q^n, Sec. 4.2) maps per-element features of the last three
converged states to a correction of the quadratic-in-time extrapolation of the stage
state:

    h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3,
    loss = mean over samples and outputs of (y - t)^2.

BF16 mode emulates the GPU kernels' rounding points: x, h1, h2, the output gradients and
the weights are rounded to bfloat16 (nearest, ties to even) where they enter a matrix
product; products and sums are then exact-ish (FP64 here, FP32 on the GPU).
"""
from __future__ import annotations

import numpy as np


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def forward(params: dict, X: np.ndarray, mode: str = "fp64"):
    """X: [B, K0].  Returns y and the activations needed by backward."""
    r = bf16 if mode == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    x = r(X)
    a1 = x @ r(W1).T + b1
    h1 = np.tanh(a1)
    a2 = r(h1) @ r(W2).T + b2
    h2 = np.tanh(a2)
    y = r(h2) @ r(W3).T + b3
    return y, dict(x=x, h1=h1, h2=h2)


def loss(y, T):
    return float(np.mean((y - T) ** 2))


def backward(params: dict, cache: dict, y: np.ndarray, T: np.ndarray, mode: str = "fp64"):
    """Gradients of the mean-squared loss with respect to every parameter."""
    r = bf16 if mode == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    B, O = y.shape
    g3 = 2.0 * (y - T) / (B * O)
    dW3 = r(g3).T @ r(cache["h2"])
    db3 = g3.sum(axis=0)
    gh2 = r(g3) @ r(params["W3"])
    g2 = gh2 * (1.0 - cache["h2"] ** 2)
    dW2 = r(g2).T @ r(cache["h1"])
    db2 = g2.sum(axis=0)
    gh1 = r(g2) @ r(params["W2"])
    g1 = gh1 * (1.0 - cache["h1"] ** 2)
    dW1 = r(g1).T @ cache["x"]
    db1 = g1.sum(axis=0)
    return dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3)


def adam(params: dict, grads: dict, state: dict, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on the FP64 parameters (bias-corrected moments)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def extrapolation_weights(c: float):
    """Quadratic Lagrange extrapolation in time through q^{n-2}, q^{n-1}, q^n (nodes 0, 1,
    2 in units of dt) to t_n + c dt: weights for (q^{n-2}, q^{n-1}, q^n)."""
    tau = 2.0 + c
    return ((tau - 1.0) * (tau - 2.0) / 2.0, -tau * (tau - 2.0), tau * (tau - 1.0) / 2.0)


def features(qn, qn1, qn2, Rn, dt, logJ, c, s, sig, qinf, K0):
    """Per-element features [E, K0] from states [nv, Np, E] (FP64):
    [(q^n - q^{n-1})/s_v, (q^{n-1} - q^{n-2})/s_v, (q^n - qinf_v)/sig_v, dt R(q^n)/s_v,
     log J / 10, c, 0...]."""
    nv, Np, E = qn.shape
    nd = nv * Np
    X = np.zeros((E, K0))
    sv = np.asarray(s)[:, None, None]
    X[:, 0:nd] = ((qn - qn1) / sv).reshape(nd, E).T
    X[:, nd:2 * nd] = ((qn1 - qn2) / sv).reshape(nd, E).T
    X[:, 2 * nd:3 * nd] = ((qn - np.asarray(qinf)[:, None, None]) / np.asarray(sig)[:, None, None]).reshape(nd, E).T
    X[:, 3 * nd:4 * nd] = (dt * Rn / sv).reshape(nd, E).T
    X[:, 4 * nd:4 * nd + Np] = (logJ / 10.0).T
    X[:, 4 * nd + Np] = c
    return X


def scales(qn, qn1, qinf):
    """Per-variable scales: s_v = RMS(q^n - q^{n-1}), sig_v = RMS(q^n - qinf_v), both at
    least 1e-8 max_v |qinf_v| (a state at rest)."""
    fl = max(1e-8 * float(np.max(np.abs(qinf))), 1e-300)
    s = np.sqrt(np.mean((qn - qn1) ** 2, axis=(1, 2)))
    sig = np.sqrt(np.mean((qn - np.asarray(qinf)[:, None, None]) ** 2, axis=(1, 2)))
    return np.maximum(s, fl), np.maximum(sig, fl)
