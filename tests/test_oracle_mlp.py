"""Pins of the MLP oracle (the learned Newton initial guess; not in the paper).

  - FP64 backward pass = central-difference gradient of the loss (relative 1e-7);
  - BF16 rounding = the bfloat16 values of a reference bit pattern table, ties to even;
  - extrapolation weights reproduce quadratics in time exactly;
  - Adam's first step moves every parameter by lr against the gradient sign."""
import numpy as np
import pytest

from oracle import mlp


def _params(rng, K0=32, H=16, O=8, scale=0.3):
    return dict(W1=rng.standard_normal((H, K0)) * scale, b1=rng.standard_normal(H) * 0.1,
                W2=rng.standard_normal((H, H)) * scale, b2=rng.standard_normal(H) * 0.1,
                W3=rng.standard_normal((O, H)) * scale, b3=rng.standard_normal(O) * 0.1)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    P = _params(rng)
    X = rng.standard_normal((24, 32))
    T = rng.standard_normal((24, 8))
    y, cache = mlp.forward(P, X)
    G = mlp.backward(P, cache, y, T)
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(P, X)[0], T)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(P, X)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)) + 1e-10, (k, idx, fd, an)


def test_bf16_rounding_nearest_even():
    # 1 + 2^-8 is exactly between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3 * 2^-8 is between 1 + 2^-7 and 1 + 2^-6 (tie): even mantissa is 1 + 2^-6
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(1).standard_normal(1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))   # half an ulp, 7 stored bits
    assert np.array_equal(mlp.bf16(r), r)


@pytest.mark.parametrize("c", [0.3, 0.6, 1.0])
def test_extrapolation_exact_on_quadratics(c):
    w = mlp.extrapolation_weights(c)
    for f in (lambda t: 1.0, lambda t: t, lambda t: 3 * t * t - t + 2):
        assert abs(w[0] * f(0) + w[1] * f(1) + w[2] * f(2) - f(2 + c)) < 1e-13


def test_adam_first_step():
    rng = np.random.default_rng(2)
    P = _params(rng)
    G = {k: rng.standard_normal(v.shape) for k, v in P.items()}
    P0 = {k: v.copy() for k, v in P.items()}
    mlp.adam(P, G, {}, lr=1e-3)
    for k in P:
        # first bias-corrected step: -lr g / (|g| + eps), i.e. lr against the sign up to lr eps / |g|
        dev = np.abs((P[k] - P0[k]) + 1e-3 * np.sign(G[k]))
        assert np.all(dev <= 1e-3 * 1e-8 / np.abs(G[k]) + 1e-15)


def test_features_and_scales_on_closed_forms():
    """q^n = q^{n-1} + a_v (a constant shift per variable), q^{n-2} = q^{n-1}: the scales are
    |a_v|, the first block is sign(a_v), the second zero; R = 1 gives dt / |a_v|."""
    rng = np.random.default_rng(4)
    nv, Np, E = 4, 9, 5
    q1 = 1.0 + rng.random((nv, Np, E))
    a = np.array([0.5, -0.25, 2.0, 1e-3])
    qn = q1 + a[:, None, None]
    qinf = np.array([1.0, 0.5, 0.0, 2.5])
    s, sig = mlp.scales(qn, q1, qinf)
    assert np.allclose(s, np.abs(a), rtol=1e-14)
    assert np.allclose(sig, np.sqrt(np.mean((qn - qinf[:, None, None]) ** 2, axis=(1, 2))), rtol=1e-14)
    logJ = np.log(1.0 + rng.random((Np, E)))
    X = mlp.features(qn, q1, q1, np.ones_like(qn), 0.1, logJ, 0.7, s, sig, qinf, 4 * nv * Np + Np + 3)
    nd = nv * Np
    assert np.allclose(X[:, :nd], np.repeat(np.sign(a), Np)[None, :], rtol=1e-14)
    assert np.all(X[:, nd:2 * nd] == 0)
    assert np.allclose(X[:, 3 * nd:4 * nd], np.repeat(0.1 / np.abs(a), Np)[None, :], rtol=1e-14)
    assert np.allclose(X[:, 4 * nd:4 * nd + Np], logJ.T / 10, rtol=1e-14)
    assert np.all(X[:, 4 * nd + Np] == 0.7) and np.all(X[:, 4 * nd + Np + 1:] == 0)
    # a state at rest: the floor keeps the scales positive
    s0, _ = mlp.scales(q1, q1, qinf)
    assert np.all(s0 == 1e-8 * 2.5)
