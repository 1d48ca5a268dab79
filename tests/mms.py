"""Manufactured solutions for the compressible Navier-Stokes residual (test helper).

The exact semi-discrete target is dq/dt = -div(f_inv(q) - f_visc(q, grad q)) (Eq. 1) for a
smooth periodic field; sympy differentiates the fluxes symbolically, independently of any
discretisation.  Used to pin the oracle's R by its order of accuracy."""
import functools

import numpy as np

GAMMA, PR = 1.4, 0.72


@functools.lru_cache(maxsize=None)
def exact_rhs(d: int, mu: float):
    sp = __import__("sympy")
    X = sp.symbols("x y z")[:d]
    x, y = X[0], X[1]
    z = X[2] if d == 3 else 0
    rho = 1 + sp.Rational(1, 5) * sp.sin(x) * sp.cos(y) + (sp.Rational(1, 10) * sp.cos(z) if d == 3 else 0)
    vel = [sp.Rational(1, 2) + sp.Rational(1, 10) * sp.sin(x) * sp.sin(y),
           sp.Rational(1, 5) * sp.cos(x) - sp.Rational(1, 10) * sp.sin(y)]
    if d == 3:
        vel[0] += sp.Rational(1, 20) * sp.sin(z)
        vel.append(sp.Rational(1, 10) * sp.cos(x + z) + sp.Rational(1, 20) * sp.sin(y))
    p = 5 + sp.Rational(3, 10) * sp.cos(x - y) + (sp.Rational(1, 10) * sp.sin(z) if d == 3 else 0)
    g = sp.Float(GAMMA)
    E = p / (g - 1) + rho * sum(u * u for u in vel) / 2
    q = [rho] + [rho * u for u in vel] + [E]
    kappa = g * sp.Float(mu) / sp.Float(PR)
    e = p / ((g - 1) * rho)
    grad = [[sp.diff(u, X[c]) for c in range(d)] for u in vel]
    div = sum(grad[j][j] for j in range(d))
    tau = [[sp.Float(mu) * (grad[i][j] + grad[j][i] - (sp.Rational(2, 3) * div if i == j else 0))
            for j in range(d)] for i in range(d)]
    rhs = [0] * (d + 2)
    for c in range(d):
        finv = [rho * vel[c]] + [rho * vel[c] * vel[j] + (p if j == c else 0) for j in range(d)] + \
               [(E + p) * vel[c]]
        fvis = [0] + [tau[j][c] for j in range(d)] + \
               [sum(vel[j] * tau[j][c] for j in range(d)) + kappa * sp.diff(e, X[c])]
        for v in range(d + 2):
            rhs[v] = rhs[v] - sp.diff(finv[v] - fvis[v], X[c])
    fq = sp.lambdify(X, q, "numpy")
    fr = sp.lambdify(X, rhs, "numpy")

    def state(P):
        vals = fq(*P)
        return np.stack([np.broadcast_to(np.asarray(v, dtype=float), P[0].shape) for v in vals])

    def target(P):
        vals = fr(*P)
        return np.stack([np.broadcast_to(np.asarray(v, dtype=float), P[0].shape) for v in vals])
    return state, target
