"""A smooth test state on which R is differentiable (test helper).

The Rusanov flux contains |v.n| and max(lambda_L, lambda_R); both are kinks of R.  A free
stream at an angle (|v.n| bounded away from 0 on every face family) with a small smooth
perturbation keeps every evaluation away from the kinks, so finite differences of R
converge to the Jacobian."""
import math

import numpy as np

from paper_2202_09733_gb300 import workloads as w


def angled_flow(mesh, p, mach=0.3, amp=0.02, seed=0):
    X = w.solution_point_coords(mesh, p)
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 1.5, size=4)
    ph = rng.uniform(0, 2 * math.pi, size=4)
    L = mesh.get("L", (10.0, 10.0))
    s = lambda i, a, b: np.sin(2 * math.pi * (a * X[0] / L[0] + b * X[1] / L[1]) + ph[i])
    rho = 1.0 + amp * s(0, 1, 0)
    u = math.cos(0.5) + amp * s(1, 0, 1)
    v = math.sin(0.5) + amp * s(2, 1, 1)
    p_ = 1.0 / (w.GAMMA * mach * mach) * (1.0 + amp * s(3, 1, -1))
    return np.ascontiguousarray(w.prim_to_cons(rho, [u, v], p_))
