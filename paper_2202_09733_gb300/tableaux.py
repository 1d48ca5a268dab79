"""Time-integration schemes in the forms the paper writes them.

The paper (Eqs. 2-3) gives the ESDIRK and Rosenbrock-Wanner forms and cites its own
second/fourth-order schemes; the two schemes used here are published members of those
families:
  ESDIRK3  - four-stage, L-stable, stiffly accurate ESDIRK of Kennedy & Carpenter (the
             implicit part of ARK3(2)4L[2]SA), coefficients as exact rationals;
  ROS34PW2 - four-stage third-order W-method of Rang & Angermann, converted from the
             standard (alpha, gamma, b) coefficients to the variables of Eq. (3):
             a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b Gamma^-1;
and the paper's own ESDIRK schemes (named in Sec. 2.1, coefficients not printed there):
  ESDIRK2  - three stages, second order, L-stable, stiffly accurate (Kennedy & Carpenter's
             review): gamma = 1 - 1/sqrt(2), c2 = 2 gamma, last row b1 = b2 = (1 - gamma)/2;
  ESDIRK4  - six stages, fourth order, L-stable, stiffly accurate, gamma = 1/4 (Bijl et
             al.; the implicit part of Kennedy & Carpenter's ARK4(3)6L[2]SA).
"""
from fractions import Fraction

import numpy as np


def esdirk3():
    """(A, b): 4x4 lower-triangular A with A[0] = 0 and b = A[3]."""
    g = Fraction(1767732205903, 4055673282236)
    rows = [[0, 0, 0, 0],
            [g, g, 0, 0],
            [Fraction(2746238789719, 10658868560708), Fraction(-640167445237, 6845629431997), g, 0],
            [Fraction(1471266399579, 7840856788654), Fraction(-4482444167858, 7529755066697),
             Fraction(11266239266428, 11593286722821), g]]
    A = np.array([[float(x) for x in r] for r in rows])
    return A, A[3].copy()


def esdirk2():
    """(A, b): 3x3, A[0] = 0, b = A[2]."""
    gam = 1.0 - 1.0 / np.sqrt(2.0)
    w = 0.5 * (1.0 - gam)
    A = np.zeros((3, 3))
    A[1, :2] = gam
    A[2] = (w, w, gam)
    return A, A[2].copy()


def esdirk4():
    """(A, b): 6x6, A[0] = 0, b = A[5], exact rationals rounded once."""
    F = Fraction
    q = F(1, 4)
    lower = {(1, 0): q,
             (2, 0): F(8611, 62500), (2, 1): F(-1743, 31250),
             (3, 0): F(5012029, 34652500), (3, 1): F(-654441, 2922500), (3, 2): F(174375, 388108),
             (4, 0): F(15267082809, 155376265600), (4, 1): F(-71443401, 120774400),
             (4, 2): F(730878875, 902184768), (4, 3): F(2285395, 8070912),
             (5, 0): F(82889, 524892), (5, 2): F(15625, 83664), (5, 3): F(69875, 102672),
             (5, 4): F(-2260, 8211)}
    A = np.zeros((6, 6))
    for (i, j), x in lower.items():
        A[i, j] = float(x)
    for i in range(1, 6):
        A[i, i] = float(q)
    return A, A[5].copy()


def ros34pw2():
    """(gamma, a, c, m) in the transformed variables of Eq. (3)."""
    gam = 0.435866521508459
    al = np.zeros((4, 4))
    al[1, 0] = 0.87173304301691801
    al[2, 0], al[2, 1] = 0.84457060015369423, -0.11299064236484185
    al[3, 2] = 1.0
    G = np.diag([gam] * 4)
    G[1, 0] = -0.87173304301691801
    G[2, 0], G[2, 1] = -0.90338057013044082, 0.054180672388095326
    G[3, 0], G[3, 1], G[3, 2] = 0.24212380706095346, -1.2232505839045147, 0.54526025533510214
    b = np.array([0.24212380706095346, -1.2232505839045147, 1.5452602553351020, 0.435866521508459])
    Gi = np.linalg.inv(G)
    return gam, np.tril(al @ Gi, -1), np.tril(np.diag(1.0 / np.diag(G)) - Gi, -1), b @ Gi
