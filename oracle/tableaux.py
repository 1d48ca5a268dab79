"""Time-integration tableaux for the oracle (TEST INFRASTRUCTURE ONLY).

The paper states the ESDIRK (Eq. 2) and Rosenbrock-Wanner (Eq. 3) forms and cites its
own second/fourth-order schemes without printing them.  The schemes here are two
published third-order members of those families:
  ESDIRK3  - Kennedy & Carpenter's four-stage, L-stable, stiffly accurate ESDIRK
             (the implicit part of ARK3(2)4L[2]SA), given as exact rationals;
  ROS34PW2 - Rang & Angermann's four-stage third-order W-method, standard
             (alpha, gamma, b) form, converted here to the transformed variables of
             Eq. (3): a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b Gamma^-1.
and the paper's own ESDIRK schemes (Sec. 2.1 names them; their coefficients are not
printed there):
  ESDIRK2  - the three-stage, L-stable, stiffly accurate second-order ESDIRK of Kennedy &
             Carpenter's review, gamma = 1 - 1/sqrt(2), c2 = 2 gamma; with an explicit first
             stage, stiff accuracy and c2 = 2 gamma the order conditions fix the last row
             to b1 = b2 = (1 - gamma) / 2;
  ESDIRK4  - the six-stage, L-stable, stiffly accurate fourth-order ESDIRK of Bijl et al.
             (the implicit part of Kennedy & Carpenter's ARK4(3)6L[2]SA, gamma = 1/4),
             given as exact rationals.
All are pinned by their order conditions in the tests.
"""
from fractions import Fraction as Fr
import numpy as np


def esdirk3():
    g = Fr(1767732205903, 4055673282236)
    A = [[Fr(0), Fr(0), Fr(0), Fr(0)],
         [g, g, Fr(0), Fr(0)],
         [Fr(2746238789719, 10658868560708), Fr(-640167445237, 6845629431997), g, Fr(0)],
         [Fr(1471266399579, 7840856788654), Fr(-4482444167858, 7529755066697),
          Fr(11266239266428, 11593286722821), g]]
    A = np.array([[float(x) for x in row] for row in A])
    b = A[3].copy()
    c = A.sum(axis=1)
    return A, b, c


def esdirk2():
    g = 1.0 - 1.0 / np.sqrt(2.0)
    bb = 0.5 * (1.0 - g)
    A = np.array([[0.0, 0.0, 0.0],
                  [g, g, 0.0],
                  [bb, bb, g]])
    return A, A[2].copy(), A.sum(axis=1)


def esdirk4():
    g = Fr(1, 4)
    z = Fr(0)
    A = [[z, z, z, z, z, z],
         [g, g, z, z, z, z],
         [Fr(8611, 62500), Fr(-1743, 31250), g, z, z, z],
         [Fr(5012029, 34652500), Fr(-654441, 2922500), Fr(174375, 388108), g, z, z],
         [Fr(15267082809, 155376265600), Fr(-71443401, 120774400), Fr(730878875, 902184768),
          Fr(2285395, 8070912), g, z],
         [Fr(82889, 524892), z, Fr(15625, 83664), Fr(69875, 102672), Fr(-2260, 8211), g]]
    c = np.array([float(sum(row)) for row in A])
    A = np.array([[float(x) for x in row] for row in A])
    return A, A[5].copy(), c


def ros34pw2_standard():
    gam = 4.3586652150845900e-01
    alpha = np.zeros((4, 4))
    alpha[1, 0] = 8.7173304301691801e-01
    alpha[2, 0] = 8.4457060015369423e-01
    alpha[2, 1] = -1.1299064236484185e-01
    alpha[3, 2] = 1.0
    G = np.zeros((4, 4))
    np.fill_diagonal(G, gam)
    G[1, 0] = -8.7173304301691801e-01
    G[2, 0] = -9.0338057013044082e-01
    G[2, 1] = 5.4180672388095326e-02
    G[3, 0] = 2.4212380706095346e-01
    G[3, 1] = -1.2232505839045147e+00
    G[3, 2] = 5.4526025533510214e-01
    b = np.array([2.4212380706095346e-01, -1.2232505839045147e+00, 1.5452602553351020e+00,
                  4.3586652150845900e-01])
    return gam, alpha, G, b


def ros34pw2():
    """(gamma, a, c, m) in the variables of Eq. (3)."""
    gam, alpha, G, b = ros34pw2_standard()
    Gi = np.linalg.inv(G)
    a = alpha @ Gi
    c = np.diag(1.0 / np.diag(G)) - Gi
    m = b @ Gi
    a = np.tril(a, -1)
    c = np.tril(c, -1)
    return gam, a, c, m
