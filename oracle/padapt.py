"""Oracle of the p-adaptation indicator and marking (Sec. 3.3), plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the product package never imports it.

Sec. 3.3 adapts each element's degree with the spectral-decay smoothness indicator
    eta_k = ||s_p - s_{p-1}||_L2 / ||s_p||_L2
of a scalar s (the x-momentum rho u unless stated), where s_{p-1} is s_p with its
highest-degree content removed, and the marking rule: raise the degree by one where
eta_k > nu_max eta_max, lower it by one where eta_k < nu_min eta_max (nu_max = 0.2,
nu_min = 1e-3, eta_max the largest indicator of the field), within [p_min, p_max].

Readings (the paper defines the indicator in words and one formula):
  - s_p is the element's nodal values on the tensor-product Gauss-Legendre points; its
    expansion in tensor products of orthonormal Legendre polynomials phi_a(xi) phi_b(eta)
    [phi_c(zeta)] follows from the Gauss-Legendre quadrature with p + 1 points per
    direction, exact for products of two degree-p polynomials; s_{p-1} keeps the modes
    whose largest index is at most p - 1 (the tensor space Q^{p-1}, the p-levels' space);
  - the L2 norms are those of the reference element (no Jacobian weighting, as the
    p-transfers of Eqs. 17-18), so by Parseval eta_k^2 is the energy of the removed modes
    over the energy of all modes; an element with s = 0 has eta = 0;
  - the nested hierarchy (the paper gives examples only, for p_max = 4 and three levels:
    gap 1 -> {4-3-2}, {3-2-1}, {2-1-0}, {1-0-0}; gap 2 -> {4-2-0}, {3-1-0}, {2-1-0},
    {1-0-0}): level l has degree min(max(p_e - gap l, L - 1 - l), max(p_{l-1} - 1, 0)),
    which reproduces all eight.
"""
from __future__ import annotations

import numpy as np


def legendre_modes(p: int):
    """(xi, w, Phi) with Phi[a, i] = phi_a(xi_i), phi_a = sqrt((2a + 1)/2) P_a: the
    orthonormal Legendre polynomials at the p + 1 Gauss-Legendre points."""
    xi, w = np.polynomial.legendre.leggauss(p + 1)
    Phi = np.empty((p + 1, p + 1))
    for a in range(p + 1):
        c = np.zeros(a + 1)
        c[a] = 1.0
        Phi[a] = np.sqrt((2 * a + 1) / 2.0) * np.polynomial.legendre.legval(xi, c)
    return xi, w, Phi


def modal_coefficients(s_nodal: np.ndarray, d: int, p: int) -> np.ndarray:
    """Coefficients c[a, b(, c)] of the nodal values s_nodal [Np] in the tensor Legendre
    basis: c_a = sum_i w_i phi_a(xi_i) s_i along every direction."""
    _, w, Phi = legendre_modes(p)
    T = Phi * w[None, :]                      # T[a, i] = w_i phi_a(xi_i)
    s = np.asarray(s_nodal, dtype=np.float64).reshape((p + 1,) * d)
    for ax in range(d):
        s = np.moveaxis(np.tensordot(T, s, axes=([1], [ax])), 0, ax)
    return s


def spectral_decay(q: np.ndarray, d: int, p: int, var: int = 1) -> np.ndarray:
    """eta_k of variable var of a state q [nv][Np][E] for every element k."""
    E = q.shape[2]
    eta = np.zeros(E)
    for e in range(E):
        c = modal_coefficients(q[var, :, e], d, p)
        top = np.zeros(c.shape, dtype=bool)
        for ax in range(d):
            idx = [slice(None)] * d
            idx[ax] = p
            top[tuple(idx)] = True               # modes whose largest index is p
        total = float(np.sum(c * c))
        eta[e] = np.sqrt(float(np.sum(c[top] ** 2)) / total) if total > 0.0 else 0.0
    return eta


def mark(eta: np.ndarray, p_elem: np.ndarray, p_min: int, p_max: int, nu_min: float = 1e-3,
         nu_max: float = 0.2) -> np.ndarray:
    """New element degrees after one adaptation of the marking rule."""
    eta = np.asarray(eta, dtype=np.float64)
    p_elem = np.asarray(p_elem, dtype=np.int64)
    emax = float(eta.max()) if eta.size else 0.0
    out = p_elem.copy()
    up = (eta > nu_max * emax) & (p_elem < p_max)
    down = (eta < nu_min * emax) & (p_elem > p_min)
    out[up] += 1
    out[down] -= 1
    return out


def nested_hierarchy(p_elem: int, gap: int, nlevels: int) -> list:
    """The element's degrees on the nlevels p-sublevels (finest first)."""
    lv = [int(p_elem)]
    for l in range(1, nlevels):
        lv.append(min(max(p_elem - gap * l, nlevels - 1 - l), max(lv[-1] - 1, 0)))
    return lv
