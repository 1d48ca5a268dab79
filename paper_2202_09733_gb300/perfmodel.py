"""Algorithmic operation and byte counts of the hot-path kernels (per element).

Flops count every +, -, *, /, sqrt, |.|, max as 1 and every fma as 2, exactly as the
kernels (and the oracle) evaluate the formulas; the counts are the algorithm's, so a
division counts 1 even though the FP64 pipe executes it as a short Newton sequence.
Bytes are the compulsory traffic of a fused implementation: read the state and the
geometric factors once, write the result once (intermediate face/gradient arrays are
not counted)."""
from __future__ import annotations


def _shape(d: int, p: int):
    n = p + 1
    nv = d + 2
    np_ = n ** d
    nfp = 2 * d * n ** (d - 1)
    return n, nv, np_, nfp


def inviscid_flops(d: int) -> int:
    # 1/rho, u_j, ke (fma chain), p, per direction: d products + p on the diagonal + (E+p) u_c
    return 1 + d + 2 * d + 3 + d * (d + 1 + 2)


def viscous_flops(d: int) -> int:
    # 1/rho, E/rho, u_j, du (3 d^2), de (d (2d + 4)), div u (d), tau (2 d^2 + 2 d),
    # energy flux (d (2 d + 2))
    return 2 + d + 3 * d * d + d * (2 * d + 4) + d + 2 * d * d + 2 * d + d * (2 * d + 2)


def residual_stage_flops(d: int, p: int) -> dict:
    n, nv, np_, nfp = _shape(d, p)
    pairs = nfp / 2.0
    I, V = inviscid_flops(d), viscous_flops(d)
    rus = 2 * I + 2 * d + 1 + 2 * (5 * d + 10) + 1 + nv * (4 * d + 6)
    pair_flux = 2 * nv + 2 * d * nv + rus + V + nv * (2 * d + 1)
    return {
        "interp": 2 * nv * nfp * n,
        "pair_common": pairs * 4 * nv,
        "grad_sp": nv * np_ * (2 * d * (n + 2) + 2 * d * d),
        "grad_fp": nv * nfp * 2 * (d * n + 1 + d * d),
        "pair_flux": pairs * pair_flux,
        "vflux": np_ * (I + V + 3 * d * d * nv),
        "face_ft": 2 * nv * nfp * n,
        "div": nv * np_ * (d * (2 * n + 7) + 1),
    }


def residual_flops(d: int, p: int) -> float:
    """FP64 flops of one residual evaluation per element."""
    return float(sum(residual_stage_flops(d, p).values()))


def residual_bytes(d: int, p: int, word: int = 8) -> float:
    """compulsory bytes per element: q, S, G, invJ, Sf, Gf read; R written"""
    n, nv, np_, nfp = _shape(d, p)
    return float(word * (nv * np_ * 2 + 2 * d * d * np_ + np_ + 2 * d * d * nfp))


def block_solve_bytes(d: int, p: int, word: int = 8) -> float:
    """one element-block LU solve: the nd x nd factor, the permutation, x in and out"""
    n, nv, np_, nfp = _shape(d, p)
    nd = nv * np_
    return float(word * nd * nd + 4 * nd + 2 * word * nd)


def block_solve_flops(d: int, p: int) -> float:
    n, nv, np_, nfp = _shape(d, p)
    nd = nv * np_
    return float(2 * nd * nd)


def assembled_product_bytes(d: int, p: int, word: int = 8, neighbours: int | None = None) -> float:
    """one element's rows of the matrix-based smoother's product y = A x: its diagonal
    block and one block per face neighbour (2d on an interior element), its own x and the
    neighbours' x read, y written"""
    n, nv, np_, nfp = _shape(d, p)
    nd = nv * np_
    nb = 2 * d if neighbours is None else neighbours
    return float(word * ((nb + 1) * nd * nd + (nb + 1) * nd + nd))


def assembled_product_flops(d: int, p: int, neighbours: int | None = None) -> float:
    n, nv, np_, nfp = _shape(d, p)
    nd = nv * np_
    nb = 2 * d if neighbours is None else neighbours
    return float(2 * (nb + 1) * nd * nd)


def mbnk_solve_bytes(d: int, p: int, m: int, word: int = 8) -> float:
    """compulsory bytes per element of one matrix-based smoothing solve with m Arnoldi
    steps: per step a block solve, the assembled product and classical Gram-Schmidt twice
    over the k + 1 basis vectors (each pass reads them twice: inner products, update) plus
    the norm and scaling; then the combination of m vectors and the final block solve"""
    n, nv, np_, nfp = _shape(d, p)
    nd = nv * np_
    per_vec = word * nd
    total = per_vec * 2                                   # norm and scaling of the start vector
    for k in range(m):
        total += block_solve_bytes(d, p, word) + per_vec  # copy in, solve in place
        total += assembled_product_bytes(d, p, word)
        total += 2 * (2 * (k + 1) * per_vec + 2 * per_vec)    # two CGS passes
        total += 3 * per_vec                              # norm (read) and scaling (read, write)
    total += (m + 1) * per_vec + block_solve_bytes(d, p, word)
    return float(total)
