"""FP64 CPU oracle for the JFNK-pMG hot path.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference leg are the only callers.  The product package never imports this module, and
this module never imports the product package's CUDA binding; the two share only the
seeded input generators (paper_2202_09733_gb300.workloads), which hold none of the
method's arithmetic.

The C sources (plain C11, FP64, -ffp-contract=off) implement, step by step:
  tables.c    Gauss-Legendre FR tables, DG correction functions, Eqs. (17)-(18)
  level.c     curved-element geometric factors, face-point connectivity
  residual.c  R(q) for compressible Navier-Stokes (Eq. 1), Rusanov + BR2
  linalg.c    element-Jacobi blocks (Eq. 9), dense LU, p-transfers
  solvers.c   FD Jv (Eq. 8), nonlinear pMG preconditioner (Eqs. 11-16, 22-26),
              FGMRES, ESDIRK + PTC (Eqs. 2, 5-7), ROW (Eq. 3), steady PTC/SER (Eq. 10)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["tables.c", "level.c", "residual.c", "linalg.c", "solvers.c", "api.c"]
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_liboracle.so with gcc (no GPU needed)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp]
        # OpenMP over elements where the toolchain has it (element results do not depend
        # on the thread count); a plain single-threaded build otherwise
        r = subprocess.run(base + ["-fopenmp"] + srcs + ["-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base + srcs + ["-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, PD, C.c_int, PI, C.c_int, PI, PD]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_residual.argtypes = [C.c_void_p, C.c_int, PD, PD]
        L.or_elem_residual.argtypes = [C.c_void_p, C.c_int, PD, C.c_int, PD, PD]
        L.or_jvp.argtypes = [C.c_void_p, PD, PD, PD, C.c_double, C.c_double, PD]
        L.or_elem_blocks.argtypes = [C.c_void_p, C.c_int, PD, C.c_double, PI, C.c_int, PD]
        L.or_lu_factor.argtypes = [C.c_int, PD, PI]
        L.or_lu_solve.argtypes = [C.c_int, PD, PI, PD]
        L.or_lu_factor_div.argtypes = [C.c_int, PD, PI]
        L.or_lu_solve_div.argtypes = [C.c_int, PD, PI, PD]
        L.or_restrict.argtypes = [C.c_void_p, C.c_int, PD, PD]
        L.or_prolong.argtypes = [C.c_void_p, C.c_int, PD, PD]
        L.or_pmg_setup.argtypes = [C.c_void_p, PD, C.c_int, PI, C.c_double, C.c_double, C.c_int, C.c_int,
                                   C.c_double]
        L.or_neighbours.argtypes = [C.c_void_p, PI]
        L.or_nbr_blocks.argtypes = [C.c_void_p, C.c_int, PD, PI, PD]
        L.or_mbnk_matvec.argtypes = [C.c_void_p, C.c_int, PD, PD]
        L.or_mbnk_solve.argtypes = [C.c_void_p, C.c_int, PD]
        L.or_mbnk_last_iters.restype = C.c_int
        L.or_mbnk_last_relres.restype = C.c_double
        L.or_pmg_apply.argtypes = [C.c_void_p, PD, PD, PD, PD]
        L.or_block_solve.argtypes = [C.c_void_p, C.c_int, PD]
        L.or_gmres.argtypes = [C.c_void_p, PD, PD, PD, PD, C.c_int, C.c_double, C.c_int, C.c_double,
                               C.c_double, C.c_int, C.c_void_p]
        L.or_esdirk_step.argtypes = [C.c_void_p, C.c_int, PD, PD, C.c_double, PD, C.c_void_p, C.c_void_p]
        L.or_row_step.argtypes = [C.c_void_p, C.c_int, C.c_double, PD, PD, PD, C.c_double, PD,
                                  C.c_void_p, C.c_void_p]
        L.or_ptc_steady.argtypes = [C.c_void_p, PD, C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_void_p, C.c_void_p, PD]
        L.or_pmg_steady.argtypes = [C.c_void_p, PD, C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_void_p, C.c_void_p, PD]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_max_threads.restype = C.c_int
        L.or_table.argtypes = [C.c_int, C.c_int, PD]
        L.or_transfer.argtypes = [C.c_int, C.c_int, PD, PD]
        L.or_jacobian.argtypes = [C.c_void_p, C.c_int, PD]
        L.or_level_np.argtypes = [C.c_void_p, C.c_int]
        L.or_level_np.restype = C.c_int
        L.or_pairs.argtypes = [C.c_void_p, C.c_int, PI, PI, PI]
        L.or_pairs.restype = C.c_int
        L.or_flux_inviscid.argtypes = [C.c_void_p, PD, PD]
        L.or_flux_viscous.argtypes = [C.c_void_p, PD, PD, C.c_int, PD]
        L.or_rusanov.argtypes = [C.c_void_p, PD, PD, PD, PD]
        L.or_roe.argtypes = [C.c_void_p, PD, PD, PD, PD]
        L.or_weiss_smith.argtypes = [C.c_void_p, PD, PD, PD, PD]
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's element loops (OpenMP builds); returns the count in effect."""
    lib().or_set_threads(int(n))
    return int(lib().or_max_threads())


def max_threads() -> int:
    return int(lib().or_max_threads())


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(PD)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(PI)


class GmresStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("relres", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("kdim", C.c_int), ("maxit_gmres", C.c_int), ("max_ptc", C.c_int), ("nlev", C.c_int),
                ("nsmooth", C.c_int * 4), ("use_pmg", C.c_int), ("tol_gmres", C.c_double),
                ("tol_newton", C.c_double), ("eps", C.c_double), ("dtau", C.c_double),
                ("inv_dtau_star", C.c_double), ("mbnk", C.c_int), ("mbnk_maxit", C.c_int),
                ("mbnk_tol", C.c_double), ("nonlinear", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("n_ptc", C.c_int), ("n_gmres", C.c_int), ("converged", C.c_int), ("final_res", C.c_double)]


def table(p: int, g: int = 2) -> dict:
    n = p + 1
    out = np.zeros(2 * n + n * n + 6 * n + 2)
    lib().or_table(p, g, _d(out))
    o = 0

    def take(k):
        nonlocal o
        r = out[o:o + k]
        o += k
        return r
    t = dict(x=take(n), w=take(n), D=take(n * n).reshape(n, n), lm=take(n), lp=take(n), dlm=take(n),
             dlp=take(n), gLd=take(n), gRd=take(n))
    t["gLf"], t["gRf"] = take(2)
    return t


def transfer(p0: int, p1: int):
    G = np.zeros((p1 + 1) * (p0 + 1))
    P = np.zeros((p0 + 1) * (p1 + 1))
    lib().or_transfer(p0, p1, _d(G), _d(P))
    return G.reshape(p1 + 1, p0 + 1), P.reshape(p0 + 1, p1 + 1)


class Oracle:
    """One mesh with its p-levels (levels[0] finest)."""

    def __init__(self, mesh: dict, phys, levels):
        self.mesh, self.levels = mesh, list(levels)
        self.d, self.E = mesh["d"], mesh["E"]
        self.nv = self.d + 2
        g = np.ascontiguousarray(mesh["gnodes"], dtype=np.float64)
        f = np.ascontiguousarray(mesh["faces"], dtype=np.int32)
        pl = np.array(self.levels, dtype=np.int32)
        ph = np.zeros(11)                           # gamma, Pr, mu, eta, qinf[5], flux code, Ur floor
        src = np.asarray(phys.packed() if hasattr(phys, "packed") else phys, dtype=np.float64)
        ph[:len(src)] = src
        if len(src) <= 10:
            ph[10] = 1.0
        self.flux = ("rusanov", "roe", "weiss_smith")[int(ph[9])]
        self._keep = (g, f, pl, ph)
        self.h = lib().or_create(self.d, self.E, mesh["qg"], _d(g), len(f), _i(f), len(pl), _i(pl), _d(ph))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def np_(self, l=0):
        return (self.levels[l] + 1) ** self.d

    def shape(self, l=0):
        return (self.nv, self.np_(l), self.E)

    def residual(self, q, l=0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        R = np.zeros(self.shape(l))
        lib().or_residual(self.h, l, _d(q), _d(R))
        return R

    def jvp(self, q, Rq, v, eps, shift):
        out = np.zeros(self.shape(0))
        lib().or_jvp(self.h, _d(np.ascontiguousarray(q)), _d(np.ascontiguousarray(Rq)),
                     _d(np.ascontiguousarray(v)), eps, shift, _d(out))
        return out

    def elem_blocks(self, q, shift, elems, l=0):
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        nd = self.nv * self.np_(l)
        M = np.zeros((len(elems), nd, nd))
        lib().or_elem_blocks(self.h, l, _d(np.ascontiguousarray(q)), shift, _i(elems), len(elems), _d(M))
        return M

    def elem_residual(self, q, e, qe, l=0):
        """R_e with q_e replaced by qe (requires residual(q, l) first)."""
        out = np.zeros((self.nv, self.np_(l)))
        lib().or_elem_residual(self.h, l, _d(np.ascontiguousarray(q)), e, _d(np.ascontiguousarray(qe)), _d(out))
        return out

    def inviscid_flux(self, q):
        """f(q) as [d][nv] for one conservative state."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        f = np.zeros((3, 5))
        lib().or_flux_inviscid(self.h, _d(q), _d(f))
        return f[:self.d, :self.nv].copy()

    def common_flux(self, qL, qR, n, kind=None):
        """The inviscid common flux along the scaled normal n ("rusanov", "roe" or
        "weiss_smith"; default: the context's physics)."""
        kind = kind or self.flux
        qL, qR, n = (np.ascontiguousarray(a, dtype=np.float64) for a in (qL, qR, n))
        F = np.zeros(5)
        fn = {"roe": lib().or_roe, "rusanov": lib().or_rusanov, "weiss_smith": lib().or_weiss_smith}[kind]
        fn(self.h, _d(qL), _d(qR), _d(n), _d(F))
        return F[:self.nv].copy()

    def restrict(self, x0, l=0):
        out = np.zeros(self.shape(l + 1))
        lib().or_restrict(self.h, l, _d(np.ascontiguousarray(x0)), _d(out))
        return out

    def prolong(self, x1, l=0):
        out = np.zeros(self.shape(l))
        lib().or_prolong(self.h, l, _d(np.ascontiguousarray(x1)), _d(out))
        return out

    def jacobian_det(self, l=0):
        out = np.zeros((self.np_(l), self.E))
        lib().or_jacobian(self.h, l, _d(out))
        return out

    def pmg_setup(self, q_ref, nsmooth, c, inv_dtau_star, coarse="ej", mbnk_maxit=5, mbnk_tol=0.1):
        """coarse: "ej" (element-Jacobi blocks on every level) or "mbnk" (the matrix-based
        Newton-Krylov smoother on the coarsest level: GMRES of at most mbnk_maxit
        iterations to the relative tolerance mbnk_tol on the assembled operator)."""
        ns = np.array(nsmooth, dtype=np.int32)
        lib().or_pmg_setup(self.h, _d(np.ascontiguousarray(q_ref)), len(ns), _i(ns), c, inv_dtau_star,
                           int(coarse == "mbnk"), int(mbnk_maxit), float(mbnk_tol))

    def neighbours(self):
        """[E, 2d] face-neighbour table (-1: boundary, self or repeated neighbour)."""
        nbr = np.zeros(self.E * 2 * self.d, dtype=np.int32)
        lib().or_neighbours(self.h, _i(nbr))
        return nbr.reshape(self.E, 2 * self.d)

    def nbr_blocks(self, q, l=0):
        """[E, 2d, nd, nd] blocks -dR_e/dq_nbr(e,f) (row-major), zero where there is no neighbour."""
        nbr = np.ascontiguousarray(self.neighbours().ravel())
        nd = self.nv * self.np_(l)
        O = np.zeros(self.E * 2 * self.d * nd * nd)
        lib().or_nbr_blocks(self.h, l, _d(np.ascontiguousarray(q)), _i(nbr), _d(O))
        return O.reshape(self.E, 2 * self.d, nd, nd)

    def mbnk_matvec(self, x, l):
        """A x with the coarsest level's assembled operator of the last pmg_setup(coarse="mbnk")."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        lib().or_mbnk_matvec(self.h, l, _d(x), _d(y))
        return y

    def mbnk_solve(self, r, l):
        """(delta, iterations, relative residual estimate) of one matrix-based smoothing solve."""
        x = np.ascontiguousarray(r, dtype=np.float64).copy()
        lib().or_mbnk_solve(self.h, l, _d(x))
        return x, int(lib().or_mbnk_last_iters()), float(lib().or_mbnk_last_relres())

    def pmg_apply(self, q, Rq, X):
        Y = np.zeros(self.shape(0))
        lib().or_pmg_apply(self.h, _d(np.ascontiguousarray(q)), _d(np.ascontiguousarray(Rq)),
                           _d(np.ascontiguousarray(X)), _d(Y))
        return Y

    def block_solve(self, x, l=0):
        x = np.ascontiguousarray(x, dtype=np.float64).copy()
        lib().or_block_solve(self.h, l, _d(x))
        return x

    def gmres(self, q, Rq, b, kdim, tol, maxit, shift, eps=1e-6, use_pmg=False):
        x = np.zeros(self.shape(0))
        st = GmresStats()
        lib().or_gmres(self.h, _d(np.ascontiguousarray(q)), _d(np.ascontiguousarray(Rq)),
                       _d(np.ascontiguousarray(b)), _d(x), kdim, tol, maxit, shift, eps, int(use_pmg),
                       C.byref(st))
        return x, dict(iters=st.iters, restarts=st.restarts, relres=st.relres)

    @staticmethod
    def opts(kdim=30, maxit_gmres=300, max_ptc=100, nsmooth=(2, 2), use_pmg=True, tol_gmres=1e-1,
             tol_newton=1e-8, eps=1e-6, dtau=1.0, inv_dtau_star=0.0, coarse="ej", mbnk_maxit=5, mbnk_tol=0.1,
             nonlinear="jfnk"):
        """nonlinear: the ESDIRK stage solver, "jfnk" (Newton-Krylov) or "pmg" (V-cycles)."""
        o = SolveOpts()
        o.nonlinear = {"jfnk": 0, "pmg": 1}[nonlinear]
        if o.nonlinear and not use_pmg:
            raise ValueError("the pMG nonlinear solver needs the pMG levels (use_pmg)")
        o.mbnk, o.mbnk_maxit, o.mbnk_tol = int(coarse == "mbnk"), int(mbnk_maxit), float(mbnk_tol)
        o.kdim, o.maxit_gmres, o.max_ptc, o.nlev = kdim, maxit_gmres, max_ptc, len(nsmooth)
        for i, n in enumerate(nsmooth):
            o.nsmooth[i] = n
        o.use_pmg, o.tol_gmres, o.tol_newton, o.eps, o.dtau = int(use_pmg), tol_gmres, tol_newton, eps, dtau
        o.inv_dtau_star = inv_dtau_star
        return o

    def esdirk_step(self, A, b, dt, q, opts):
        A = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        st = StepStats()
        lib().or_esdirk_step(self.h, len(b), _d(A), _d(b), dt, _d(q), C.byref(opts), C.byref(st))
        return q, dict(n_ptc=st.n_ptc, n_gmres=st.n_gmres, converged=st.converged, final_res=st.final_res)

    def row_step(self, gam, a, c, m, dt, q, opts):
        a, c, m = (np.ascontiguousarray(x, dtype=np.float64) for x in (a, c, m))
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        st = StepStats()
        lib().or_row_step(self.h, len(m), gam, _d(a), _d(c), _d(m), dt, _d(q), C.byref(opts), C.byref(st))
        return q, dict(n_ptc=st.n_ptc, n_gmres=st.n_gmres, converged=st.converged, final_res=st.final_res)

    def pmg_steady(self, q, dtau_init, dtau_max, tol_rel, max_it, opts):
        """The pMG nonlinear solver (one nonlinear V-cycle per iteration, Sec. 3.1)."""
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        st = StepStats()
        hist = np.zeros(max_it + 1)
        lib().or_pmg_steady(self.h, _d(q), dtau_init, dtau_max, tol_rel, max_it, C.byref(opts), C.byref(st),
                            _d(hist))
        return q, dict(n_ptc=st.n_ptc, converged=st.converged, final_res=st.final_res, hist=hist[:st.n_ptc + 1])

    def ptc_steady(self, q, dtau_init, dtau_max, tol_rel, max_it, opts):
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        st = StepStats()
        hist = np.zeros(max_it + 1)
        lib().or_ptc_steady(self.h, _d(q), dtau_init, dtau_max, tol_rel, max_it, C.byref(opts), C.byref(st),
                            _d(hist))
        return q, dict(n_ptc=st.n_ptc, n_gmres=st.n_gmres, converged=st.converged, final_res=st.final_res,
                       hist=hist[:st.n_ptc + 1])
