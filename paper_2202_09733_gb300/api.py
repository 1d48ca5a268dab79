"""Thin Python binding of the frpmg C ABI.

The functions carry the C names and only marshal arguments: torch CUDA tensors supply
device memory (their data pointers) and the current torch stream supplies the CUDA
stream.  Every step of the computation runs in libfrpmg.so; if the library is missing
the first call raises (there is no CPU path)."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as N


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t: torch.Tensor, dtype=torch.float64, name="tensor"):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return C.c_void_p(t.data_ptr())


@dataclass
class Context:
    handle: C.c_void_p
    d: int
    E: int
    levels: list
    nv: int
    _keep: tuple = field(default=(), repr=False)

    def np_(self, level=0):
        return (self.levels[level] + 1) ** self.d

    def shape(self, level=0):
        return (self.nv, self.np_(level), self.E)

    def nd(self, level=0):
        return self.nv * self.np_(level)

    def empty(self, level=0):
        return torch.empty(self.shape(level), dtype=torch.float64, device="cuda")

    def num_colors(self):
        n = C.c_int()
        N.check(N.load().fr_num_colors(self.handle, C.byref(n)), "fr_num_colors")
        return n.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                N.load().fr_destroy(h)
            except Exception:
                pass
            self.handle = C.c_void_p()


def fr_create(mesh: dict, phys, levels) -> Context:
    """Create a context on the current CUDA device (mesh/physics as produced by
    paper_2202_09733_gb300.workloads)."""
    lib = N.load()
    torch.cuda.init()
    g = np.ascontiguousarray(mesh["gnodes"], dtype=np.float64)
    f = np.ascontiguousarray(mesh["faces"], dtype=np.int32)
    pl = np.ascontiguousarray(levels, dtype=np.int32)
    md = N.MeshDesc(mesh["d"], mesh["E"], mesh["qg"], g.ctypes.data_as(N.PD), len(f), f.ctypes.data_as(N.PI),
                    len(pl), pl.ctypes.data_as(N.PI))
    ph = N.Physics()
    ph.gamma, ph.prandtl, ph.mu, ph.eta = phys.gamma, phys.Pr, phys.mu, phys.eta
    for v, x in enumerate(phys.qinf):
        ph.qinf[v] = float(x)
    ph.flux = int(getattr(phys, "flux_code", 0))
    ph.ws_umin = float(getattr(phys, "ws_umin", 1.0))
    h = C.c_void_p()
    N.check(lib.fr_create(C.byref(h), C.byref(md), C.byref(ph)), "fr_create")
    return Context(h, mesh["d"], mesh["E"], list(levels), mesh["d"] + 2)


def fr_residual(ctx: Context, level: int, q: torch.Tensor, R: torch.Tensor | None = None, stream=None):
    R = ctx.empty(level) if R is None else R
    N.check(N.load().fr_residual(ctx.handle, level, _dev(q, name="q"), _dev(R, name="R"), _stream(stream)),
            "fr_residual")
    return R


def fr_jvp(ctx, q, Rq, v, eps=1e-6, shift=0.0, Av=None, stream=None):
    Av = ctx.empty(0) if Av is None else Av
    N.check(N.load().fr_jvp(ctx.handle, _dev(q), _dev(Rq), _dev(v), float(eps), float(shift), _dev(Av),
                            _stream(stream)), "fr_jvp")
    return Av


def fr_elem_blocks(ctx, level, q, shift, M=None, stream=None):
    """Blocks as a [E, nd(col j), nd(row r)] tensor (column-major per element)."""
    nd = ctx.nd(level)
    M = torch.empty((ctx.E, nd, nd), dtype=torch.float64, device="cuda") if M is None else M
    N.check(N.load().fr_elem_blocks(ctx.handle, level, _dev(q), float(shift), _dev(M), _stream(stream)),
            "fr_elem_blocks")
    return M


def fr_elem_blocks_f32(ctx, level, q32, shift, method="local", M=None, stream=None):
    """FP32 blocks of the FP32 state q32 as a [E, nd(col j), nd(row r)] float32 tensor;
    method "local" (element by element) or "colour" (whole-level evaluations)."""
    nd = ctx.nd(level)
    M = torch.empty((ctx.E, nd, nd), dtype=torch.float32, device="cuda") if M is None else M
    meth = {"local": 0, "colour": 1}[method]
    N.check(N.load().fr_elem_blocks_f32(ctx.handle, level, _dev(q32, torch.float32, "q32"), float(shift),
                                        _dev(M, torch.float32, "M"), meth, _stream(stream)), "fr_elem_blocks_f32")
    return M


def fr_set_block_method(ctx, method):
    """The method pmg_setup uses for the FP32 blocks: "local" (default) or "colour"."""
    N.check(N.load().fr_set_block_method(ctx.handle, {"local": 0, "colour": 1}[method]), "fr_set_block_method")


def fr_nbr_blocks(ctx, level, q, shift, stream=None):
    """(M, O): element blocks [E, nd(col), nd(row)] and face-neighbour blocks
    [E, 2d, nd(col), nd(row)] (column-major per block) of the shifted Jacobian."""
    nd, nf = ctx.nd(level), 2 * ctx.d
    M = torch.empty((ctx.E, nd, nd), dtype=torch.float64, device="cuda")
    O = torch.empty((ctx.E, nf, nd, nd), dtype=torch.float64, device="cuda")
    N.check(N.load().fr_nbr_blocks(ctx.handle, level, _dev(q), float(shift), _dev(M), _dev(O), _stream(stream)),
            "fr_nbr_blocks")
    return M, O


def fr_neighbour_table(ctx):
    """[E, 2d] face-neighbour table (-1: boundary, self or repeated neighbour)."""
    nbr = np.zeros(2 * ctx.d * ctx.E, dtype=np.int32)
    N.check(N.load().fr_neighbour_table(ctx.handle, nbr.ctypes.data_as(N.PI)), "fr_neighbour_table")
    return nbr.reshape(2 * ctx.d, ctx.E).T.copy()


def fr_mbnk_operator(ctx, level, precision="fp64", stream=None):
    """(Md, O) of the last pmg_setup(coarse="mbnk"): [E, nd(col), nd(row)] and
    [E, 2d, nd(col), nd(row)] in the cycle's precision; level is the coarsest level used."""
    nd, nf = ctx.nd(level), 2 * ctx.d
    dt = torch.float32 if _prec(precision) else torch.float64
    Md = torch.empty((ctx.E, nd, nd), dtype=dt, device="cuda")
    O = torch.empty((ctx.E, nf, nd, nd), dtype=dt, device="cuda")
    N.check(N.load().fr_mbnk_operator(ctx.handle, _dev(Md, dt), _dev(O, dt), _stream(stream)), "fr_mbnk_operator")
    return Md, O


def fr_mbnk_last(ctx):
    """(iterations, relative residual estimate) of the last matrix-based smoothing solve."""
    it, rel = C.c_int(), C.c_double()
    N.check(N.load().fr_mbnk_last(ctx.handle, C.byref(it), C.byref(rel)), "fr_mbnk_last")
    return it.value, rel.value


def fr_block_factor(ctx, level, M, perm=None, stream=None):
    perm = torch.empty((ctx.E, ctx.nd(level)), dtype=torch.int32, device="cuda") if perm is None else perm
    N.check(N.load().fr_block_factor(ctx.handle, level, _dev(M), _dev(perm, torch.int32), _stream(stream)),
            "fr_block_factor")
    return perm


def fr_block_solve(ctx, level, M, perm, x, stream=None):
    N.check(N.load().fr_block_solve(ctx.handle, level, _dev(M), _dev(perm, torch.int32), _dev(x), _stream(stream)),
            "fr_block_solve")
    return x


LU_METHODS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}


def fr_block_factor_f32(ctx, level, M, method="auto", perm=None, stream=None):
    """In-place LU of FP32 blocks M [E, nd, nd] (column-major per element); method "auto"
    (tensor cores where the block size allows), "cuda_cores" or "tensor_cores"."""
    perm = torch.empty((ctx.E, ctx.nd(level)), dtype=torch.int32, device="cuda") if perm is None else perm
    N.check(N.load().fr_block_factor_f32(ctx.handle, level, _dev(M, torch.float32, "M"), _dev(perm, torch.int32),
                                         LU_METHODS[method], _stream(stream)), "fr_block_factor_f32")
    return perm


def fr_block_solve_f32(ctx, level, M, perm, x, stream=None):
    N.check(N.load().fr_block_solve_f32(ctx.handle, level, _dev(M, torch.float32, "M"), _dev(perm, torch.int32),
                                        _dev(x, torch.float32, "x"), _stream(stream)), "fr_block_solve_f32")
    return x


def fr_set_lu_method(ctx, method):
    """The FP32 factorisation pmg_setup uses: "auto" (default) or "cuda_cores"."""
    N.check(N.load().fr_set_lu_method(ctx.handle, {"auto": 0, "cuda_cores": 1}[method]), "fr_set_lu_method")


def fr_block_to_half(ctx, level, M, stream=None):
    """(H, dg): half-width copy of FP32 factors M [E, nd, nd]: H float16 [E, nd, ldh]
    (column k of L and column-scaled U in H[e, k, :nd], ldh = nd rounded up to even), dg
    float32 [E, nd, 2] = (1/u_kk, column scale)."""
    E, nd = M.shape[0], M.shape[1]
    H = torch.empty((E, nd, (nd + 1) // 2 * 2), dtype=torch.float16, device="cuda")
    dg = torch.empty((E, nd, 2), dtype=torch.float32, device="cuda")
    N.check(N.load().fr_block_to_half(ctx.handle, level, _dev(M, torch.float32, "M"), _dev(H, torch.float16, "H"),
                                      _dev(dg, torch.float32, "dg"), _stream(stream)), "fr_block_to_half")
    return H, dg


def fr_block_solve_half(ctx, level, H, dg, perm, x, stream=None):
    N.check(N.load().fr_block_solve_half(ctx.handle, level, _dev(H, torch.float16, "H"), _dev(dg, torch.float32, "dg"),
                                         _dev(perm, torch.int32), _dev(x, torch.float32, "x"), _stream(stream)),
            "fr_block_solve_half")
    return x


def fr_spectral_decay(ctx, level, q, var=1, eta=None, stream=None):
    """Sec. 3.3 spectral-decay indicator per element (device float64 [E]) of variable var."""
    eta = torch.empty(ctx.E, dtype=torch.float64, device="cuda") if eta is None else eta
    N.check(N.load().fr_spectral_decay(ctx.handle, int(level), _dev(q), int(var), _dev(eta, torch.float64, "eta"),
                                       _stream(stream)), "fr_spectral_decay")
    return eta


def fr_padapt_mark(ctx, eta, p_in, p_min=1, p_max=4, nu_min=1e-3, nu_max=0.2, stream=None):
    """Sec. 3.3 marking rule: the new element degrees (device int32 [E])."""
    p_out = torch.empty_like(p_in)
    N.check(N.load().fr_padapt_mark(ctx.handle, _dev(eta, torch.float64, "eta"), _dev(p_in, torch.int32, "p_in"),
                                    int(p_min), int(p_max), float(nu_min), float(nu_max),
                                    _dev(p_out, torch.int32, "p_out"), _stream(stream)), "fr_padapt_mark")
    return p_out


def fr_nested_hierarchy(p_elem, gap, nlevels):
    """Sec. 3.3 nested p-hierarchy of one element (host)."""
    out = (C.c_int * int(nlevels))()
    N.check(N.load().fr_nested_hierarchy(int(p_elem), int(gap), int(nlevels), out), "fr_nested_hierarchy")
    return [int(x) for x in out]


def fr_set_cycle_scaling(ctx, on):
    """Drive the FP64 preconditioner cycle with a scaled X (as the FP32 one is)."""
    N.check(N.load().fr_set_cycle_scaling(ctx.handle, int(bool(on))), "fr_set_cycle_scaling")


def fr_set_precision_fallback(ctx, on):
    """ptc_steady: switch a stalled FP32 preconditioner to the FP64 cycle (default True)."""
    N.check(N.load().fr_set_precision_fallback(ctx.handle, int(bool(on))), "fr_set_precision_fallback")


def fr_set_lu_storage(ctx, storage):
    """How pmg_setup keeps the FP32 factors for the smoother's solves: "fp32" (default) or
    "half" (binary16 entries with per-column scales, half the bytes per solve)."""
    N.check(N.load().fr_set_lu_storage(ctx.handle, {"fp32": 0, "half": 1}[storage]), "fr_set_lu_storage")


def fr_restrict(ctx, level, xf, xc=None, stream=None):
    xc = ctx.empty(level + 1) if xc is None else xc
    N.check(N.load().fr_restrict(ctx.handle, level, _dev(xf), _dev(xc), _stream(stream)), "fr_restrict")
    return xc


def fr_prolong(ctx, level, xc, xf=None, stream=None):
    xf = ctx.empty(level) if xf is None else xf
    N.check(N.load().fr_prolong(ctx.handle, level, _dev(xc), _dev(xf), _stream(stream)), "fr_prolong")
    return xf


def _coarse(coarse):
    if coarse not in ("ej", "mbnk"):
        raise ValueError('coarse must be "ej" (element-Jacobi) or "mbnk" (matrix-based Newton-Krylov)')
    return int(coarse == "mbnk")


def pmg_setup(ctx, q_ref, nsmooth, c, inv_dtau_star, precision="fp64", stream=None, coarse="ej", mbnk_maxit=5,
              mbnk_tol=0.1):
    """precision: "fp64" (reproducible) or "mixed" (FP32 cycle, blocks and LU).  coarse:
    "ej" (element-Jacobi smoothing everywhere) or "mbnk" (the matrix-based Newton-Krylov
    smoother on the coarsest level: GMRES of at most mbnk_maxit iterations to mbnk_tol)."""
    o = N.PmgOpts()
    o.nlevels = len(nsmooth)
    for i, n in enumerate(nsmooth):
        o.nsmooth[i] = int(n)
    o.c, o.inv_dtau_star = float(c), float(inv_dtau_star)
    o.precision = _prec(precision)
    o.coarse_smoother, o.mbnk_maxit, o.mbnk_tol = _coarse(coarse), int(mbnk_maxit), float(mbnk_tol)
    N.check(N.load().pmg_setup(ctx.handle, _dev(q_ref), C.byref(o), _stream(stream)), "pmg_setup")


def pmg_precondition(ctx, q, Rq, X, Y=None, stream=None):
    Y = ctx.empty(0) if Y is None else Y
    N.check(N.load().pmg_precondition(ctx.handle, _dev(q), _dev(Rq), _dev(X), _dev(Y), _stream(stream)),
            "pmg_precondition")
    return Y


def gmres_solve(ctx, q, Rq, b, x=None, kdim=30, maxit=300, tol=1e-1, eps=1e-6, shift=0.0, use_pmg=False,
                stream=None):
    x = ctx.empty(0) if x is None else x
    o = N.GmresOpts(int(kdim), int(maxit), int(bool(use_pmg)), float(tol), float(eps), float(shift))
    st = N.GmresStats()
    N.check(N.load().gmres_solve(ctx.handle, _dev(q), _dev(Rq), _dev(b), _dev(x), C.byref(o), C.byref(st),
                                 _stream(stream)), "gmres_solve")
    return x, dict(iters=st.iters, restarts=st.restarts, relres=st.relres)


def _prec(p):
    if p in ("fp64", 0, None):
        return 0
    if p in ("mixed", "fp32", 1):
        return 1
    raise ValueError(f"precision must be 'fp64' or 'mixed', not {p!r}")


def solve_opts(kdim=30, maxit_gmres=300, max_ptc=100, nsmooth=(2, 2), use_pmg=True, tol_gmres=1e-1,
               tol_newton=1e-8, eps=1e-6, dtau=1.0, inv_dtau_star=0.0, precision="fp64", guess="qn",
               train_iters=0, train_batch=4096, lr=1e-3, coarse="ej", mbnk_maxit=5, mbnk_tol=0.1,
               nonlinear="jfnk"):
    """guess: "qn" (the paper's q^n), "extrap" (best of q^n and the quadratic extrapolation
    in time) or "mlp" (also the network-corrected extrapolation); train_iters > 0 trains
    the attached network after every ESDIRK step.  coarse, mbnk_maxit, mbnk_tol: the
    coarsest level's smoother, as in pmg_setup.  nonlinear: the ESDIRK stage solver,
    "jfnk" (pseudo-time Newton updates by FGMRES) or "pmg" (one V-cycle per update)."""
    o = N.SolveOpts()
    o.kdim, o.maxit_gmres, o.max_ptc, o.nlevels = int(kdim), int(maxit_gmres), int(max_ptc), len(nsmooth)
    for i, n in enumerate(nsmooth):
        o.nsmooth[i] = int(n)
    o.use_pmg, o.tol_gmres, o.tol_newton, o.eps = int(bool(use_pmg)), float(tol_gmres), float(tol_newton), float(eps)
    o.dtau, o.inv_dtau_star = float(dtau), float(inv_dtau_star)
    o.precision = _prec(precision)
    guesses = {"qn": 0, "extrap": 1, "mlp": 2}
    if guess not in guesses:
        raise ValueError(f"guess must be one of {sorted(guesses)}")
    o.guess, o.train_iters, o.train_batch, o.lr = guesses[guess], int(train_iters), int(train_batch), float(lr)
    o.coarse_smoother, o.mbnk_maxit, o.mbnk_tol = _coarse(coarse), int(mbnk_maxit), float(mbnk_tol)
    if nonlinear not in ("jfnk", "pmg"):
        raise ValueError('nonlinear must be "jfnk" or "pmg"')
    o.nonlinear = int(nonlinear == "pmg")
    return o


def _stats(st):
    return dict(n_ptc=st.n_ptc, n_gmres=st.n_gmres, converged=st.converged, final_res=st.final_res,
                guess_rms=list(st.guess_rms), guess_pick=list(st.guess_pick), guess_beta=st.guess_beta,
                train_loss=st.train_loss, prec_switch_it=st.prec_switch_it)


def esdirk_step(ctx, A, b, dt, q, opts, stream=None, allow_not_converged=True):
    A = np.asarray(A, dtype=np.float64)
    s = len(b)
    tab = N.EsdirkTableau()
    tab.stages = s
    for i in range(s):
        tab.b[i] = float(b[i])
        for j in range(s):
            tab.A[i * s + j] = float(A[i, j])
    st = N.StepStats()
    rc = N.load().esdirk_step(ctx.handle, C.byref(tab), float(dt), _dev(q), C.byref(opts), C.byref(st),
                              _stream(stream))
    N.check(rc, "esdirk_step", allow=(-4,) if allow_not_converged else ())
    return _stats(st)


def row_step(ctx, gamma, a, c, m, dt, q, opts, stream=None, allow_not_converged=True):
    s = len(m)
    tab = N.RowTableau()
    tab.stages, tab.gamma = s, float(gamma)
    for i in range(s):
        tab.m[i] = float(m[i])
        for j in range(s):
            tab.a[i * s + j] = float(a[i][j])
            tab.c[i * s + j] = float(c[i][j])
    st = N.StepStats()
    rc = N.load().row_step(ctx.handle, C.byref(tab), float(dt), _dev(q), C.byref(opts), C.byref(st), _stream(stream))
    N.check(rc, "row_step", allow=(-4,) if allow_not_converged else ())
    return _stats(st)


def ptc_steady(ctx, q, dtau_init, dtau_max, tol_rel, max_it, opts, stream=None):
    hist = np.zeros(max_it + 1)
    st = N.StepStats()
    rc = N.load().ptc_steady(ctx.handle, _dev(q), float(dtau_init), float(dtau_max), float(tol_rel), int(max_it),
                             C.byref(opts), C.byref(st), hist.ctypes.data_as(N.PD), _stream(stream))
    N.check(rc, "ptc_steady", allow=(-4,))
    out = _stats(st)
    out["hist"] = hist[:st.n_ptc + 1]
    return out


def pmg_solve_steady(ctx, q, dtau_init, dtau_max, tol_rel, max_it, opts, stream=None):
    """The pMG nonlinear solver (one nonlinear V-cycle per iteration)."""
    hist = np.zeros(max_it + 1)
    st = N.StepStats()
    rc = N.load().pmg_solve_steady(ctx.handle, _dev(q), float(dtau_init), float(dtau_max), float(tol_rel),
                                   int(max_it), C.byref(opts), C.byref(st), hist.ctypes.data_as(N.PD),
                                   _stream(stream))
    N.check(rc, "pmg_solve_steady", allow=(-4,))
    out = _stats(st)
    out["hist"] = hist[:st.n_ptc + 1]
    return out


class MLP:
    """Per-element BF16 network of the Newton initial guess (libfrpmg mlp_*)."""

    def __init__(self, in_dim, hidden, out_dim, params: np.ndarray):
        params = np.ascontiguousarray(params, dtype=np.float32)
        self.in_dim, self.hidden, self.out_dim = int(in_dim), int(hidden), int(out_dim)
        self.nparams = hidden * in_dim + hidden + hidden * hidden + hidden + out_dim * hidden + out_dim
        if params.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {params.size}")
        h = C.c_void_p()
        N.check(N.load().mlp_create(C.byref(h), self.in_dim, self.hidden, self.out_dim,
                                    params.ctypes.data_as(N.PF)), "mlp_create")
        self.handle = h

    def params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        N.check(N.load().mlp_get_params(self.handle, out.ctypes.data_as(N.PF)), "mlp_get_params")
        return out

    def forward(self, X: torch.Tensor, Y: torch.Tensor | None = None, stream=None):
        """X: CUDA bfloat16 [B, in]; returns float32 [B, out]."""
        B = X.shape[0]
        if Y is None:
            Y = torch.empty((B, self.out_dim), dtype=torch.float32, device=X.device)
        N.check(N.load().mlp_forward(self.handle, B, _dev(X, torch.bfloat16, "X"), _dev(Y, torch.float32, "Y"),
                                     _stream(stream)), "mlp_forward")
        return Y

    def train_step(self, X: torch.Tensor, T: torch.Tensor, lr=1e-3, grads: torch.Tensor | None = None,
                   want_loss=True, stream=None):
        loss = C.c_float()
        N.check(N.load().mlp_train_step(self.handle, X.shape[0], _dev(X, torch.bfloat16, "X"),
                                        _dev(T, torch.float32, "T"), float(lr),
                                        C.byref(loss) if want_loss else None,
                                        _dev(grads, torch.float32, "grads") if grads is not None else None,
                                        _stream(stream)), "mlp_train_step")
        return loss.value if want_loss else None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                N.load().mlp_destroy(h)
            except Exception:
                pass
            self.handle = None


def fr_mlp_dims(ctx):
    i, o = C.c_int(), C.c_int()
    N.check(N.load().fr_mlp_dims(ctx.handle, C.byref(i), C.byref(o)), "fr_mlp_dims")
    return i.value, o.value


def fr_set_mlp(ctx, mlp: MLP | None):
    N.check(N.load().fr_set_mlp(ctx.handle, mlp.handle if mlp is not None else None), "fr_set_mlp")
    ctx._mlp = mlp   # keep the network alive while attached


def fr_guess_features(ctx, qn, q1, q2, Rn, dt, c, stream=None):
    """Network inputs (CUDA bfloat16 [E, in]) and the per-variable scales (s, sig)."""
    K0, _ = fr_mlp_dims(ctx)
    X = torch.empty((ctx.E, K0), dtype=torch.bfloat16, device="cuda")
    sc = np.zeros(10)
    N.check(N.load().fr_guess_features(ctx.handle, _dev(qn), _dev(q1), _dev(q2), _dev(Rn), float(dt), float(c),
                                       _dev(X, torch.bfloat16, "X"), sc.ctypes.data_as(N.PD), _stream(stream)),
            "fr_guess_features")
    return X, sc[:ctx.nv], sc[5:5 + ctx.nv]


def fr_autotune(ctx, fp64=True, fp32=False, retune=False, reps=5):
    """Tune the launch shapes of the context's levels; returns the report lines."""
    buf = C.create_string_buffer(8192)
    flags = (1 if fp64 else 0) | (2 if fp32 else 0) | (4 if retune else 0)
    N.check(N.load().fr_autotune(ctx.handle, flags, int(reps), buf, len(buf)), "fr_autotune")
    return buf.value.decode().splitlines()


def fr_get_tiles(ctx, level, precision=0):
    t = np.zeros(9, dtype=np.int32)
    N.check(N.load().fr_get_tiles(ctx.handle, int(level), int(precision), t.ctypes.data_as(N.PI)), "fr_get_tiles")
    return [int(x) for x in t]


def fr_set_tiles(ctx, level, tiles, precision=0):
    t = np.ascontiguousarray(tiles, dtype=np.int32)
    if t.size != 9:
        raise ValueError("tiles: 8 CTA sizes and the solve's G")
    N.check(N.load().fr_set_tiles(ctx.handle, int(level), int(precision), t.ctypes.data_as(N.PI)), "fr_set_tiles")


def fr_kernel_timeouts(clear=True):
    return int(N.load().fr_kernel_timeouts(int(bool(clear))))


def fr_selftest_wait_timeout():
    N.check(N.load().fr_selftest_wait_timeout(), "fr_selftest_wait_timeout")


def fr_autotune_save(path):
    N.check(N.load().fr_autotune_save(str(path).encode()), "fr_autotune_save")


def fr_autotune_load(path):
    N.check(N.load().fr_autotune_load(str(path).encode()), "fr_autotune_load")


def fr_checkpoint_save(ctx, mlp=None) -> bytes:
    """The library-side state of a time-stepping run (history, training ring, network)."""
    lib = N.load()
    h = mlp.handle if mlp is not None else None
    n = C.c_longlong()
    N.check(lib.fr_checkpoint_size(ctx.handle, h, C.byref(n)), "fr_checkpoint_size")
    buf = C.create_string_buffer(n.value)
    N.check(lib.fr_checkpoint_save(ctx.handle, h, buf, n.value), "fr_checkpoint_save")
    return buf.raw


def fr_checkpoint_load(ctx, data: bytes, mlp=None):
    buf = C.create_string_buffer(data, len(data))
    N.check(N.load().fr_checkpoint_load(ctx.handle, mlp.handle if mlp is not None else None, buf, len(data)),
            "fr_checkpoint_load")


def fr_reset_history(ctx):
    N.check(N.load().fr_reset_history(ctx.handle), "fr_reset_history")


class Batch:
    """Many independent problems advanced together (libfrpmg fr_batch_*).  problems: list of
    (mesh dict, levels); physics shared."""

    def __init__(self, problems, phys):
        lib = N.load()
        torch.cuda.init()
        self._keep = []
        descs = (N.MeshDesc * len(problems))()
        self.shapes = []
        for k, (mesh, levels) in enumerate(problems):
            g = np.ascontiguousarray(mesh["gnodes"], dtype=np.float64)
            f = np.ascontiguousarray(mesh["faces"], dtype=np.int32)
            pl = np.ascontiguousarray(levels, dtype=np.int32)
            self._keep += [g, f, pl]
            descs[k] = N.MeshDesc(mesh["d"], mesh["E"], mesh["qg"], g.ctypes.data_as(N.PD), len(f),
                                  f.ctypes.data_as(N.PI), len(pl), pl.ctypes.data_as(N.PI))
            np_ = (levels[0] + 1) ** mesh["d"]
            self.shapes.append((mesh["d"] + 2, np_, mesh["E"]))
        ph = N.Physics()
        ph.gamma, ph.prandtl, ph.mu, ph.eta = phys.gamma, phys.Pr, phys.mu, phys.eta
        for v, x in enumerate(phys.qinf):
            ph.qinf[v] = float(x)
        ph.flux = int(getattr(phys, "flux_code", 0))
        ph.ws_umin = float(getattr(phys, "ws_umin", 1.0))
        h = C.c_void_p()
        N.check(lib.fr_batch_create(C.byref(h), len(problems), descs, C.byref(ph)), "fr_batch_create")
        self.handle = h
        self.nprob = len(problems)

    def info(self):
        ng = C.c_int()
        grp = np.zeros(self.nprob, dtype=np.int32)
        off = np.zeros(self.nprob, dtype=np.int32)
        N.check(N.load().fr_batch_info(self.handle, C.byref(ng), grp.ctypes.data_as(N.PI), off.ctypes.data_as(N.PI)),
                "fr_batch_info")
        return ng.value, grp, off

    def autotune(self, fp64=True, fp32=False, retune=False, reps=5):
        buf = C.create_string_buffer(16384)
        flags = (1 if fp64 else 0) | (2 if fp32 else 0) | (4 if retune else 0)
        N.check(N.load().fr_batch_autotune(self.handle, flags, int(reps), buf, len(buf)), "fr_batch_autotune")
        return buf.value.decode().splitlines()

    def set_graphs(self, on: bool):
        N.check(N.load().fr_batch_set_graphs(self.handle, int(bool(on))), "fr_batch_set_graphs")

    def _ptrs(self, qs):
        if len(qs) != self.nprob:
            raise ValueError(f"expected {self.nprob} states")
        arr = (C.c_void_p * self.nprob)()
        for k, (t, shp) in enumerate(zip(qs, self.shapes)):
            if tuple(t.shape) != shp:
                raise ValueError(f"state {k} has shape {tuple(t.shape)}, expected {shp}")
            arr[k] = _dev(t).value
        return arr

    def residual(self, qs, Rs=None, stream=None):
        if Rs is None:
            Rs = [torch.empty_like(q) for q in qs]
        N.check(N.load().fr_batch_residual(self.handle, self._ptrs(qs), self._ptrs(Rs), _stream(stream)),
                "fr_batch_residual")
        return Rs

    def esdirk_step(self, A, b, dt, qs, opts, stream=None, allow_not_converged=True):
        A = np.asarray(A, dtype=np.float64)
        s = len(b)
        tab = N.EsdirkTableau()
        tab.stages = s
        for i in range(s):
            tab.b[i] = float(b[i])
            for j in range(s):
                tab.A[i * s + j] = float(A[i, j])
        st = (N.StepStats * self.nprob)()
        rc = N.load().fr_batch_esdirk_step(self.handle, C.byref(tab), float(dt), self._ptrs(qs), C.byref(opts), st,
                                           _stream(stream))
        N.check(rc, "fr_batch_esdirk_step", allow=(-4,) if allow_not_converged else ())
        return [_stats(x) for x in st]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                N.load().fr_batch_destroy(h)
            except Exception:
                pass
            self.handle = None
