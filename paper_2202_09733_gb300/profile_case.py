"""Run one operation of the hot path a fixed number of times on a named workload, for
external profilers (ncu):  python -m paper_2202_09733_gb300.profile_case --case tgv3d --op residual

Operations: residual (FP64), residual32 (the FP32 residual of the mixed preconditioner:
a cycle with no smoothing, one FP32 residual per level), jvp, pmg (one preconditioner
application, --precision fp64|mixed; its block solves, transfers and residuals can be
picked out with the profiler's kernel filter), lu_factor (the FP32 LU of the fine level's
element blocks, --lu auto|cuda_cores|tensor_cores, from a fresh copy of the blocks each
run), row_step (from the same state every run),
esdirk_step (ESDIRK3 at the 1e-8 Newton tolerance, successive steps).  The setup (context, blocks and
factors where the operation needs them) runs first; then --reps runs of the operation,
each followed by a device synchronisation.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np
import torch

from . import api, workloads as w, tableaux as T
from . import build as B


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="tgv3d", choices=["tgv3d", "cylinder_unsteady", "vortex2d"])
    ap.add_argument("--n", type=int, default=32, help="tgv3d: elements per direction")
    ap.add_argument("--op", default="residual",
                    choices=["residual", "residual32", "jvp", "pmg", "row_step", "esdirk_step", "lu_factor"])
    ap.add_argument("--lu-storage", default="fp32", choices=["fp32", "half"],
                    help="mixed preconditioner: the smoother's solves from FP32 or half-width factors")
    ap.add_argument("--lu", default="auto", choices=["auto", "cuda_cores", "tensor_cores"],
                    help="lu_factor: the FP32 factorisation of the fine level's element blocks")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--solve-g", type=int, default=0,
                    help="block-solve variant on every level (0 default, 1 bulk-copy kernel, 2/4/8 columns in flight)")
    a = ap.parse_args(argv)
    B.build()
    if a.case == "tgv3d":
        W = w.tgv3d(n=a.n)
    elif a.case == "cylinder_unsteady":
        W = w.cylinder_unsteady()
    else:
        W = w.vortex2d()
    ctx = api.fr_create(W.mesh, W.phys, W.levels)
    api.fr_set_lu_storage(ctx, a.lu_storage)
    if a.autotune:
        api.fr_autotune(ctx, fp64=True, fp32=True, reps=3)
    if a.solve_g:
        for l in range(len(W.levels)):
            for prec in (0, 1):
                api.fr_set_tiles(ctx, l, api.fr_get_tiles(ctx, l, prec)[:8] + [a.solve_g], precision=prec)
    q = torch.from_numpy(np.ascontiguousarray(W.q0)).cuda()
    R = api.fr_residual(ctx, 0, q)
    v = torch.from_numpy(np.random.default_rng(0).standard_normal(q.shape)).cuda()
    v /= v.norm()
    dt = W.dt
    c = 1.0 / dt + 1.0 / (0.4358665215084590 * dt)
    if a.op == "pmg":
        api.pmg_setup(ctx, q, (2,) * len(W.levels), c, 1.0 / dt, precision=a.precision)
    torch.cuda.synchronize()

    def once():
        if a.op == "residual":
            api.fr_residual(ctx, 0, q, R)
        elif a.op == "residual32":
            # the FP32 residual runs inside the mixed preconditioner; a cycle with no
            # smoothing evaluates it exactly once per level
            api.pmg_precondition(ctx, q, R, v)
        elif a.op == "jvp":
            api.fr_jvp(ctx, q, R, v, 1e-6, c)
        elif a.op == "lu_factor":
            Mw.copy_(M0)
            api.fr_block_factor_f32(ctx, 0, Mw, a.lu, perm=pw)
        elif a.op == "pmg":
            api.pmg_precondition(ctx, q, R, v)
        elif a.op == "esdirk_step":
            A, bb = T.esdirk3()
            o = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2,) * len(W.levels), tol_gmres=1e-2,
                               tol_newton=1e-8, dtau=dt, inv_dtau_star=1.0 / dt, precision=a.precision)
            api.esdirk_step(ctx, A, bb, dt, qs, o)
        elif a.op == "row_step":
            g, aa, cc, m = T.ros34pw2()
            o = api.solve_opts(kdim=30, maxit_gmres=300, nsmooth=(2,) * len(W.levels), tol_gmres=1e-6,
                               inv_dtau_star=1.0 / dt, precision=a.precision)
            qq = q.clone()
            api.row_step(ctx, g, aa, cc, m, dt, qq, o)

    qs = q.clone()   # esdirk_step: successive runs advance this state
    if a.op == "lu_factor":
        # the FP32 element blocks of the fine level at q (the mixed preconditioner's), copied
        # afresh before every factorisation
        M0 = api.fr_elem_blocks_f32(ctx, 0, q.float().contiguous(), c)
        Mw = torch.empty_like(M0)
        pw = torch.empty((ctx.E, ctx.nd(0)), dtype=torch.int32, device="cuda")
    if a.op == "residual32":
        api.pmg_setup(ctx, q, (0,) * len(W.levels), c, 1.0 / dt, precision="mixed")
    from . import _native as N
    lib = N.load()
    counts = []
    for _ in range(a.reps):
        n0 = lib.fr_kernel_launches()
        once()
        torch.cuda.synchronize()
        counts.append(int(lib.fr_kernel_launches() - n0))
    print(f"{a.case} {a.op} {a.precision}: {a.reps} runs done; kernel launches before the runs "
          f"{int(lib.fr_kernel_launches()) - sum(counts)}, per run {counts}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
