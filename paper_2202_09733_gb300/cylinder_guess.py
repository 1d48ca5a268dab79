"""The learned-guess protocol on the unsteady low-Mach cylinder: ESDIRK3 steps of the 96 x 192
O-mesh (p = 3, Ma 0.05, Re 150, CFL 50, pMG p{3-2} n{2-2}, Newton tolerance 1e-8 on
RMS(a_ii dt F)), the per-element network trained online on the first --train-steps steps
and then used without further training; each variant runs the same number of steps from
the same state, and the steps after the training window are timed with CUDA events.

    python -m paper_2202_09733_gb300.cylinder_guess [--steps 400] [--train-steps 100]
                                                    [--variants fp64_qn,mixed_qn,mixed_extrap,mixed_mlp]

Variants: fp64_qn (the plain FP64 method, the paper's guess q^n), mixed_qn (FP32
preconditioner), mixed_extrap (best of q^n and the quadratic extrapolation in time),
mixed_mlp (also the network-corrected extrapolation; 10 Adam steps of 4096 samples after
each of the first --train-steps steps).  Prints one JSON line: per variant the seconds per
timed step, Newton and FGMRES iterations per timed step, candidate picks, and the final
state's distance to the first variant's.
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np
import torch

from . import api, workloads as w, tableaux as T
from . import build as B


def make_net(ctx, seed=0, hidden=128):
    K0, O = api.fr_mlp_dims(ctx)
    rng = np.random.default_rng(seed)
    P = [rng.standard_normal((hidden, K0)) / math.sqrt(K0), np.zeros(hidden),
         rng.standard_normal((hidden, hidden)) / math.sqrt(hidden), np.zeros(hidden),
         rng.standard_normal((O, hidden)) / math.sqrt(hidden) * 0.1, np.zeros(O)]
    return api.MLP(K0, hidden, O, np.concatenate([x.reshape(-1) for x in P]).astype(np.float32))


def run(steps=400, train_steps=100, variants=("fp64_qn", "mixed_qn", "mixed_extrap", "mixed_mlp"), nr=96, nt=192):
    wl = w.cylinder_unsteady(nr=nr, nt=nt)
    A, b = T.esdirk3()
    out = {"workload": f"cylinder_unsteady {nr}x{nt} O-mesh p=3 (Ma 0.05, Re 150), ESDIRK3 dt = 50x explicit, "
                       "Newton tol 1e-8, pMG p{3-2} n{2-2}, FGMRES(30) tol 1e-2",
           "steps": steps, "train_steps": train_steps, "timed_steps": steps - train_steps, "variants": {}}
    ref = None
    for name in variants:
        prec = "fp64" if name.startswith("fp64") else "mixed"
        guess = name.split("_", 1)[1]
        ctx = api.fr_create(wl.mesh, wl.phys, wl.levels)
        net = None
        if guess == "mlp":
            net = make_net(ctx)
            api.fr_set_mlp(ctx, net)

        def opts(train):
            return api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2,
                                  tol_newton=1e-8, dtau=wl.dt, inv_dtau_star=1.0 / wl.dt, precision=prec,
                                  guess=guess, train_iters=10 if train else 0, train_batch=4096, lr=1e-3)
        q = torch.from_numpy(np.ascontiguousarray(wl.q0)).cuda()
        o_train, o_use = opts(guess == "mlp"), opts(False)
        losses = []
        for k in range(train_steps):
            st = api.esdirk_step(ctx, A, b, wl.dt, q, o_train)
            if guess == "mlp":
                losses.append(st["train_loss"])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sts = []
        e0.record()
        for k in range(steps - train_steps):
            sts.append(api.esdirk_step(ctx, A, b, wl.dt, q, o_use))
        e1.record()
        torch.cuda.synchronize()
        if ref is None:
            ref = q.clone()
        nt_ = max(1, len(sts))
        v = {"s_per_step": e0.elapsed_time(e1) / 1e3 / nt_,
             "newton_per_step": float(np.mean([s["n_ptc"] for s in sts])),
             "gmres_per_step": float(np.mean([s["n_gmres"] for s in sts])),
             "picks_qn_extrap_mlp": [int(sum(s["guess_pick"][i] for s in sts)) for i in range(3)],
             "converged_steps": int(sum(s["converged"] for s in sts)),
             "state_vs_first_variant_maxrel": float(((q - ref).abs().max() / ref.abs().max()).item())}
        if losses:
            v["train_loss_first_last"] = [losses[0], losses[-1]]
        out["variants"][name] = v
        del ctx
        torch.cuda.empty_cache()
    vv = out["variants"]
    if "fp64_qn" in vv:
        for name in vv:
            if name != "fp64_qn":
                out[f"speedup_{name}_vs_fp64_qn"] = vv["fp64_qn"]["s_per_step"] / vv[name]["s_per_step"]
    if "mixed_extrap" in vv and "mixed_mlp" in vv:
        out["mlp_vs_extrap"] = vv["mixed_extrap"]["s_per_step"] / vv["mixed_mlp"]["s_per_step"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--train-steps", type=int, default=100)
    ap.add_argument("--variants", default="fp64_qn,mixed_qn,mixed_extrap,mixed_mlp")
    ap.add_argument("--nr", type=int, default=96)
    ap.add_argument("--nt", type=int, default=192)
    a = ap.parse_args(argv)
    B.build()
    torch.cuda.set_device(0)
    print(json.dumps(run(a.steps, a.train_steps, tuple(a.variants.split(",")), a.nr, a.nt)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
