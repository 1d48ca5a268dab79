#!/usr/bin/env python
"""Benchmark of the JFNK-pMG hot path on one GB300 (or N replicas under torchrun).

Workload (the 3-D throughput case): compressible Navier-Stokes, FR p = 3 on 32^3 periodic
affine hexes (2.1 M solution points x 5 variables), Taylor-Green field plus seeded
Fourier noise (modes <= 4, amplitude 1e-3), Ma = 0.1, Re = 1600.  One step = one
ROS34PW2 step (dt = 20x the explicit limit) with the nonlinear pMG p{3-2} n{2-2}
preconditioner (element blocks and their LU evaluated at q^n inside the step, as the
paper does once per physical step) and FGMRES(30) to the paper's ROW tolerance 1e-6:
FP64 residual, Jv, Gram-Schmidt and update; the preconditioner's cycle, blocks and LU in
FP32 (the LU's trailing updates on the tensor cores), its block solves from factors
stored as binary16 with FP32 column scales (--lu-storage fp32 keeps them FP32).  The
plain FP64 step is timed beside it.  Inputs are larger than L2 (84 MB state, 13 GB of
FP32 element blocks), so no L2 flush is needed between steps.

Output: one JSON line with the step wall time (value), the FP64 residual throughput
(GDOF/s), the roofline of the residual, the end-to-end time through host buffers, the
oracle baseline on the host cores, the kernel-launch count and the SM clocks.

--impl reference times the FP64 CPU oracle (the method has no other implementation to
compare with) on a bounded sample of the same workload (an 8^3 slice at the same CFL on all host cores,
scaled to 32^3 by the element count).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "implicit step wall time @1e-8 tol: mixed/learned pMG vs FP64; residual GDOF/s"
FP64_PEAK_NOMINAL = 1.25e12        # GB300 FP64 (vector = tensor), nominal
SAMPLE_N = 8                       # oracle step sample: 8^3 hexes, scaled by (32/8)^3
PROFILES = os.path.join(ROOT, "profiles")


def profile_figure(name, key):
    """A figure an ncu summary states on a line "key: value" (None if the summary or the
    line is absent: the counters were not taken for the kernels as they stand)."""
    import re
    try:
        with open(os.path.join(PROFILES, name + ".md")) as f:
            for line in f:
                m = re.match(r"^\s*%s:\s*([0-9.eE+-]+)" % re.escape(key), line)
                if m:
                    return float(m.group(1))
    except OSError:
        pass
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="frpmg", choices=["frpmg", "reference"])
    ap.add_argument("--n", type=int, default=32, help="elements per direction")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="preconditioner precision of the timed step (the FP64 step is timed alongside)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ESDIRK3 initial-guess comparison (cylinder) and the batched step")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--lu-storage", default="half", choices=["fp32", "half"],
                    help="mixed preconditioner: the smoother's block solves read half-width factors (binary16 "
                         "with FP32 column scales: TF32's 10-bit mantissa) or FP32 ones")
    return ap.parse_args()



def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy, burst)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def half_solve_roofline(api, torch, ctx, q0, c, E, nd, reps=10):
    """Roofline of the step's dominant kernel with half-width factors, the fine-level
    block solve k_lu_solve_half: the level's FP32 blocks at q0 (shift c), factored and
    converted as pmg_setup does, one application timed with CUDA events on the stream it
    runs on (the mean of reps, after one warm-up), against its algorithmic bytes: the
    binary16 factors (nd x ldh per block), the (1/u_kk, g_k) pairs, the permutation and the
    vector read and written."""
    M = api.fr_elem_blocks_f32(ctx, 0, q0.float().contiguous(), c)
    perm = api.fr_block_factor_f32(ctx, 0, M)
    H, dg = api.fr_block_to_half(ctx, 0, M)
    del M
    x = torch.randn((nd, E), device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()
    api.fr_block_solve_half(ctx, 0, H, dg, perm, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        api.fr_block_solve_half(ctx, 0, H, dg, perm, x)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1) / reps
    ldh = H.shape[2]
    algo = E * nd * ldh * 2 + E * nd * 8 + E * nd * 4 + 2 * E * nd * 4
    peak, src = hbm_peak()
    t16 = profile_figure("lu_solve_half_tgv3d16", "dram_bytes_per_launch_half")
    del H, dg
    return {"kernel": f"k_lu_solve_half (fine-level block solve from binary16 factors, {E} blocks of {nd}x{nd}, "
                      "one application)",
            "bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": src, "algorithmic_bytes": algo,
            "achieved": algo / (t_ms * 1e-3) / 1e9, "frac": algo / (t_ms * 1e-3) / 1e9 / peak, "ms_per_launch": t_ms,
            "traffic": t16 * E / 4096 if t16 else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on tgv3d 16^3 "
                              "(4096 elements), scaled by the element count (committed ncu summary)",
            "share_of_step": "the largest kernel family of the mixed step (committed launch list)"}


def solve_roofline(tune, E, nd):
    """Roofline of the step's dominant kernel, the FP32 fine-level block solve: its time per
    launch as the autotuner measured it in this run (CUDA events, the chosen variant, on
    the blocks the first step factored) against the algorithmic bytes of one application:
    the E nd^2 FP32 factors, the permutation and the vector read and written."""
    import re
    t_ms = None
    for line in tune or []:
        if line.startswith("d=3 p=3 fp32") and "ms per G" in line:
            t_ms = min(float(x.split(":")[1]) for x in re.search(r"ms per G ([^)]*)\)", line).group(1).split())
    peak, src = hbm_peak()
    algo = E * nd * nd * 4 + E * nd * 4 + 2 * E * nd * 4
    t16 = profile_figure("lu_solve_tgv3d16_fp32_fp64", "dram_bytes_per_launch_fp32")
    out = {"kernel": f"k_lu_solve (FP32 fine-level block solve, {E} LU factors of {nd}x{nd}, one application)",
           "bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": src, "algorithmic_bytes": algo,
           "traffic": t16 * E / 4096 if t16 else None,
           "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on tgv3d 16^3 "
                             "(4096 elements), scaled by the element count (committed ncu summary)",
           "share_of_step": "the largest kernel family of the mixed step (committed launch list)"}
    if t_ms:
        out.update({"achieved": algo / (t_ms * 1e-3) / 1e9, "frac": algo / (t_ms * 1e-3) / 1e9 / peak,
                    "ms_per_launch": t_ms})
    else:
        out.update({"achieved": None, "frac": None, "note": "autotuner did not time the solve (--no-autotune)"})
    return out


def max_over_ranks(x, ws, device):
    """The largest of every rank's x (replica timings: the job takes as long as its
    slowest rank); x itself on a single rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ oracle (CPU) arm
def oracle_step_time(n_sample=SAMPLE_N, threads=None):
    """Seconds for one oracle ROS34PW2 step on an n_sample^3 slice of the workload at its CFL
    (the pMG p{3-2} n{2-2} preconditioner, FGMRES(30) to 1e-6), on `threads` host threads
    (all cores if None), with the step's stats."""
    import oracle
    from oracle import tableaux as TB
    from paper_2202_09733_gb300 import workloads as w
    used = oracle.set_threads(threads or os.cpu_count() or 1)
    W = w.tgv3d(n=n_sample)
    O = oracle.Oracle(W.mesh, W.phys, W.levels)
    g, a, c, m = TB.ros34pw2()
    opts = O.opts(kdim=30, maxit_gmres=300, nsmooth=(2, 2), tol_gmres=1e-6, inv_dtau_star=1.0 / W.dt)
    t0 = time.perf_counter()
    q, st = O.row_step(g, a, c, m, W.dt, W.q0, opts)
    return time.perf_counter() - t0, st, used


def oracle_baseline(n_full=32):
    """The oracle on this machine's host cores: R and Jv on the full workload, one thread and
    all cores; the ROS34PW2 step on an 8^3 slice (all cores) and a 4^3 slice (one thread).
    value = the 8^3 step scaled by the element count (an estimate: the slice's FGMRES count
    is reported beside it)."""
    import numpy as np
    import oracle
    from paper_2202_09733_gb300 import workloads as w
    oracle.build()
    ncores = os.cpu_count() or 1
    W = w.tgv3d(n=n_full)
    O = oracle.Oracle(W.mesh, W.phys, W.levels)
    v = np.random.default_rng(0).standard_normal(W.q0.shape)
    v /= np.linalg.norm(v)
    shift = 1.0 / W.dt + 1.0 / (0.4358665215084590 * W.dt)
    out = {}
    for label, nt in (("1", 1), ("all", ncores)):
        used = oracle.set_threads(nt)
        t0 = time.perf_counter()
        R = O.residual(W.q0)
        t1 = time.perf_counter()
        O.jvp(W.q0, R, v, 1e-6, shift)
        t2 = time.perf_counter()
        out[f"residual_s_{label}"] = t1 - t0
        out[f"jvp_s_{label}"] = t2 - t1
        out[f"threads_{label}"] = used
    del O
    t8, st8, used8 = oracle_step_time(SAMPLE_N, ncores)
    t4, st4, _ = oracle_step_time(4, 1)
    scale = (n_full / SAMPLE_N) ** 3
    out.update({"step_8cube_s_all": t8, "step_8cube_gmres": st8["n_gmres"], "step_4cube_s_1": t4,
                "step_4cube_gmres": st4["n_gmres"], "value": t8 * scale, "unit": "s/step", "cores": used8,
                "kind": "oracle", "estimated": True,
                "residual_gdofs_1": W.q0.size / out["residual_s_1"] / 1e9,
                "residual_gdofs_all": W.q0.size / out["residual_s_all"] / 1e9,
                "sample": (f"R and Jv on the full {n_full}^3 workload (one thread, {out['threads_all']} threads); the "
                           f"ROS34PW2 step on an {SAMPLE_N}^3 slice at the same CFL on {used8} threads "
                           f"({t8:.1f} s, {st8['n_gmres']} FGMRES iterations) scaled by the element count "
                           f"x{int(scale)} = value (estimated), and on a 4^3 slice on one thread "
                           f"({t4:.1f} s, {st4['n_gmres']} FGMRES iterations)")})
    return out


def oracle_baseline_in_child():
    """oracle_baseline() in a child process (the GPU arm's process never loads the oracle)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print('ORACLE ' + json.dumps(bench.oracle_baseline()))") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    for line in r.stdout.splitlines():
        if line.startswith("ORACLE "):
            return json.loads(line[len("ORACLE "):])
    return {"error": (r.stderr or r.stdout)[-1000:]}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    scale = (32 // SAMPLE_N) ** 3
    times, its, used = [], [], 1
    for i in range(args.warmup + args.steps):
        t, st, used = oracle_step_time(SAMPLE_N, None)
        if i >= args.warmup:
            times.append(t * scale)
            its.append(st["n_gmres"])
    value = statistics.mean(times)
    sample = (f"oracle ROS34PW2 step, pMG p{{3-2}} n{{2-2}}, FGMRES(30) to 1e-6, on an {SAMPLE_N}^3-hex slice "
              f"of the 32^3 workload at the same CFL ({statistics.mean(its):.0f} FGMRES iterations), "
              f"{used} host threads, scaled by the element count x{scale} (estimated)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/step", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "tgv3d 32^3 hex p=3 (Ma 0.1, Re 1600), ROS34PW2 step, pMG p{3-2} n{2-2}, "
                                   "FGMRES(30) tol 1e-6", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "s/step", "cores": used, "kind": "oracle", "sample": sample,
                             "estimated": True, "measured_s_per_sample_step": value / scale},
            "e2e": {"value": value, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- GPU arm
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def esdirk_guess_compare(api, w, T, np, torch, warm=15, timed=6):
    """ESDIRK3 steps at the 1e-8 Newton tolerance on the unsteady low-Mach cylinder
    (O-mesh 96 x 192, p = 3, Ma 0.05, Re 150, CFL 50, pMG p{3-2} n{2-2}, dtau = dt as in the
    paper): the plain FP64 method (guess q^n, the paper's) against the mixed preconditioner
    with the initial-guess candidates.  Each variant runs `warm` steps from the same state
    (the history and the network's training data) and then `timed` steps, timed with CUDA
    events.  fp64_ej_qn is the paper's JFNK-EJ baseline (element-Jacobi preconditioner);
    mixed_mbnk_extrap smooths the coarsest level (p = 2) with the matrix-based Newton-Krylov
    smoother (GMRES of at most 5 iterations to 1e-1 on the assembled operator) instead of
    element-Jacobi blocks."""
    import math
    wl = w.cylinder_unsteady()
    A, b = T.esdirk3()
    out = {"workload": "cylinder_unsteady 96x192 O-mesh quads p=3 (Ma 0.05, Re 150), ESDIRK3, dt = 50x explicit, "
                       "Newton tol 1e-8 (RMS of a_ii dt F), pMG p{3-2} n{2-2}, FGMRES(30) tol 1e-2",
           "warm_steps": warm, "timed_steps": timed, "variants": {}}
    ref = None
    for name, prec, guess, train in (("fp64_qn", "fp64", "qn", 0), ("mixed_qn", "mixed", "qn", 0),
                                     ("mixed_extrap", "mixed", "extrap", 0), ("mixed_mbnk_extrap", "mixed", "extrap", 0),
                                     ("mixed_mlp", "mixed", "mlp", 10), ("fp64_ej_qn", "fp64", "qn", 0)):
        G = api.fr_create(wl.mesh, wl.phys, wl.levels)
        if guess == "mlp":
            K0, O = api.fr_mlp_dims(G)
            rng = np.random.default_rng(0)
            H = 128
            P = [rng.standard_normal((H, K0)) / math.sqrt(K0), np.zeros(H), rng.standard_normal((H, H)) / math.sqrt(H),
                 np.zeros(H), rng.standard_normal((O, H)) / math.sqrt(H) * 0.1, np.zeros(O)]
            net = api.MLP(K0, H, O, np.concatenate([x.reshape(-1) for x in P]).astype(np.float32))
            api.fr_set_mlp(G, net)
        # "_ej": the paper's JFNK-EJ baseline, the element-Jacobi preconditioner (one fine
        # pseudo step with 1/dtau* = 0: the pMG cycle's special case)
        ej = name.endswith("_ej_qn")
        o = api.solve_opts(kdim=30, maxit_gmres=300 if not ej else 3000, max_ptc=40,
                           nsmooth=(2, 2) if not ej else (1,), tol_gmres=1e-2, tol_newton=1e-8,
                           dtau=wl.dt, inv_dtau_star=1.0 / wl.dt if not ej else 0.0, precision=prec, guess=guess,
                           train_iters=train, train_batch=4096, lr=1e-3,
                           coarse="mbnk" if "_mbnk" in name else "ej")
        q = torch.from_numpy(np.ascontiguousarray(wl.q0)).cuda()
        try:
            for _ in range(warm):
                api.esdirk_step(G, A, b, wl.dt, q, o)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sts = []
            e0.record()
            for _ in range(timed):
                sts.append(api.esdirk_step(G, A, b, wl.dt, q, o))
            e1.record()
            torch.cuda.synchronize()
        except RuntimeError as ex:              # a library error in one variant: record it, keep the rest
            out["variants"][name] = {"error": str(ex)[:300]}
            continue
        if ref is None:
            ref = q.clone()
        dq = float(((q - ref).abs().max() / ref.abs().max()).item())
        out["variants"][name] = {
            "s_per_step": e0.elapsed_time(e1) / 1e3 / timed,
            "newton_per_step": float(np.mean([s_["n_ptc"] for s_ in sts])),
            "gmres_per_step": float(np.mean([s_["n_gmres"] for s_ in sts])),
            "picks_qn_extrap_mlp": [int(sum(s_["guess_pick"][k] for s_ in sts)) for k in range(3)],
            "state_vs_fp64_qn_maxrel": dq,
            "state_abs_sum": float(q.abs().sum().item()),
        }
    v = out["variants"]
    out["speedup_mixed_extrap_vs_fp64_qn"] = v["fp64_qn"]["s_per_step"] / v["mixed_extrap"]["s_per_step"]
    out["speedup_mixed_mlp_vs_fp64_qn"] = v["fp64_qn"]["s_per_step"] / v["mixed_mlp"]["s_per_step"]
    out["speedup_fp64_pmg_vs_fp64_ej"] = v["fp64_ej_qn"]["s_per_step"] / v["fp64_qn"]["s_per_step"]
    if "s_per_step" in v["mixed_mbnk_extrap"]:
        out["speedup_mbnk_vs_ej_coarse_smoother"] = v["mixed_extrap"]["s_per_step"] / v["mixed_mbnk_extrap"]["s_per_step"]
    return out


def batched_step(api, w, T, np, torch, N):
    """One ESDIRK3 step of 256 independent periodic vortex problems (n x n quads, n in
    4..48, p in 1..4, seeded), grouped by p-levels on merged meshes, Arnoldi steps under
    CUDA graphs, autotuned launch shapes; one warm step then one timed step per precision."""
    probs, states, phys, dt = w.vortex_batch()
    A, b = T.esdirk3()
    out = {"workload": f"{len(probs)} periodic vortex problems, n x n quads n~U{{4..48}}, p~U{{1..4}}, "
                       f"levels p{{p-(p-1)}} (p=1: one level), ESDIRK3, common dt {dt:.4g}, Newton tol 1e-8",
           "elements": int(sum(m["E"] for m, _ in probs)),
           "dofs": int(sum(4 * (lv[0] + 1) ** 2 * m["E"] for m, lv in probs))}
    for prec in ("fp64", "mixed"):
        Bt = api.Batch(probs, phys)
        go = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-8,
                            dtau=dt, inv_dtau_star=1.0 / dt, precision=prec)
        qs = [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in states]
        Bt.esdirk_step(A, b, dt, [x.clone() for x in qs], go)
        Bt.autotune(fp64=True, fp32=(prec == "mixed"), retune=False, reps=3)
        Bt.esdirk_step(A, b, dt, [x.clone() for x in qs], go)     # graphs captured with the tuned shapes
        torch.cuda.synchronize()
        n0 = N.load().fr_kernel_launches()
        # the batch runs on its own stream, ordered after and before the current stream,
        # so events on the current stream bracket its work
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = Bt.esdirk_step(A, b, dt, qs, go)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[prec] = {"s_per_step": t, "problems_per_s": len(probs) / t,
                     "converged": int(sum(s_["converged"] for s_ in st)),
                     "gmres_total": int(sum(s_["n_gmres"] for s_ in st)),
                     "kernel_launches": int(N.load().fr_kernel_launches() - n0)}
    return out


def steady_lowmach(api, w, np, torch, max_it=150):
    """The steady low-Mach cylinder (O-mesh 64 x 128, stretched to aspect ratio 1e3 at the
    wall, p{4-2-1} n{2-2-5}, Ma 1e-3, Re 40, Rusanov, impulsive start): pseudo-transient
    continuation with SER from dtau = 0.1 h_min / (|u| + c), FGMRES(30) to 1e-3 in at most 60
    iterations per pseudo step, the FD step of Jv 1e-2 (the state is ~1/(gamma Ma^2) ~ 7e5:
    a step of 1e-6 times a unit-norm vector is below its FP64 resolution), with the FP64
    preconditioner (its X scaled as the FP32 cycle's is) and with the mixed one (FP32
    cycle, blocks, LU; no switch to FP64 when it stalls); per precision the relative
    residual reached after max_it pseudo steps, the pseudo steps and seconds to reach drops
    of 1e-2 / 1e-3 / 1e-4, and the iteration counts (CUDA events around the whole march)."""
    W = w.cylinder_steady()
    mach = 1e-3
    dtau0 = 0.1 * W.mesh["h_min"] / (1.0 + 1.0 / mach)
    out = {"workload": "cylinder_steady 64x128 O-mesh p{4-2-1} n{2-2-5} (Ma 1e-3, Re 40, Rusanov), PTC + SER, "
                       f"FGMRES(30) tol 1e-3 maxit 60, FD step 1e-2, {max_it} pseudo steps", "precisions": {}}
    for prec in ("fp64", "mixed"):
        G = api.fr_create(W.mesh, W.phys, W.levels)
        api.fr_set_cycle_scaling(G, True)
        api.fr_set_precision_fallback(G, False)
        o = api.solve_opts(kdim=30, maxit_gmres=60, nsmooth=(2, 2, 5), tol_gmres=1e-3, inv_dtau_star=-1.0,
                           precision=prec, eps=1e-2)
        q = torch.from_numpy(np.ascontiguousarray(W.q0)).cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        st = api.ptc_steady(G, q, dtau0, 1e6, 1e-10, max_it, o)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        h = np.asarray(st["hist"])
        rel = h / h[0]
        reach = {}
        for tol in (1e-2, 1e-3, 1e-4):
            k = int(np.argmax(rel <= tol)) if np.any(rel <= tol) else None
            reach[f"{tol:g}"] = {"pseudo_steps": k, "s": (wall * k / max(1, len(h) - 1)) if k else None}
        out["precisions"][prec] = {"relative_residual": float(rel[-1]), "pseudo_steps": int(st["n_ptc"]),
                                   "gmres_total": int(st["n_gmres"]), "s": e0.elapsed_time(e1) / 1e3,
                                   "converged_1e-10": bool(st["converged"]), "reached": reach}
    return out


def padapt_indicator(api, w, np, torch):
    """The p-adaptation indicator and marking (Sec. 3.3) on the 32^3 Taylor-Green state
    (p = 3, x-momentum): the marking the paper's rule (nu_max 0.2, nu_min 1e-3, p in
    [1, 4]) makes, and the indicator's time per launch (CUDA events, 20 launches)."""
    W = w.tgv3d(n=32)
    G = api.fr_create(W.mesh, W.phys, W.levels)
    q = torch.from_numpy(np.ascontiguousarray(W.q0)).cuda()
    eta = api.fr_spectral_decay(G, 0, q, var=1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        api.fr_spectral_decay(G, 0, q, var=1, eta=eta)
    e1.record()
    torch.cuda.synchronize()
    p_in = torch.full((G.E,), 3, dtype=torch.int32, device="cuda")
    p_out = api.fr_padapt_mark(G, eta, p_in, 1, 4).cpu().numpy()
    e = eta.cpu().numpy()
    return {"workload": "tgv3d 32^3 p=3 initial state, indicator of rho u", "ms_per_launch": e0.elapsed_time(e1) / 20,
            "eta_max": float(e.max()), "eta_median": float(np.median(e)),
            "raised": int((p_out > 3).sum()), "kept": int((p_out == 3).sum()), "lowered": int((p_out < 3).sum())}


def run_extras_in_child():
    """The ESDIRK guess comparison and the batched step, in a child process of their own
    (a clean library state, and a failure there cannot take the main measurement down)."""
    code = ("import json, sys; sys.path.insert(0, %r); import numpy as np, torch, bench; "
            "from paper_2202_09733_gb300 import api, workloads as w, tableaux as T, _native as N; "
            "torch.cuda.set_device(0); "
            "out = {'esdirk_cylinder': bench.esdirk_guess_compare(api, w, T, np, torch), "
            "'batched_vortex': bench.batched_step(api, w, T, np, torch, N), "
            "'steady_lowmach_cylinder': bench.steady_lowmach(api, w, np, torch), "
            "'padapt_indicator': bench.padapt_indicator(api, w, np, torch)}; "
            "print('EXTRAS ' + json.dumps(out))") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    for line in r.stdout.splitlines():
        if line.startswith("EXTRAS "):
            return json.loads(line[len("EXTRAS "):])
    return {"extras_error": (r.stderr or r.stdout)[-2000:]}


def gpu_arm(args):
    import numpy as np
    import torch
    from paper_2202_09733_gb300 import api, workloads as w, tableaux as T, perfmodel as PM
    from paper_2202_09733_gb300 import build as B, _native as N

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    lib = N.load()

    W = w.tgv3d(n=args.n)
    part = None
    if ws > 1:
        # the mesh split over the ranks (one GPU each): ghosts exchanged and inner products
        # summed over NCCL by the library's communicator
        from paper_2202_09733_gb300.distributed import PartitionedContext, TorchDistTransport
        part = PartitionedContext(W.mesh, W.phys, W.levels, rank, ws, TorchDistTransport())
        ctx = part.ctx
        q0 = part.local_state(W.q0)
    else:
        ctx = api.fr_create(W.mesh, W.phys, W.levels)
        q0 = torch.from_numpy(W.q0).cuda()
    api.fr_set_lu_storage(ctx, args.lu_storage)
    q = q0.clone()
    g, a, c, m = T.ros34pw2()
    opts = api.solve_opts(kdim=30, maxit_gmres=300, nsmooth=(2, 2), tol_gmres=1e-6, inv_dtau_star=1.0 / W.dt,
                          precision=args.precision)
    opts64 = api.solve_opts(kdim=30, maxit_gmres=300, nsmooth=(2, 2), tol_gmres=1e-6, inv_dtau_star=1.0 / W.dt,
                            precision="fp64")
    stream = torch.cuda.current_stream()

    def step(o=opts):
        q.copy_(q0)
        return api.row_step(ctx, g, a, c, m, W.dt, q, o)

    tune = None
    if not args.no_autotune and part is None:     # every rank would have to tune in lockstep
        # launch shapes of this GPU for the residual kernels; G of the block solves after
        # one step has factored the blocks (no result bit depends on either)
        step()
        tune = api.fr_autotune(ctx, fp64=True, fp32=True, retune=True, reps=3)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()

    # ---- timed steps (device-resident inputs)
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    n0 = lib.fr_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = lib.fr_kernel_launches() - n0
    clocks = clk.stop()
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    t_step = max_over_ranks(t_step, ws, "cuda")

    q_mixed = q.clone()

    # ---- the same mixed step with FP32 factors for the smoother's solves (the other storage)
    t_other = None
    if args.precision != "fp64" and part is None:
        other = "fp32" if args.lu_storage == "half" else "half"
        api.fr_set_lu_storage(ctx, other)
        step()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        st_other = step()
        g1.record(stream)
        torch.cuda.synchronize()
        t_other = {"lu_storage": other, "s_per_step": g0.elapsed_time(g1) / 1e3,
                   "gmres_iterations": st_other["n_gmres"]}
        api.fr_set_lu_storage(ctx, args.lu_storage)

    # ---- the plain FP64 JFNK-pMG step on the same input, for comparison
    t_fp64, st64, dq = None, None, None
    if args.precision != "fp64" and not args.no_fp64_compare:
        st64 = step(opts64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        st64 = step(opts64)
        f1.record(stream)
        torch.cuda.synchronize()
        t_fp64 = max_over_ranks(f0.elapsed_time(f1) / 1e3, ws, "cuda")
        dq = float(((q_mixed - q).abs().max() / q.abs().max()).item())

    # ---- residual throughput and roofline (same stream, CUDA events)
    R = torch.empty_like(q0)
    for _ in range(3):
        api.fr_residual(ctx, 0, q0, R)
    nrep = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nrep):
        api.fr_residual(ctx, 0, q0, R)
    e1.record(stream)
    torch.cuda.synchronize()
    t_R = e0.elapsed_time(e1) / 1e3 / nrep
    t_R = max_over_ranks(t_R, ws, "cuda")
    E = W.mesh["E"]
    ndof = int(W.q0.size)
    flops = PM.residual_flops(3, 3) * E
    gdofs = ndof / t_R / 1e9

    # ---- end to end through host buffers (pinned), H2D + step + D2H inside the region
    q_host = q0.cpu().pin_memory()
    out_host = torch.empty_like(q_host).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q.copy_(q_host, non_blocking=True)
        api.row_step(ctx, g, a, c, m, W.dt, q, opts)
        out_host.copy_(q, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps, ws, "cuda")
    barrier()

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras_in_child()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_baseline_in_child()

    roof = roof32 = solve_roofline(tune, E, 5 * 64)
    if rank == 0 and args.lu_storage == "half" and args.precision != "fp64" and part is None:
        cshift = 1.0 / W.dt + 1.0 / (0.4358665215084590 * W.dt)
        roof = half_solve_roofline(api, torch, ctx, q0, cshift, E, 5 * 64)

    if rank == 0:
        ng = [s_["n_gmres"] for s_ in stats]
        line = {
            "metric": METRIC, "value": t_step, "unit": "s/step", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": f"tgv3d {args.n}^3 hex p=3 (Ma 0.1, Re 1600), ROS34PW2 step dt=20x explicit, "
                                   "pMG p{3-2} n{2-2} (blocks + LU at q^n inside the step), FGMRES(30) tol 1e-6",
                       "precision": ("FP64 throughout" if args.precision == "fp64" else
                                     "mixed: FP64 residual, Jv, Gram-Schmidt, update; FP32 pMG cycle, blocks, LU "
                                     "(tensor-core trailing updates)" +
                                     ("; the smoother's block solves read the factors stored as binary16 with FP32 "
                                      "column scales (TF32's 10-bit mantissa), FP32 arithmetic"
                                      if args.lu_storage == "half" else "; FP32 factors")),
                       "ndof": ndof, "elements": E, "l2": "inputs larger than L2 (state 84 MB, FP32 blocks 13 GB): no flush",
                       "parallelism": (f"element partition over {ws} GPUs (recursive bisection, one ghost "
                                       "layer; ghost exchange and inner-product sums over NCCL)") if ws > 1
                                      else "single GPU"},
            "fp64_step_s": t_fp64,
            "speedup_vs_fp64_step": (t_fp64 / t_step) if t_fp64 else None,
            "fp64_step_gmres_iterations": st64["n_gmres"] if st64 else None,
            "mixed_vs_fp64_state_maxrel": dq,
            "residual_gdofs": gdofs,
            "residual_ms": t_R * 1e3,
            "gmres_iterations_per_step": statistics.mean(ng),
            "roofline": roof,
            "roofline_fp32_solve": roof32 if args.lu_storage == "half" else None,
            "other_lu_storage_step": t_other,
            "roofline_residual": {"kernel": "fr_residual (FP64 FR residual, 7 kernels per launch)", "bound": "alu",
                         "achieved": flops / t_R / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12, "unit": "TFLOP/s",
                         "frac": (flops / t_R) / FP64_PEAK_NOMINAL,
                         "traffic": profile_figure("residual_tgv3d32_fp64_dram", "dram_bytes_per_launch"),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the kernels of one "
                                           "residual on this workload (committed ncu summary)",
                         "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (MEASURED_PEAKS.json has no FP64 entry); "
                                        "independent DFMA chains measured %s TFLOP/s on this part"
                                        % profile_figure("fp_rates_gb300", "dfma_tflops")},
            "e2e": {"value": t_e2e, "unit": "s/step", "h2d_bytes_per_step": q_host.numel() * 8,
                    "d2h_bytes_per_step": q_host.numel() * 8},
            "cpu_baseline": cpu,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "autotune": tune,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
