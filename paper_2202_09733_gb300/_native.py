"""ctypes declarations of the frpmg C ABI (include/frpmg.h).

Loading fails loudly when the in-tree libfrpmg.so is missing: there is no fallback."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfrpmg.so")

PD, PI, PF = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_float)
VP = C.c_void_p

FR_OK = 0
ERRORS = {-1: "FR_ERR_INVALID_ARG", -2: "FR_ERR_CUDA", -3: "FR_ERR_OOM", -4: "FR_ERR_NOT_CONVERGED",
          -5: "FR_ERR_NONFINITE", -6: "FR_ERR_BREAKDOWN", -7: "FR_ERR_UNIMPLEMENTED", -8: "FR_ERR_NOT_READY"}

# every symbol the header declares
EXPORTS = ["fr_create", "fr_destroy", "fr_last_error", "fr_kernel_launches", "fr_level_info", "fr_num_colors", "fr_residual",
           "fr_residual_noalloc", "fr_jvp",
           "fr_elem_blocks", "fr_elem_blocks_f32", "fr_set_block_method", "fr_set_comm", "fr_nbr_blocks", "fr_neighbour_table", "fr_mbnk_last", "fr_mbnk_operator", "fr_block_factor", "fr_block_solve", "fr_block_factor_f32", "fr_block_solve_f32", "fr_set_lu_method", "fr_block_to_half", "fr_block_solve_half", "fr_set_lu_storage", "fr_set_cycle_scaling", "fr_set_precision_fallback", "fr_spectral_decay", "fr_padapt_mark", "fr_nested_hierarchy", "fr_restrict", "fr_prolong", "pmg_setup",
           "pmg_precondition", "gmres_solve", "esdirk_step", "row_step", "ptc_steady",
           "mlp_create", "mlp_destroy", "mlp_get_params", "mlp_forward", "mlp_train_step", "fr_mlp_dims",
           "fr_set_mlp", "fr_reset_history", "fr_guess_features", "fr_batch_create", "fr_batch_destroy",
           "fr_batch_info", "fr_batch_set_graphs", "fr_batch_residual", "fr_batch_esdirk_step", "fr_autotune",
           "fr_get_tiles", "fr_set_tiles", "fr_autotune_save", "fr_autotune_load", "fr_batch_autotune", "fr_kernel_timeouts",
           "fr_selftest_wait_timeout", "pmg_solve_steady", "fr_checkpoint_size", "fr_checkpoint_save",
           "fr_checkpoint_load"]


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelem", C.c_int), ("qg", C.c_int), ("gnodes", PD), ("nfaces", C.c_int),
                ("faces", PI), ("nlevels", C.c_int), ("plevels", PI)]


class Physics(C.Structure):
    _fields_ = [("gamma", C.c_double), ("prandtl", C.c_double), ("mu", C.c_double), ("eta", C.c_double),
                ("qinf", C.c_double * 5), ("flux", C.c_int), ("ws_umin", C.c_double)]


class PmgOpts(C.Structure):
    _fields_ = [("nlevels", C.c_int), ("nsmooth", C.c_int * 4), ("c", C.c_double), ("inv_dtau_star", C.c_double),
                ("precision", C.c_int), ("coarse_smoother", C.c_int), ("mbnk_maxit", C.c_int),
                ("mbnk_tol", C.c_double)]


HaloFn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_longlong, C.c_void_p)
AllreduceFn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int)


class Comm(C.Structure):
    _fields_ = [("n_owned", C.c_int), ("n_owned_total", C.c_longlong), ("nsend", C.c_int), ("send_idx", PI), ("send_buf", VP), ("recv_buf", VP),
                ("halo", HaloFn), ("allreduce", AllreduceFn), ("user", VP)]


class GmresOpts(C.Structure):
    _fields_ = [("kdim", C.c_int), ("maxit", C.c_int), ("use_pmg", C.c_int), ("tol", C.c_double),
                ("eps", C.c_double), ("shift", C.c_double)]


class GmresStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("relres", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("kdim", C.c_int), ("maxit_gmres", C.c_int), ("max_ptc", C.c_int), ("nlevels", C.c_int),
                ("nsmooth", C.c_int * 4), ("use_pmg", C.c_int), ("tol_gmres", C.c_double),
                ("tol_newton", C.c_double), ("eps", C.c_double), ("dtau", C.c_double),
                ("inv_dtau_star", C.c_double), ("precision", C.c_int), ("guess", C.c_int),
                ("train_iters", C.c_int), ("train_batch", C.c_int), ("lr", C.c_double),
                ("coarse_smoother", C.c_int), ("mbnk_maxit", C.c_int), ("mbnk_tol", C.c_double),
                ("nonlinear", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("n_ptc", C.c_int), ("n_gmres", C.c_int), ("converged", C.c_int), ("final_res", C.c_double),
                ("guess_rms", C.c_double * 3), ("guess_pick", C.c_int * 3), ("guess_beta", C.c_double),
                ("train_loss", C.c_double), ("prec_switch_it", C.c_int)]


class EsdirkTableau(C.Structure):
    _fields_ = [("stages", C.c_int), ("A", C.c_double * 36), ("b", C.c_double * 6)]


class RowTableau(C.Structure):
    _fields_ = [("stages", C.c_int), ("gamma", C.c_double), ("a", C.c_double * 36), ("c", C.c_double * 36),
                ("m", C.c_double * 6)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfrpmg.so and declare its signatures (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"frpmg CUDA library not built ({path} missing): run __graft_entry__.build()")
    L = C.CDLL(path)
    sig = {
        "fr_create": ([C.POINTER(VP), C.POINTER(MeshDesc), C.POINTER(Physics)], C.c_int),
        "fr_destroy": ([VP], C.c_int),
        "fr_last_error": ([], C.c_char_p),
        "fr_kernel_launches": ([], C.c_ulonglong),
        "fr_level_info": ([VP, C.c_int, PI, PI, C.POINTER(C.c_longlong)], C.c_int),
        "fr_num_colors": ([VP, PI], C.c_int),
        "fr_residual": ([VP, C.c_int, VP, VP, VP], C.c_int),
        "fr_residual_noalloc": ([VP, C.c_int, VP, VP, VP], C.c_int),
        "fr_jvp": ([VP, VP, VP, VP, C.c_double, C.c_double, VP, VP], C.c_int),
        "fr_elem_blocks": ([VP, C.c_int, VP, C.c_double, VP, VP], C.c_int),
        "fr_elem_blocks_f32": ([VP, C.c_int, VP, C.c_double, VP, C.c_int, VP], C.c_int),
        "fr_set_block_method": ([VP, C.c_int], C.c_int),
        "fr_set_comm": ([VP, C.POINTER(Comm)], C.c_int),
        "fr_nbr_blocks": ([VP, C.c_int, VP, C.c_double, VP, VP, VP], C.c_int),
        "fr_neighbour_table": ([VP, PI], C.c_int),
        "fr_mbnk_last": ([VP, PI, PD], C.c_int),
        "fr_mbnk_operator": ([VP, VP, VP, VP], C.c_int),
        "fr_block_factor": ([VP, C.c_int, VP, VP, VP], C.c_int),
        "fr_block_solve": ([VP, C.c_int, VP, VP, VP, VP], C.c_int),
        "fr_block_factor_f32": ([VP, C.c_int, VP, VP, C.c_int, VP], C.c_int),
        "fr_block_solve_f32": ([VP, C.c_int, VP, VP, VP, VP], C.c_int),
        "fr_set_lu_method": ([VP, C.c_int], C.c_int),
        "fr_block_to_half": ([VP, C.c_int, VP, VP, VP, VP], C.c_int),
        "fr_block_solve_half": ([VP, C.c_int, VP, VP, VP, VP, VP], C.c_int),
        "fr_set_lu_storage": ([VP, C.c_int], C.c_int),
        "fr_set_cycle_scaling": ([VP, C.c_int], C.c_int),
        "fr_spectral_decay": ([VP, C.c_int, VP, C.c_int, VP, VP], C.c_int),
        "fr_padapt_mark": ([VP, VP, VP, C.c_int, C.c_int, C.c_double, C.c_double, VP, VP], C.c_int),
        "fr_nested_hierarchy": ([C.c_int, C.c_int, C.c_int, PI], C.c_int),
        "fr_set_precision_fallback": ([VP, C.c_int], C.c_int),
        "fr_restrict": ([VP, C.c_int, VP, VP, VP], C.c_int),
        "fr_prolong": ([VP, C.c_int, VP, VP, VP], C.c_int),
        "pmg_setup": ([VP, VP, C.POINTER(PmgOpts), VP], C.c_int),
        "pmg_precondition": ([VP, VP, VP, VP, VP, VP], C.c_int),
        "gmres_solve": ([VP, VP, VP, VP, VP, C.POINTER(GmresOpts), C.POINTER(GmresStats), VP], C.c_int),
        "esdirk_step": ([VP, C.POINTER(EsdirkTableau), C.c_double, VP, C.POINTER(SolveOpts),
                         C.POINTER(StepStats), VP], C.c_int),
        "row_step": ([VP, C.POINTER(RowTableau), C.c_double, VP, C.POINTER(SolveOpts), C.POINTER(StepStats), VP],
                     C.c_int),
        "ptc_steady": ([VP, VP, C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(SolveOpts),
                        C.POINTER(StepStats), PD, VP], C.c_int),
        "mlp_create": ([C.POINTER(VP), C.c_int, C.c_int, C.c_int, PF], C.c_int),
        "mlp_destroy": ([VP], C.c_int),
        "mlp_get_params": ([VP, PF], C.c_int),
        "mlp_forward": ([VP, C.c_int, VP, VP, VP], C.c_int),
        "mlp_train_step": ([VP, C.c_int, VP, VP, C.c_float, PF, VP, VP], C.c_int),
        "fr_mlp_dims": ([VP, PI, PI], C.c_int),
        "fr_set_mlp": ([VP, VP], C.c_int),
        "fr_reset_history": ([VP], C.c_int),
        "fr_guess_features": ([VP, VP, VP, VP, VP, C.c_double, C.c_double, VP, PD, VP], C.c_int),
        "fr_batch_create": ([C.POINTER(VP), C.c_int, C.POINTER(MeshDesc), C.POINTER(Physics)], C.c_int),
        "fr_batch_destroy": ([VP], C.c_int),
        "fr_batch_info": ([VP, PI, PI, PI], C.c_int),
        "fr_batch_set_graphs": ([VP, C.c_int], C.c_int),
        "fr_batch_residual": ([VP, C.POINTER(VP), C.POINTER(VP), VP], C.c_int),
        "fr_batch_esdirk_step": ([VP, C.POINTER(EsdirkTableau), C.c_double, C.POINTER(VP), C.POINTER(SolveOpts),
                                  C.POINTER(StepStats), VP], C.c_int),
        "fr_autotune": ([VP, C.c_int, C.c_int, C.c_char_p, C.c_int], C.c_int),
        "fr_get_tiles": ([VP, C.c_int, C.c_int, PI], C.c_int),
        "fr_set_tiles": ([VP, C.c_int, C.c_int, PI], C.c_int),
        "fr_autotune_save": ([C.c_char_p], C.c_int),
        "fr_autotune_load": ([C.c_char_p], C.c_int),
        "fr_batch_autotune": ([VP, C.c_int, C.c_int, C.c_char_p, C.c_int], C.c_int),
        "fr_kernel_timeouts": ([C.c_int], C.c_int),
        "fr_selftest_wait_timeout": ([], C.c_int),
        "pmg_solve_steady": ([VP, VP, C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(SolveOpts),
                              C.POINTER(StepStats), PD, VP], C.c_int),
        "fr_checkpoint_size": ([VP, VP, C.POINTER(C.c_longlong)], C.c_int),
        "fr_checkpoint_save": ([VP, VP, VP, C.c_longlong], C.c_int),
        "fr_checkpoint_load": ([VP, VP, VP, C.c_longlong], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes, f.restype = args, res
    _lib = L
    return L


class FrError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().fr_last_error().decode(errors="replace")
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str, allow=()):
    if code != FR_OK and code not in allow:
        raise FrError(code, where)
    return code
