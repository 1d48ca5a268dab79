"""Half-width storage of the FP32 block factors for the smoother's solves
(fr_block_to_half, fr_block_solve_half, fr_set_lu_storage "half").

L (|l| <= 1 under partial pivoting) is stored as binary16 and every column of U divided
by its largest magnitude; 1/u_kk and the column scales stay FP32.  Checks:
  - on factors whose entries binary16 holds exactly (L on a 1/2048 grid, U on a 1/64 grid
    of a power-of-two column scale that is the column's largest entry), the half-width
    solve equals the FP32-factor solve bit
    for bit: the scaled update u'' (g x) is then the same product u x, so this pins the
    kernel's indexing, permutation and column scaling against the FP32 kernel;
  - on the element blocks of the 3-D p = 3 / p = 2 levels, the solve is within the
    first-order perturbation bound of an FP64 solve: relative error <= 4 * 2^-11 * kappa
    per block (binary16 rounding perturbs each factor entry by at most 2^-11 of its
    column scale; kappa = the block's infinity-norm condition number);
  - an ESDIRK3 step with the mixed preconditioner reading half-width factors converges
    to the FP64 step's state within the Newton tolerance bar the mixed step meets
    (1e-10 relative at tol 1e-12): the factors only change the preconditioner."""
import math

import numpy as np
import pytest
import torch

from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B
from paper_2202_09733_gb300 import tableaux as GT

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _ctx():
    mesh = w.box3d(4, 2 * math.pi)
    ph = w.Physics(mu=0.02, qinf=w.freestream(3, 0.3))
    return api.fr_create(mesh, ph, [3, 2]), mesh


def _exact_factors(E, nd, seed):
    """In-place factor storage F[e, j, r] (column-major) with entries binary16 holds
    exactly: L entries on a 1/2048 grid in [-1/512, 1/512], U entries on a 1/64 grid of
    their column's scale 2^m (m in -12..-8), each U column's largest entry exactly +-2^m,
    1/u_kk in [0.5, 1.5) on the diagonal (it stays FP32).  Small off-diagonal entries keep
    the substitutions' growth bounded over nd = 320 rows."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    r = torch.arange(nd, device="cuda")
    lower = (r[:, None] > r[None, :])[None]                            # [1, row, column]
    upper = (r[:, None] < r[None, :])[None]
    Lv = torch.randint(-4, 5, (E, nd, nd), generator=g, device="cuda").float() / 2048.0
    scale = 2.0 ** torch.randint(-12, -7, (E, 1, nd), generator=g, device="cuda").float()
    Uv = torch.randint(-64, 65, (E, nd, nd), generator=g, device="cuda").float() / 64.0 * scale
    Uv[:, 0, :] = scale[:, 0, :]            # the largest |entry| of every U column is its scale
    A = torch.where(lower, Lv, torch.where(upper, Uv, torch.zeros_like(Uv)))   # [e, r, j]
    diag = 0.5 + torch.rand((E, nd), generator=g, device="cuda")
    A[:, r, r] = 1.0 / diag
    perm = torch.stack([torch.randperm(nd, device="cuda") for _ in range(E)]).int()
    return A.transpose(1, 2).contiguous(), perm


def test_exactly_representable_factors_solve_bit_for_bit():
    G, mesh = _ctx()
    for level in (0, 1):
        nd = G.nd(level)
        F, perm = _exact_factors(G.E, nd, 5 + level)
        H, dg = api.fr_block_to_half(G, level, F)
        assert torch.equal(H.float().transpose(1, 2)[:, torch.arange(nd), torch.arange(nd)],
                           torch.zeros((G.E, nd), device="cuda"))
        b = torch.randn((nd, G.E), device="cuda", dtype=torch.float32)
        x32 = api.fr_block_solve_f32(G, level, F, perm, b.clone())
        x16 = api.fr_block_solve_half(G, level, H, dg, perm, b.clone())
        torch.cuda.synchronize()
        assert torch.isfinite(x32).all() and x32.abs().max().item() > 0
        assert torch.equal(x16, x32), (level, (x16 - x32).abs().max().item())


def test_element_block_solves_within_the_perturbation_bound():
    G, mesh = _ctx()
    X = w.solution_point_coords(mesh, 3)
    vel = [0.3 + 0.02 * np.sin(X[0]), 0.02 * np.cos(X[1]), 0.01 * np.sin(X[2])]
    q = w.prim_to_cons(1.0 + 0.01 * np.sin(X[0]), vel, (1 / (w.GAMMA * 0.3 ** 2)) * (1 + 0.01 * np.cos(X[1])))
    ql = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    for level in (0, 1):
        if level:
            ql = api.fr_restrict(G, 0, ql)
        M = api.fr_elem_blocks_f32(G, level, ql.float().contiguous(), 3.0)
        F = M.clone()
        perm = api.fr_block_factor_f32(G, level, F)
        H, dg = api.fr_block_to_half(G, level, F)
        nd = M.shape[1]
        b = torch.randn((nd, G.E), device="cuda", dtype=torch.float32)
        x16 = api.fr_block_solve_half(G, level, H, dg, perm, b.clone()).double()
        A = M.double().transpose(1, 2)
        ref = torch.linalg.solve(A, b.double().T.unsqueeze(-1)).squeeze(-1).T
        err = (x16 - ref).abs().amax(dim=0) / ref.abs().amax(dim=0)
        kappa = torch.linalg.matrix_norm(A, ord=float("inf")) * torch.linalg.matrix_norm(torch.linalg.inv(A),
                                                                                         ord=float("inf"))
        assert (err <= 4 * 2.0 ** -11 * kappa).all(), (level, err.max().item(), kappa.min().item())


def test_esdirk_step_with_half_width_factors_converges_to_the_fp64_state():
    W = w.tgv3d(n=3)
    G64 = api.fr_create(W.mesh, W.phys, W.levels)
    Gh = api.fr_create(W.mesh, W.phys, W.levels)
    api.fr_set_lu_storage(Gh, "half")
    A, b = GT.esdirk3()
    dt = W.dt
    q64 = torch.from_numpy(np.ascontiguousarray(W.q0)).cuda()
    qh = q64.clone()
    o64 = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12,
                         dtau=dt, inv_dtau_star=1.0 / dt)
    oh = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12,
                        dtau=dt, inv_dtau_star=1.0 / dt, precision="mixed")
    s64 = api.esdirk_step(G64, A, b, dt, q64, o64)
    sh = api.esdirk_step(Gh, A, b, dt, qh, oh)
    assert s64["converged"] and sh["converged"]
    rel = ((qh - q64).abs().max() / q64.abs().max()).item()
    assert rel <= 1e-10, rel
    q0 = torch.from_numpy(np.ascontiguousarray(W.q0)).cuda()
    assert ((q64 - q0).abs().max() / q0.abs().max()).item() > 1e-6
