"""FP32 block LU with the trailing updates on the tensor cores (fr_block_factor_f32,
method "tensor_cores"; pmg_setup's default for FP32 blocks of size 65..384).

The factorisation is LU with partial pivoting of every element block (the element-Jacobi
blocks of Eq. 9 that the Sec. 3.2 smoother solves with).  Checked against a plain PyTorch
FP64 reference of the same operation and against the CUDA-core FP32 kernels:
  - perm is a permutation and P A = L U holds per block to FP32 accuracy: the backward
    error max|P A - L U| / max|A| stays within 4x the CUDA-core factors' own plus 1e-6
    (FP32 elimination on n = 320 with growth g leaves about n u g; the split TF32
    products add about 2^-22 per product, below u = 2^-24 times the K = 32 terms);
  - the block solve with these factors is as close to the FP64 solve as the CUDA-core
    factors' solve (4x their error plus 1e-6), on Gaussian blocks, which need row
    interchanges, and on the element blocks of the 3-D p = 3 / p = 2 and the 2-D p = 4
    wall-resolved levels;
  - blocks whose size is not a multiple of the 32-column panel (100, 135) and one that is
    (320); block sizes outside 65..384 are refused by method "tensor_cores";
  - the mixed pMG cycle stays within its 5e-3 bar of the FP64 cycle with either
    factorisation, and no further from it with the tensor-core factors (the cycle's FP32
    state differences, about 1e-3 of its largest entry, not the factors, set the gap).
"""
import math

import numpy as np
import pytest
import torch

from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _ctx(kind):
    if kind == "box3d_p3":          # nd = 5 * 64 = 320, coarse 5 * 27 = 135
        mesh, levels = w.box3d(4, 2 * math.pi), [3, 2]
    elif kind == "omesh_p4":        # nd = 4 * 25 = 100 (wall cells of aspect ratio 1e2)
        mesh, levels = w.omesh(6, 12, 0.5, 5.0, 0.01, jitter=0.05, seed=3), [4, 2]
    else:
        raise KeyError(kind)
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3))
    return api.fr_create(mesh, ph, levels), mesh, levels


def _unpack(F, perm):
    """L (unit lower), U, perm of in-place factors F[e, j, r] (column-major per block)."""
    A = F.double().transpose(1, 2)                    # [e, r, j]
    nd = A.shape[-1]
    eye = torch.eye(nd, dtype=torch.float64, device=A.device)
    L = torch.tril(A, -1) + eye
    U = torch.triu(A, 1) + torch.diag_embed(1.0 / torch.diagonal(A, dim1=1, dim2=2))
    return L, U


def _backward_error(M, F, perm):
    A = M.double().transpose(1, 2)
    L, U = _unpack(F, perm)
    PA = torch.gather(A, 1, perm.long().unsqueeze(-1).expand_as(A))
    return ((PA - L @ U).abs().amax(dim=(1, 2)) / A.abs().amax(dim=(1, 2))).max().item()


def _solve_error(G, level, M, F, perm):
    E, nd = M.shape[0], M.shape[1]
    rng = np.random.default_rng(7)
    b = torch.from_numpy(rng.standard_normal((nd, E))).cuda()
    x = api.fr_block_solve_f32(G, level, F, perm, b.float().contiguous())
    A = M.double().transpose(1, 2)
    ref = torch.linalg.solve(A, b.float().double().T.unsqueeze(-1)).squeeze(-1).T
    return ((x.double() - ref).abs().amax(dim=0) / ref.abs().amax(dim=0)).max().item()


def _check(G, level, M):
    nd = M.shape[1]
    F_tc, F_cc = M.clone(), M.clone()
    p_tc = api.fr_block_factor_f32(G, level, F_tc, "tensor_cores")
    p_cc = api.fr_block_factor_f32(G, level, F_cc, "cuda_cores")
    torch.cuda.synchronize()
    srt = torch.sort(p_tc.long(), dim=1).values
    assert torch.equal(srt, torch.arange(nd, device="cuda").expand_as(srt)), "perm is not a permutation"
    be_tc, be_cc = _backward_error(M, F_tc, p_tc), _backward_error(M, F_cc, p_cc)
    assert be_tc <= 4 * be_cc + 1e-6, (nd, be_tc, be_cc)
    se_tc, se_cc = _solve_error(G, level, M, F_tc, p_tc), _solve_error(G, level, M, F_cc, p_cc)
    assert se_tc <= 4 * se_cc + 1e-6, (nd, se_tc, se_cc)
    return p_tc, p_cc


@pytest.mark.parametrize("kind,level", [("box3d_p3", 0), ("box3d_p3", 1), ("omesh_p4", 0)])
def test_gaussian_blocks_with_interchanges(kind, level):
    G, mesh, levels = _ctx(kind)
    nd = G.nd(level)
    g = torch.Generator(device="cuda").manual_seed(11 + level)
    M = torch.randn((G.E, nd, nd), generator=g, device="cuda", dtype=torch.float32)
    p_tc, p_cc = _check(G, level, M)
    ident = torch.arange(nd, device="cuda", dtype=torch.int32)
    assert (p_tc != ident).any(dim=1).all(), "Gaussian blocks should all need interchanges"
    # the pivot rows follow from comparisons of values that the two methods round
    # differently; near-ties aside they are the same rows
    assert (p_tc == p_cc).all(dim=1).float().mean().item() >= 0.9


@pytest.mark.parametrize("kind", ["box3d_p3", "omesh_p4"])
def test_element_blocks_of_the_levels(kind):
    G, mesh, levels = _ctx(kind)
    X = w.solution_point_coords(mesh, levels[0])
    rng = np.random.default_rng(1)
    d = mesh["d"]
    vel = [0.3 + 0.02 * np.sin(X[0] + rng.uniform()), 0.02 * np.cos(X[1])] + ([0.01 * np.sin(X[2])] if d == 3 else [])
    q = w.prim_to_cons(1.0 + 0.01 * np.sin(X[0]), vel, (1 / (w.GAMMA * 0.3 ** 2)) * (1 + 0.01 * np.cos(X[1])))
    q = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    ql = q
    for l in range(len(levels)):
        if l > 0:
            ql = api.fr_restrict(G, l - 1, ql)
        M = api.fr_elem_blocks_f32(G, l, ql.float().contiguous(), 3.0)
        if 65 <= G.nd(l) <= 384:
            _check(G, l, M)


def test_sizes_outside_the_tensor_core_range_are_refused():
    mesh = w.box2d(4, 4, 10, 10, qg=2)
    G = api.fr_create(mesh, w.Physics(mu=0.01, qinf=w.freestream(2, 0.3)), [2, 1])   # nd = 36
    M = torch.randn((G.E, 36, 36), device="cuda", dtype=torch.float32) + 8 * torch.eye(36, device="cuda")
    with pytest.raises(Exception):
        api.fr_block_factor_f32(G, 0, M.clone(), "tensor_cores")
    F = M.clone()
    perm = api.fr_block_factor_f32(G, 0, F, "auto")      # falls back to the CUDA-core kernel
    assert _backward_error(M, F, perm) <= 1e-5


def test_mixed_cycle_same_with_either_factorisation():
    W = w.tgv3d(n=4)
    G = api.fr_create(W.mesh, W.phys, W.levels)
    q = torch.from_numpy(np.ascontiguousarray(W.q0)).cuda()
    R = api.fr_residual(G, 0, q)
    v = torch.from_numpy(np.random.default_rng(0).standard_normal(W.q0.shape)).cuda()
    v /= v.norm()
    c = 1.0 / W.dt + 1.0 / (0.4358665215084590 * W.dt)
    api.pmg_setup(G, q, [2, 2], c, 1.0 / W.dt, precision="fp64")
    y64 = api.pmg_precondition(G, q, R, v).clone()
    scale = y64.abs().max().item()
    err = {}
    for meth in ("auto", "cuda_cores"):
        api.fr_set_lu_method(G, meth)
        api.pmg_setup(G, q, [2, 2], c, 1.0 / W.dt, precision="mixed")
        err[meth] = (api.pmg_precondition(G, q, R, v) - y64).abs().max().item() / scale
    # the mixed cycle's own bar against the FP64 cycle (its FP32 state differences set
    # it), met by both, and the tensor-core factors no further from the FP64 cycle
    assert err["auto"] <= 5e-3 and err["cuda_cores"] <= 5e-3, err
    assert err["auto"] <= 2 * err["cuda_cores"] + 1e-4, err
    assert api.fr_kernel_timeouts(True) == 0
