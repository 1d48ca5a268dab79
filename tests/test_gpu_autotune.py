"""Launch shapes change no result bit: the residual under any CTA sizes, the FP32
preconditioner under any solve G, and the autotuned batched step are bit-identical to the
default shapes (and the residual to the oracle)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import tableaux as OT
from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B
from paper_2202_09733_gb300 import tableaux as GT

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


CASES = {
    "quad_p4": (w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [4, 2]),
    "hex_p3": (w.box3d(5, 2 * math.pi), [3, 2]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_bits_do_not_depend_on_tiles(name):
    mesh, lv = CASES[name]
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3))
    O = oracle.Oracle(mesh, ph, lv)
    G = api.fr_create(mesh, ph, lv)
    rng = np.random.default_rng(1)
    X = w.solution_point_coords(mesh, lv[0])
    q = np.ascontiguousarray(w.prim_to_cons(1 + 0.05 * np.sin(X[0]), [0.3 + 0.1 * np.cos(X[1])] +
                                            [0.1 * np.sin(X[0] + X[1])] * (mesh["d"] - 1),
                                            (1 / (1.4 * 0.09)) * np.ones_like(X[0])))
    R_or = O.residual(q)
    qg = torch.from_numpy(q).cuda()
    for trial in range(4):
        tiles = [int(x) for x in rng.choice([32, 64, 96, 128, 160, 256], size=8)] + [0]
        api.fr_set_tiles(G, 0, tiles)
        assert api.fr_get_tiles(G, 0)[:8] == tiles[:8]
        assert np.array_equal(api.fr_residual(G, 0, qg).cpu().numpy(), R_or), tiles
    rep = api.fr_autotune(G, fp64=True, fp32=True, retune=True, reps=2)
    assert len(rep) == 2 * len(lv) and all("tiles" in r for r in rep)
    assert np.array_equal(api.fr_residual(G, 0, qg).cpu().numpy(), R_or)
    with pytest.raises(Exception):
        api.fr_set_tiles(G, 0, [100] * 8 + [0])


def test_fp32_preconditioner_bits_do_not_depend_on_solve_G():
    mesh, lv = CASES["quad_p4"]
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, 0.3))
    G = api.fr_create(mesh, ph, lv)
    X = w.solution_point_coords(mesh, lv[0])
    q = np.ascontiguousarray(w.prim_to_cons(1 + 0.05 * np.sin(X[0]), [0.3 + 0.1 * np.cos(X[1]), 0.1 * np.sin(X[0])],
                                            (1 / (1.4 * 0.09)) * np.ones_like(X[0])))
    qg = torch.from_numpy(q).cuda()
    Rq = api.fr_residual(G, 0, qg)
    v = torch.from_numpy(np.random.default_rng(2).standard_normal(q.shape)).cuda()
    outs = []
    for g in (1, 2, 4, 8):
        for l in range(len(lv)):
            api.fr_set_tiles(G, l, [0] * 8 + [g], precision=1)
        api.pmg_setup(G, qg, [2, 2], 10.0, 3.0, precision="mixed")
        outs.append(api.pmg_precondition(G, qg, Rq, v))
    for o in outs[1:]:
        assert torch.equal(outs[0], o)
    assert api.fr_kernel_timeouts() == 0


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_block_solve_variants_match_oracle_bitwise(name):
    """The register kernels (G = 2, 4, 8) and the bulk-copy kernel (G = 1) apply the same
    fma sequence to every row: the solves agree with each other and the oracle bit for bit."""
    mesh, lv = CASES[name]
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3))
    O = oracle.Oracle(mesh, ph, lv)
    G = api.fr_create(mesh, ph, lv)
    X = w.solution_point_coords(mesh, lv[0])
    q = np.ascontiguousarray(w.prim_to_cons(1 + 0.05 * np.sin(X[0]), [0.3 + 0.1 * np.cos(X[1])] +
                                            [0.1 * np.sin(X[0] + X[1])] * (mesh["d"] - 1),
                                            (1 / (1.4 * 0.09)) * np.ones_like(X[0])))
    qg = torch.from_numpy(q).cuda()
    M = api.fr_elem_blocks(G, 0, qg, 7.5)
    perm = api.fr_block_factor(G, 0, M)
    O.pmg_setup(q, [1], 7.5, 0.0)
    rhs = np.random.default_rng(4).standard_normal(q.shape)
    ref = O.block_solve(rhs)
    outs = []
    for g in (1, 2, 4, 8):
        api.fr_set_tiles(G, 0, [0] * 8 + [g])
        outs.append(api.fr_block_solve(G, 0, M, perm, torch.from_numpy(rhs.copy()).cuda()).cpu().numpy())
    for o in outs:
        assert np.array_equal(o, ref)
    assert api.fr_kernel_timeouts() == 0


def test_autotuned_batch_step_is_bit_identical():
    probs, states, phys, dt = w.vortex_batch(nprob=6, nmin=3, nmax=6, pmin=1, pmax=4, seed=5, cfl=10.0)
    Ag, bg = GT.esdirk3()
    go = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-10,
                        dtau=dt, inv_dtau_star=1.0 / dt, precision="mixed")
    res = []
    for tune in (False, True):
        Bt = api.Batch(probs, phys)
        qs = [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in states]
        if tune:
            # a step first, so that the blocks are factored and the solve's G is tuned too
            Bt.esdirk_step(Ag, bg, dt, [q.clone() for q in qs], go)
            rep = Bt.autotune(fp64=True, fp32=True, retune=True, reps=2)
            assert any("solve G" in r and "not tuned" not in r for r in rep)
        Bt.esdirk_step(Ag, bg, dt, qs, go, allow_not_converged=False)
        res.append(qs)
    for a, b_ in zip(*res):
        assert torch.equal(a, b_)


def test_bounded_wait_times_out_and_leaves_the_context_usable():
    """A stage barrier that nothing completes: the bounded wait gives up, the failure is
    reported to the host, and the next solve still runs (and is exact)."""
    mesh, lv = CASES["quad_p4"]
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, 0.3))
    G = api.fr_create(mesh, ph, lv)
    api.fr_kernel_timeouts(clear=True)
    api.fr_selftest_wait_timeout()
    assert api.fr_kernel_timeouts(clear=True) == 1
    assert api.fr_kernel_timeouts() == 0
    X = w.solution_point_coords(mesh, lv[0])
    q = np.ascontiguousarray(w.prim_to_cons(1 + 0.05 * np.sin(X[0]), [0.3 + 0.1 * np.cos(X[1]), 0.1 * np.sin(X[0])],
                                            (1 / (1.4 * 0.09)) * np.ones_like(X[0])))
    qg = torch.from_numpy(q).cuda()
    M = api.fr_elem_blocks(G, 0, qg, 7.5)
    perm = api.fr_block_factor(G, 0, M)
    rhs = torch.from_numpy(np.random.default_rng(6).standard_normal(q.shape)).cuda()
    outs = []
    for g in (1, 2):
        api.fr_set_tiles(G, 0, [0] * 8 + [g])
        outs.append(api.fr_block_solve(G, 0, M, perm, rhs.clone()))
    assert torch.equal(outs[0], outs[1]) and api.fr_kernel_timeouts() == 0
