"""The batched solver (many independent problems of uneven size and degree in one step)
against the oracle, problem by problem, and against the one-problem GPU path.

Tolerances: the batched residual is the one-problem residual bit for bit (the same
kernels evaluate each element from its own problem's data); one converged ESDIRK3 step
(Newton tolerance 1e-12) agrees with the oracle's to 1e-10, as the one-problem step does;
graphs on and off run the same kernels on the same data and agree bit for bit."""
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


def relerr(a, b):
    a = a.detach().cpu().numpy() if torch.is_tensor(a) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def small():
    # 7 problems, n in 3..5, p in 1..3: three groups, ragged element counts
    probs, states, phys, dt = w.vortex_batch(nprob=7, nmin=3, nmax=5, pmin=1, pmax=3, seed=11, cfl=10.0)
    return probs, states, phys, dt


def _dev(states):
    return [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in states]


def test_batch_groups_and_residual_bitwise(small):
    probs, states, phys, dt = small
    Bt = api.Batch(probs, phys)
    ng, grp, off = Bt.info()
    assert ng == len({tuple(lv) for _, lv in probs})
    for k in range(len(probs)):
        same = [j for j in range(k) if grp[j] == grp[k]]
        assert off[k] == sum(probs[j][0]["E"] for j in same)
    qs = _dev(states)
    Rs = Bt.residual(qs)
    for k, (mesh, lv) in enumerate(probs):
        G = api.fr_create(mesh, phys, lv)
        R1 = api.fr_residual(G, 0, qs[k])
        assert torch.equal(Rs[k], R1), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_esdirk_step_matches_oracle(small, precision):
    probs, states, phys, dt = small
    Bt = api.Batch(probs, phys)
    Ag, bg = GT.esdirk3()
    A, b, _ = OT.esdirk3()
    go = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12,
                        dtau=dt, inv_dtau_star=1.0 / dt, precision=precision)
    qs = _dev(states)
    stats = Bt.esdirk_step(Ag, bg, dt, qs, go, allow_not_converged=False)
    assert all(st["converged"] for st in stats)
    for k, (mesh, lv) in enumerate(probs):
        O = oracle.Oracle(mesh, phys, lv)
        oo = O.opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2)[:len(lv)], tol_gmres=1e-2,
                    tol_newton=1e-12, dtau=dt, inv_dtau_star=1.0 / dt)
        q_or, st_or = O.esdirk_step(A, b, dt, states[k], oo)
        assert st_or["converged"]
        assert relerr(qs[k], q_or) <= 1e-10, (k, precision, relerr(qs[k], q_or))
        assert relerr(qs[k], states[k]) > 1e-6


def test_batch_matches_single_problem_path_and_graphs_are_exact(small):
    probs, states, phys, dt = small
    Ag, bg = GT.esdirk3()
    go = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-10,
                        dtau=dt, inv_dtau_star=1.0 / dt)
    runs = []
    for graphs in (True, False):
        Bt = api.Batch(probs, phys)
        Bt.set_graphs(graphs)
        qs = _dev(states)
        stats = Bt.esdirk_step(Ag, bg, dt, qs, go, allow_not_converged=False)
        runs.append((qs, stats))
    for a, b_ in zip(runs[0][0], runs[1][0]):
        assert torch.equal(a, b_)
    assert [s["n_gmres"] for s in runs[0][1]] == [s["n_gmres"] for s in runs[1][1]]
    for k, (mesh, lv) in enumerate(probs):
        G = api.fr_create(mesh, phys, lv)
        go1 = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2)[:len(lv)], tol_gmres=1e-2,
                             tol_newton=1e-10, dtau=dt, inv_dtau_star=1.0 / dt)
        q1 = torch.from_numpy(np.ascontiguousarray(states[k])).cuda()
        st1 = api.esdirk_step(G, Ag, bg, dt, q1, go1, allow_not_converged=False)
        assert relerr(runs[0][0][k], q1.cpu().numpy()) <= 1e-9
        # the same iteration, up to the rounding of the inner products
        assert abs(st1["n_gmres"] - runs[0][1][k]["n_gmres"]) <= 2 + st1["n_gmres"] // 10
        assert st1["n_ptc"] == runs[0][1][k]["n_ptc"]


def test_batch_rejects_bad_input(small):
    probs, states, phys, dt = small
    Bt = api.Batch(probs, phys)
    with pytest.raises(ValueError):
        Bt.residual(_dev(states)[:-1])
    Ag, bg = GT.esdirk3()
    with pytest.raises(Exception, match="guess"):
        Bt.esdirk_step(Ag, bg, dt, _dev(states), api.solve_opts(guess="extrap", dtau=dt))
