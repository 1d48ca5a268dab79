"""The per-element BF16 MLP of the Newton initial guess: GPU kernels vs the oracle's
BF16-emulating mode, training on the GPU, and the guess inside the ESDIRK driver.

Tolerances.  Both sides round the same operands to bfloat16 (nearest, ties to even) and
differ only in how they sum: FP32 on the tensor cores against FP64 in the oracle, and
tanhf against numpy's tanh.  Those differences (~1e-6 relative) matter only where an
activation sits within them of a bfloat16 rounding midpoint; there the two sides round
h (or an output gradient) to neighbouring bfloat16 values, 2^-8 |h| apart.  At the
sizes here that happens to a few entries in 10^4, each moving its outputs by at most
2^-8 max|W| |h|.  So: 99% of the entries agree to 1e-4 of the output's max norm and
all of them to 2e-2 (a handful of flips, each below 2^-8 x 4 of the scale)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as OM
from oracle import tableaux as OT
from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B
from paper_2202_09733_gb300 import tableaux as GT

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _init(rng, K0, H, O, out_scale=1.0):
    P = dict(W1=rng.standard_normal((H, K0)) / math.sqrt(K0), b1=rng.standard_normal(H) * 0.1,
             W2=rng.standard_normal((H, H)) / math.sqrt(H), b2=rng.standard_normal(H) * 0.1,
             W3=rng.standard_normal((O, H)) / math.sqrt(H) * out_scale, b3=rng.standard_normal(O) * 0.1)
    return {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}


def _flat(P):
    return np.concatenate([P[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def _unflat(v, K0, H, O):
    out, o = {}, 0
    for k, shp in (("W1", (H, K0)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))):
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def _agree(g, o, what, q99=1e-4):
    scale = max(np.abs(o).max(), 1e-30)
    d = np.abs(g - o) / scale
    assert np.quantile(d, 0.99) <= q99, (what, np.quantile(d, 0.99))
    assert d.max() <= 2e-2, (what, d.max())
    return float(d.max())


SIZES = [(32, 128, 64, 300), (224, 128, 64, 1000), (48, 64, 16, 7)]


@pytest.mark.parametrize("K0,H,O,Bn", SIZES)
def test_forward_matches_oracle_bf16(K0, H, O, Bn):
    rng = np.random.default_rng(K0 + Bn)
    P = _init(rng, K0, H, O)
    X32 = rng.standard_normal((Bn, K0)).astype(np.float32)
    net = api.MLP(K0, H, O, _flat(P))
    Y = net.forward(torch.from_numpy(X32).cuda().to(torch.bfloat16)).cpu().numpy()
    Yo, _ = OM.forward(P, X32.astype(np.float64), mode="bf16")
    _agree(Y, Yo, "y")
    # and the network really is the BF16 one: FP64 inputs differ from it by ~2^-8
    assert np.abs(OM.forward(P, X32.astype(np.float64))[0] - Yo).max() > 1e-4


@pytest.mark.parametrize("K0,H,O,Bn", SIZES)
def test_gradients_match_oracle_bf16(K0, H, O, Bn):
    rng = np.random.default_rng(7 * K0 + Bn)
    P = _init(rng, K0, H, O)
    X32 = rng.standard_normal((Bn, K0)).astype(np.float32)
    T32 = rng.standard_normal((Bn, O)).astype(np.float32)
    net = api.MLP(K0, H, O, _flat(P))
    grads = torch.zeros(net.nparams, dtype=torch.float32, device="cuda")
    loss = net.train_step(torch.from_numpy(X32).cuda().to(torch.bfloat16), torch.from_numpy(T32).cuda(), lr=0.0,
                          grads=grads)
    yo, cache = OM.forward(P, X32.astype(np.float64), mode="bf16")
    Go = OM.backward(P, cache, yo, T32.astype(np.float64), mode="bf16")
    assert abs(loss - OM.loss(yo, T32)) <= 1e-4 * OM.loss(yo, T32)
    G = _unflat(grads.cpu().numpy(), K0, H, O)
    for k in Go:
        # a weight gradient sums Bn products; a flipped bf16 operand moves one of them by
        # 2^-8 of itself, i.e. ~2^-8 / sqrt(Bn) of the sum's scale
        _agree(G[k], Go[k], k, q99=max(1e-4, 4 * 2.0 ** -8 / math.sqrt(Bn)))
    # lr = 0 leaves the master weights alone
    assert np.array_equal(net.params(), _flat(P))


def test_adam_step_matches_oracle():
    K0, H, O, Bn = 32, 64, 16, 256
    rng = np.random.default_rng(11)
    P = _init(rng, K0, H, O)
    X = torch.from_numpy(rng.standard_normal((Bn, K0)).astype(np.float32)).cuda().to(torch.bfloat16)
    T = torch.from_numpy(rng.standard_normal((Bn, O)).astype(np.float32)).cuda()
    net = api.MLP(K0, H, O, _flat(P))
    state = {}
    Pk = {k: v.copy() for k, v in P.items()}
    grads = torch.zeros(net.nparams, dtype=torch.float32, device="cuda")
    for it in range(3):
        net.train_step(X, T, lr=1e-3, grads=grads)
        # the oracle's FP64 Adam driven by the GPU's gradients, from the GPU's weights
        Pk = _unflat(_flat(Pk), K0, H, O)
        Pk = OM.adam(Pk, _unflat(grads.cpu().numpy(), K0, H, O), state, lr=1e-3)
        got = _unflat(net.params(), K0, H, O)
        for k in Pk:
            assert np.abs(got[k] - Pk[k]).max() <= 1e-7, (it, k)
        Pk = got


def test_training_fits_a_teacher():
    """Training on the GPU (own forward, backward and Adam kernels) fits a random teacher
    network of the same shape."""
    K0, H, O, Bn = 64, 128, 32, 2048
    rng = np.random.default_rng(5)
    teacher = _init(rng, K0, H, O)
    X32 = rng.standard_normal((Bn, K0)).astype(np.float32)
    T = OM.forward(teacher, X32.astype(np.float64))[0].astype(np.float32)
    net = api.MLP(K0, H, O, _flat(_init(rng, K0, H, O)))
    Xg = torch.from_numpy(X32).cuda().to(torch.bfloat16)
    Tg = torch.from_numpy(T).cuda()
    losses = [net.train_step(Xg, Tg, lr=2e-3) for _ in range(400)]
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    assert all(np.isfinite(losses))
    # and the trained weights predict the teacher through the inference kernel
    Y = net.forward(Xg).cpu().numpy()
    assert np.mean((Y - T) ** 2) < 0.1 * np.mean(T ** 2)


def test_mlp_rejects_bad_arguments():
    with pytest.raises(Exception):
        api.MLP(33, 16, 8, np.zeros(33 * 16 + 16 + 256 + 16 + 128 + 8, dtype=np.float32))   # odd width
    net = api.MLP(32, 16, 8, np.zeros(32 * 16 + 16 + 256 + 16 + 128 + 8, dtype=np.float32))
    with pytest.raises(ValueError):
        net.forward(torch.zeros((4, 32), dtype=torch.float32, device="cuda"))               # not bf16


# ----------------------------------------------------------------- inside the solver
def _cyl_case():
    """Impulsively started low-Mach cylinder (O-mesh 24 x 48, first cell 0.01, p = 3,
    Ma 0.05, Re 150) at CFL 50: the unsteady shape of the paper's cylinder case, small."""
    return w.cylinder_unsteady(nr=24, nt=48, p=3)


def _run(wl, guess, nsteps, net=None, train_iters=0, precision="fp64", tol_newton=1e-9):
    G = api.fr_create(wl.mesh, wl.phys, wl.levels)
    if net is not None:
        api.fr_set_mlp(G, net)
    A, b = GT.esdirk3()
    dt = wl.dt
    o = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=tol_newton,
                       dtau=dt, inv_dtau_star=1.0 / dt, precision=precision, guess=guess,
                       train_iters=train_iters, train_batch=4096, lr=1e-3)
    q = torch.from_numpy(np.ascontiguousarray(wl.q0)).cuda()
    hist, states = [], []
    for n in range(nsteps):
        st = api.esdirk_step(G, A, b, dt, q, o, allow_not_converged=False)
        hist.append(st)
        states.append(q.cpu().numpy().copy())
    return hist, states


def test_guess_features_match_oracle():
    wl = _cyl_case()
    G = api.fr_create(wl.mesh, wl.phys, wl.levels)
    O = oracle.Oracle(wl.mesh, wl.phys, wl.levels)
    rng = np.random.default_rng(9)
    q2 = np.ascontiguousarray(wl.q0)
    q1 = q2 * (1 + 1e-3 * rng.standard_normal(q2.shape))
    qn = q1 * (1 + 1e-3 * rng.standard_normal(q2.shape))
    Rn = O.residual(qn)
    dt, c = wl.dt, 0.87
    X, s, sig = api.fr_guess_features(G, *(torch.from_numpy(a).cuda() for a in (qn, q1, q2, Rn)), dt, c)
    so, sigo = OM.scales(qn, q1, wl.phys.qinf)
    assert np.abs(s - so).max() <= 1e-13 * so.max() and np.abs(sig - sigo).max() <= 1e-13 * sigo.max()
    K0 = X.shape[1]
    logJ = np.log(np.abs(O.jacobian_det(0)))
    Xo = OM.bf16(OM.features(qn, q1, q2, Rn, dt, logJ, c, so, sigo, wl.phys.qinf, K0))
    Xg = X.float().cpu().numpy().astype(np.float64)
    # bf16 of FP64 values whose last bits differ (tree vs sequential sums in the scales,
    # log of the stored 1/J): equal, or one bf16 ulp apart at a rounding midpoint
    d = np.abs(Xg - Xo)
    assert np.all(d <= 2.0 ** -7 * np.abs(Xo) + 1e-30)
    assert np.mean(d == 0) > 0.999


def test_extrapolated_guess_keeps_the_answer_and_saves_newton_iterations():
    wl = _cyl_case()
    nsteps = 24
    h0, s0 = _run(wl, "qn", nsteps)
    h1, s1 = _run(wl, "extrap", nsteps)
    for a, b_ in zip(s0, s1):
        assert np.abs(a - b_).max() <= 1e-7 * np.abs(a).max()
    # past the impulsive start (where the history is a poor predictor and q^n wins)
    late = h1[12:]
    assert all(st["guess_rms"][1] < st["guess_rms"][0] for st in late)
    assert sum(st["guess_pick"][1] for st in late) == 3 * len(late)
    n0 = sum(st["n_ptc"] for st in h0[12:])
    n1 = sum(st["n_ptc"] for st in late)
    assert n1 < n0, (n0, n1)


def test_learned_guess_trains_online_and_keeps_the_answer():
    """The network trains on the stages the solver converges (own BF16 kernels), its
    candidate is judged by the FP64 stage residual, and the converged trajectory does not
    change.  Reported: which candidate each stage starts from, the mean stage residual of
    each candidate, and the Newton iterations against the q^n run (the paper's guess)."""
    wl = _cyl_case()
    G0 = api.fr_create(wl.mesh, wl.phys, wl.levels)
    K0, O = api.fr_mlp_dims(G0)
    assert K0 % 16 == 0 and K0 >= 4 * O + 16 + 1 and O == 4 * 16
    rng = np.random.default_rng(3)
    net = api.MLP(K0, 128, O, _flat(_init(rng, K0, 128, O, out_scale=0.1)))
    nsteps = 24
    h2, s2 = _run(wl, "mlp", nsteps, net=net, train_iters=30)
    h0, s0 = _run(wl, "qn", nsteps)
    for a, b_ in zip(s0, s2):
        assert np.abs(a - b_).max() <= 1e-7 * np.abs(a).max()
    losses = [st["train_loss"] for st in h2[3:]]
    assert all(np.isfinite(losses)) and losses[-1] < losses[0]
    late = h2[12:]
    picks = [sum(st["guess_pick"][k] for st in late) for k in range(3)]
    rms = [float(np.mean([st["guess_rms"][k] for st in late])) for k in range(3)]
    n0 = sum(st["n_ptc"] for st in h0[12:])
    n2 = sum(st["n_ptc"] for st in late)
    print("learned guess, steps 13..24: picks (q^n, extrap, mlp)", picks, "mean RMS", rms,
          "mean beta", float(np.mean([st["guess_beta"] for st in late])),
          "Newton its q^n run", n0, "learned run", n2)
    assert rms[2] < rms[0]          # the trained network beats the paper's guess
    assert picks[0] == 0 and n2 < n0


def test_guess_requires_a_network():
    wl = _cyl_case()
    G = api.fr_create(wl.mesh, wl.phys, wl.levels)
    A, b = GT.esdirk3()
    o = api.solve_opts(guess="mlp", dtau=wl.dt)
    q = torch.from_numpy(np.ascontiguousarray(wl.q0)).cuda()
    with pytest.raises(Exception, match="network"):
        api.esdirk_step(G, A, b, wl.dt, q, o)
    with pytest.raises(Exception):
        api.fr_set_mlp(G, api.MLP(32, 16, 8, np.zeros(32 * 16 + 16 + 256 + 16 + 128 + 8, dtype=np.float32)))


def test_checkpoint_resume_is_bit_identical():
    """Save the learned guess's state (history, training ring, network and Adam moments)
    after five steps, restore it into a fresh context and a fresh network, and step on:
    the resumed run reproduces the uninterrupted one bit for bit."""
    wl = _cyl_case()
    A, b = GT.esdirk3()
    dt = wl.dt
    o = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-9,
                       dtau=dt, inv_dtau_star=1.0 / dt, guess="mlp", train_iters=5, train_batch=1024, lr=1e-3)

    def fresh(seed):
        G = api.fr_create(wl.mesh, wl.phys, wl.levels)
        K0, O = api.fr_mlp_dims(G)
        net = api.MLP(K0, 64, O, _flat(_init(np.random.default_rng(seed), K0, 64, O, out_scale=0.1)))
        api.fr_set_mlp(G, net)
        return G, net

    G1, net1 = fresh(1)
    q = torch.from_numpy(np.ascontiguousarray(wl.q0)).cuda()
    for _ in range(5):
        api.esdirk_step(G1, A, b, dt, q, o, allow_not_converged=False)
    ck = api.fr_checkpoint_save(G1, net1)
    q_saved = q.clone()
    for _ in range(3):
        st1 = api.esdirk_step(G1, A, b, dt, q, o, allow_not_converged=False)
    G2, net2 = fresh(2)                        # other initial weights: the checkpoint must carry them
    api.fr_checkpoint_load(G2, ck, net2)
    q2 = q_saved.clone()
    for _ in range(3):
        st2 = api.esdirk_step(G2, A, b, dt, q2, o, allow_not_converged=False)
    assert torch.equal(q, q2)
    assert st1["guess_pick"] == st2["guess_pick"] and st1["n_gmres"] == st2["n_gmres"]
    assert np.array_equal(net1.params(), net2.params())
    # a checkpoint of another mesh is refused
    G3 = api.fr_create(w.cylinder_unsteady(nr=12, nt=24, p=3).mesh, wl.phys, wl.levels)
    with pytest.raises(Exception, match="mesh"):
        api.fr_checkpoint_load(G3, ck, net2)
