"""p-adaptation on the GPU (Sec. 3.3): the spectral-decay indicator (fr_spectral_decay)
against the oracle's numpy definition to 1e-12 (the two sum the modal energies in
different orders), on 2-D levels p = 1..4 and 3-D p = 2, 3, curved and periodic meshes,
for smooth and rough states; the marking rule (fr_padapt_mark) exactly."""
import math

import numpy as np
import pytest
import torch

from oracle import padapt as PA
from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


CASES = [
    ("omesh", lambda: w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [4, 3, 2, 1]),
    ("box2d", lambda: w.box2d(5, 5, 10, 10, qg=2, warp=0.1), [3, 2, 1]),
    ("box3d", lambda: w.box3d(3, 2 * math.pi), [3, 2]),
]


@pytest.mark.parametrize("name,make,levels", CASES, ids=[c[0] for c in CASES])
def test_indicator_and_marking_equal_the_oracle(name, make, levels):
    mesh = make()
    d = mesh["d"]
    G = api.fr_create(mesh, w.Physics(mu=0.01, qinf=w.freestream(d, 0.3)), levels)
    rng = np.random.default_rng(5)
    for l, p in enumerate(levels):
        X = w.solution_point_coords(mesh, p)
        smooth = np.sin(0.7 * X[0]) * np.cos(0.4 * X[1])
        q = np.zeros((d + 2, (p + 1) ** d, mesh["E"]))
        q[0] = 1.0
        q[1] = smooth + 1e-3 * rng.standard_normal(smooth.shape) * (np.arange(mesh["E"]) % 3 == 0)
        q[2] = rng.standard_normal(smooth.shape)
        eta_or = PA.spectral_decay(q, d, p, var=1)
        eta = api.fr_spectral_decay(G, l, torch.from_numpy(q).cuda(), var=1).cpu().numpy()
        assert np.max(np.abs(eta - eta_or)) <= 1e-12 * max(1.0, eta_or.max()), (name, p)
        eta2 = api.fr_spectral_decay(G, l, torch.from_numpy(q).cuda(), var=2).cpu().numpy()
        assert np.max(np.abs(eta2 - PA.spectral_decay(q, d, p, var=2))) <= 1e-12
        p_in = rng.integers(1, 5, size=mesh["E"]).astype(np.int32)
        p_out = api.fr_padapt_mark(G, torch.from_numpy(eta_or).cuda(), torch.from_numpy(p_in).cuda(), 1, 4)
        assert p_out.cpu().numpy().tolist() == PA.mark(eta_or, p_in, 1, 4).tolist()
