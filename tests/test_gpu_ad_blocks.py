"""FP32 element blocks (Eq. 9, Sec. 3.2) assembled element by element (fr_elem_blocks_f32,
method "local": each element's residual differentiated with the other side of every face
frozen except for the common solution's pull on the neighbour's BR2 lifting).

Checks, on meshes spanning periodic, curved, wall and far-field faces, 2-D and 3-D, both
inviscid fluxes:
  - the element-local blocks equal the whole-level forward-mode blocks over the element
    colouring, and both equal the oracle's FP64 forward-difference blocks, to 5e-4 of
    max |M|.  The two GPU paths round differently (opposite normals at the faces, other
    evaluation order) and sit at the same distance from the FP64 blocks: measured up to
    2.0e-4 on the 5^3 box at p = 2 (restricted from p = 3), 3e-5 on the other 3-D levels
    and below 1e-6 in 2-D, so the FP32 arithmetic, not the method, sets the difference;
  - a mesh whose faces join an element to itself is refused by the local method."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _wavy_state(mesh, p, mach=0.3, seed=0):
    X = w.solution_point_coords(mesh, p)
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.3, 1.2, size=(4, mesh["d"]))
    s = [np.sin(sum(k[i, c] * X[c] for c in range(mesh["d"])) + i) for i in range(4)]
    rho = 1.0 + 0.05 * s[0]
    vel = [math.cos(0.4) + 0.1 * s[1], math.sin(0.4) + 0.1 * s[2]] + ([0.05 * s[3]] if mesh["d"] == 3 else [])
    pr = (1.0 / (w.GAMMA * mach ** 2)) * (1 + 0.05 * s[3])
    return np.ascontiguousarray(w.prim_to_cons(rho, vel, pr))


CASES = {
    "vortex2d_p2": (lambda: w.box2d(8, 8, 10, 10, qg=2, warp=0.1), [2, 1], "rusanov"),
    "omesh_p4": (lambda: w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [4, 2, 1], "rusanov"),
    "omesh_p3_roe": (lambda: w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [3, 2], "roe"),
    "box3d_p3": (lambda: w.box3d(5, 2 * math.pi), [3, 2], "rusanov"),
    "box3d_p2": (lambda: w.box3d(3, 2.0), [2, 1], "rusanov"),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


@pytest.mark.parametrize("name", sorted(CASES))
def test_local_blocks_equal_colour_blocks_and_oracle(name):
    make, levels, flux = CASES[name]
    mesh = make()
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3), flux=flux)
    G = api.fr_create(mesh, ph, levels)
    O = oracle.Oracle(mesh, ph, levels)
    q = _wavy_state(mesh, levels[0])
    shift = 4.2
    for l in range(len(levels)):
        ql = q
        for k in range(l):
            ql = O.restrict(ql, k)
        q32 = torch.from_numpy(ql.astype(np.float32)).cuda()
        M_loc = api.fr_elem_blocks_f32(G, l, q32, shift, "local")
        M_col = api.fr_elem_blocks_f32(G, l, q32, shift, "colour")
        torch.cuda.synchronize()
        scale = M_col.abs().max().item()
        d_lc = (M_loc - M_col).abs().max().item() / scale
        assert d_lc <= 5e-4, (name, l, d_lc)
        if mesh["E"] <= 128:
            M_or = O.elem_blocks(ql, shift, np.arange(mesh["E"]), l)        # [e][r][j]
            M_or = torch.from_numpy(M_or).transpose(1, 2).cuda()              # -> [e][j][r]
            d_lo = (M_loc.double() - M_or).abs().max().item() / M_or.abs().max().item()
            assert d_lo <= 5e-4, (name, l, d_lo)


def test_local_method_refused_when_a_face_joins_an_element_to_itself():
    mesh = w.box3d(1, 2.0)
    ph = w.Physics(mu=0.02, qinf=w.freestream(3, 0.3))
    G = api.fr_create(mesh, ph, [2])
    q32 = torch.from_numpy(_wavy_state(mesh, 2).astype(np.float32)).cuda()
    with pytest.raises(Exception):
        api.fr_elem_blocks_f32(G, 0, q32, 2.0, "local")
    M = api.fr_elem_blocks_f32(G, 0, q32, 2.0, "colour")
    assert torch.isfinite(M).all()
