"""The seeded input generators (host only): meshes are watertight (every element face is
listed exactly once, as an interior pair or a boundary), shared face nodes coincide,
Jacobians are positive, the batch generator is deterministic in its seed and spans the
stated size and degree ranges."""
import math

import numpy as np
import pytest

from paper_2202_09733_gb300 import workloads as w


def _face_census(mesh):
    d, E = mesh["d"], mesh["E"]
    seen = np.zeros((E, 2 * d), dtype=int)
    nbound = 0
    for eL, fL, eR, fR, orient, bc in mesh["faces"]:
        seen[eL, fL] += 1
        if eR >= 0:
            seen[eR, fR] += 1
        else:
            assert bc in (1, 2)
            nbound += 1
    return seen, nbound


@pytest.mark.parametrize("mesh", [w.box2d(5, 3, 10, 6, qg=2, warp=0.1), w.box3d(3, 2.0),
                                  w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3)],
                         ids=["box2d", "box3d", "omesh"])
def test_every_face_listed_once(mesh):
    seen, nbound = _face_census(mesh)
    assert np.all(seen == 1)
    if mesh.get("kind") == "box2d" or mesh["d"] == 3:
        assert nbound == 0                      # periodic boxes
    else:
        assert nbound == 2 * 12                 # wall and far field rings


def test_omesh_shared_nodes_coincide_and_stretch():
    mesh = w.omesh(8, 16, 0.5, 20.0, 0.01, jitter=0.05, seed=1)
    m = mesh["qg"] + 1
    g = mesh["gnodes"].reshape(mesh["E"], m, m, 2)      # [e][a1][a0][xy]
    for eL, fL, eR, fR, orient, bc in mesh["faces"]:
        if eR < 0 or fL != 1:
            continue                                     # radial neighbours: xi = +1 of eL meets xi = -1 of eR
        a = g[eL, :, -1, :]
        b = g[eR, :, 0, :]
        assert np.abs(a - b).max() < 1e-12
    r = np.hypot(g[..., 0], g[..., 1])
    assert abs(r.min() - 0.5) < 1e-12 and abs(r.max() - 20.0) < 1e-9
    assert abs(mesh["h_min"] - 0.01) < 1e-3


def test_vortex_batch_is_seeded_and_spans_its_ranges():
    p1, s1, ph1, dt1 = w.vortex_batch(nprob=40, seed=7)
    p2, s2, ph2, dt2 = w.vortex_batch(nprob=40, seed=7)
    p3, s3, _, _ = w.vortex_batch(nprob=40, seed=8)
    assert dt1 == dt2 and all(np.array_equal(a, b) for a, b in zip(s1, s2))
    assert not all(a.shape == b.shape and np.array_equal(a, b) for a, b in zip(s1, s3))
    ns = [int(round(math.sqrt(m["E"]))) for m, _ in p1]
    ps = [lv[0] for _, lv in p1]
    assert min(ns) >= 4 and max(ns) <= 48 and set(ps) <= {1, 2, 3, 4}
    for (m, lv), q in zip(p1, s1):
        assert lv == ([lv[0], lv[0] - 1] if lv[0] > 1 else [1])
        assert q.shape == (4, (lv[0] + 1) ** 2, m["E"])
        assert np.all(q[0] > 0)                            # positive density
    # one dt for the batch: the smallest explicit limit times 20
    assert abs(dt1 - 20.0 * min(w.explicit_dt(m, lv[0], q) for (m, lv), q in zip(p1, s1))) < 1e-15


def test_states_are_physical():
    for wl in (w.vortex2d(), w.tgv3d(n=4), w.cylinder_unsteady(nr=6, nt=12)):
        q = wl.q0
        d = wl.mesh["d"]
        rho = q[0]
        ke = 0.5 * np.sum(q[1:1 + d] ** 2, axis=0) / rho
        p = (w.GAMMA - 1.0) * (q[d + 1] - ke)
        assert np.all(rho > 0) and np.all(p > 0)
        assert wl.dt > 0

