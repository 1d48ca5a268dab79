"""Host connectivity of the matrix-based smoother, without a GPU: the library's face-
neighbour table (built in C from the face list) equals the oracle's (built independently),
and its greedy distance-2 colouring gives no two elements within two face steps the same
colour, on a curved O-mesh with boundaries, periodic boxes one and two elements wide in a
direction, and hexes."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2202_09733_gb300 import workloads as w

MESHES = {
    "omesh": lambda: w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3),
    "box2d_two_wide": lambda: w.box2d(2, 5, 4.0, 6.0, qg=2, warp=0.1),
    "box2d": lambda: w.box2d(7, 5, 7.0, 5.0, qg=2, warp=0.1),
    "box3d": lambda: w.box3d(4, 2.0),
}


@pytest.fixture(scope="module")
def lib():
    from paper_2202_09733_gb300 import build as B, _native as N
    B.build()
    L = N.load()
    PI = C.POINTER(C.c_int)
    L.frh_neighbours.argtypes = [C.c_int, C.c_int, C.c_int, PI, PI]
    L.frh_neighbours.restype = C.c_int
    L.frh_color2.argtypes = [C.c_int, C.c_int, PI, PI]
    L.frh_color2.restype = C.c_int
    return L


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


@pytest.mark.parametrize("name", sorted(MESHES))
def test_neighbours_and_distance2_colouring(lib, name):
    mesh = MESHES[name]()
    d, E = mesh["d"], mesh["E"]
    nf = 2 * d
    faces = np.ascontiguousarray(mesh["faces"], dtype=np.int32)
    nbr = np.zeros(nf * E, dtype=np.int32)
    assert lib.frh_neighbours(E, nf, len(faces), _pi(faces), _pi(nbr)) == 0
    nbr = nbr.reshape(nf, E).T                       # [e][f]
    O = oracle.Oracle(mesh, w.Physics(mu=0.0, qinf=np.zeros(d + 2)), [1])
    assert np.array_equal(nbr, O.neighbours())
    col = np.zeros(E, dtype=np.int32)
    ncol = lib.frh_color2(E, nf, _pi(np.ascontiguousarray(nbr.T)), _pi(col))
    assert 0 < ncol == col.max() + 1
    adj = [set(int(n) for n in nbr[e] if n >= 0) for e in range(E)]
    for e in range(E):
        within2 = set(adj[e])
        for n in adj[e]:
            within2 |= adj[n]
        within2.discard(e)
        assert all(col[m] != col[e] for m in within2), (e, sorted(within2))
