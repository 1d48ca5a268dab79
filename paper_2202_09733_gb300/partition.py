"""Element partition of one mesh across processes (one GPU each).

The residual couples an element only to the elements across its faces, so a process that
holds its owned elements plus one layer of ghost copies (every element sharing a face
with an owned one) evaluates the owned part of R exactly, provided the ghosts carry
their owners' current states.  Everything element-local (element blocks, LU, transfers,
the updates) needs no data from other processes; inner products need one sum over
processes.  This module builds, on the host:

  partition(mesh, nparts)        owner rank of every element: recursive coordinate
                                 bisection of the element centroids (deterministic)
  local_problem(mesh, owner, r)  rank r's mesh: owned elements (ascending global id),
                                 then ghosts grouped by owner rank (ascending global id
                                 within a rank); faces between local elements keep their
                                 orientation; a ghost's face towards a non-local element
                                 becomes a far-field face (it changes only that ghost's
                                 own residual, which nothing reads)
  exchange_plan(...)             per rank: the owned elements to send to each peer, in
                                 the order the peer stores its ghosts, and the ghost
                                 counts received from each peer
"""
from __future__ import annotations

import numpy as np


def element_centroids(mesh: dict) -> np.ndarray:
    return np.asarray(mesh["gnodes"], dtype=np.float64).mean(axis=1)


def partition(mesh: dict, nparts: int) -> np.ndarray:
    """owner[e] in 0..nparts-1; part sizes differ by at most one element per bisection."""
    E = mesh["E"]
    if nparts < 1 or nparts > E:
        raise ValueError(f"cannot split {E} elements into {nparts} parts")
    c = element_centroids(mesh)
    owner = np.zeros(E, dtype=np.int32)

    def rcb(idx, parts, base):
        if parts == 1:
            owner[idx] = base
            return
        ext = c[idx].max(axis=0) - c[idx].min(axis=0)
        ax = int(np.argmax(ext))
        order = idx[np.lexsort((idx, c[idx, ax]))]     # by coordinate, ties by element id
        k = parts // 2
        n0 = (len(idx) * k + parts // 2) // parts
        rcb(order[:n0], k, base)
        rcb(order[n0:], parts - k, base + k)

    rcb(np.arange(E), nparts, 0)
    return owner


def local_problem(mesh: dict, owner: np.ndarray, rank: int) -> dict:
    """rank's local mesh with its owned elements and one ghost layer (see module doc)."""
    faces = np.asarray(mesh["faces"], dtype=np.int64)
    owned = np.flatnonzero(owner == rank)
    if len(owned) == 0:
        raise ValueError(f"rank {rank} owns no element")
    is_owned = owner == rank
    interior = faces[:, 2] >= 0
    eL, eR = faces[:, 0], faces[:, 2]
    g1 = eR[interior & is_owned[eL] & ~is_owned[np.where(eR >= 0, eR, 0)]]
    g2 = eL[interior & is_owned[np.where(eR >= 0, eR, 0)] & ~is_owned[eL]]
    ghosts = np.unique(np.concatenate([g1, g2]))
    ghosts = ghosts[np.lexsort((ghosts, owner[ghosts]))]          # grouped by owner rank
    local = np.concatenate([owned, ghosts]).astype(np.int64)
    g2l = np.full(mesh["E"], -1, dtype=np.int64)
    g2l[local] = np.arange(len(local))
    rows = []
    for f in faces:
        a, fa, b, fb, orient, bc = (int(x) for x in f)
        la = g2l[a]
        lb = g2l[b] if b >= 0 else -1
        if b < 0:
            if la >= 0:
                rows.append((la, fa, -1, -1, 0, bc))
        elif la >= 0 and lb >= 0:
            rows.append((la, fa, lb, fb, orient, bc))
        elif la >= 0:
            rows.append((la, fa, -1, -1, 0, 1))      # ghost a's face towards a non-local element
        elif lb >= 0:
            rows.append((lb, fb, -1, -1, 0, 1))
    m = dict(mesh)
    m["E"] = int(len(local))
    m["gnodes"] = np.ascontiguousarray(np.asarray(mesh["gnodes"])[local])
    m["faces"] = np.array(rows, dtype=np.int32).reshape(-1, 6)
    m["kind"] = f"{mesh.get('kind', 'mesh')} part {rank}"
    return dict(mesh=m, local=local, owned=owned, ghosts=ghosts, n_owned=int(len(owned)),
                ghost_owner=owner[ghosts].astype(np.int32))


def exchange_plan(owner: np.ndarray, locals_: list) -> list:
    """Per rank r: send[p] = r's local indices of the owned elements that rank p holds as
    ghosts, in p's ghost order; recv_counts[p] = ghosts of r owned by p (contiguous in r's
    ghost range, peers ascending)."""
    nranks = len(locals_)
    pos = []                                  # global id -> local index on its owner
    for r in range(nranks):
        d = np.full(len(owner), -1, dtype=np.int64)
        d[locals_[r]["owned"]] = np.arange(locals_[r]["n_owned"])
        pos.append(d)
    plans = []
    for r in range(nranks):
        send = []
        for p in range(nranks):
            if p == r:
                send.append(np.zeros(0, dtype=np.int32))
                continue
            gp = locals_[p]["ghosts"][locals_[p]["ghost_owner"] == r]
            send.append(pos[r][gp].astype(np.int32))
        recv_counts = [int(np.sum(locals_[r]["ghost_owner"] == p)) for p in range(nranks)]
        plans.append(dict(send=send, send_counts=[len(x) for x in send], recv_counts=recv_counts))
    return plans


def scatter_state(q: np.ndarray, loc: dict) -> np.ndarray:
    """The local [nv][Np][E_local] state (owned and ghost elements) of a global state."""
    return np.ascontiguousarray(np.asarray(q)[:, :, loc["local"]])


def owned_part(x_local, loc: dict):
    return x_local[:, :, :loc["n_owned"]]


def pack_owned(x: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """The exchange layout of the library's ghost exchange: element by element (slot-major),
    each element's nv Np values in [v][i] order, as raw bytes."""
    return np.ascontiguousarray(np.transpose(np.asarray(x)[:, :, idx], (2, 0, 1))).view(np.uint8).ravel()


def unpack_ghosts(x: np.ndarray, buf: np.ndarray, n_owned: int) -> None:
    """Write the received elements (exchange layout) into x's ghost elements, in place."""
    nv, npt, E = x.shape
    vals = np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=x.dtype).reshape(E - n_owned, nv, npt)
    x[:, :, n_owned:] = np.transpose(vals, (1, 2, 0))
