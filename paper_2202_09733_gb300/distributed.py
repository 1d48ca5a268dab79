"""Element-partitioned solves: one process (one GPU) per part of the mesh.

Each process creates its context on its local mesh (owned elements, then one ghost layer;
partition.local_problem) and registers a communicator (fr_set_comm).  The library then
asks, before every residual evaluation, for the ghosts' current values (it packs the
owned elements that other processes hold as ghosts into send_buf and unpacks recv_buf
into its ghosts), and sums every inner product over the processes.  This module supplies
the two callbacks over a transport:

  TorchDistTransport   torch.distributed (NCCL between GPUs, gloo on the host): batched
                       point-to-point sends and receives of each peer's chunk, all_reduce
  LoopbackGroup        all ranks inside one process, one host thread each: the chunks
                       are copied device to device between the ranks' buffers after a
                       host barrier (no kernel waits on another)

and PartitionedContext, which owns the local context, the exchange buffers and the
callbacks.  Data movement only: every arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import threading
import traceback

import numpy as np
import torch

from . import api, partition as PT, _native as N


class TorchDistTransport:
    """Exchange and reductions over the default torch.distributed process group."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()
        self.backend = dist.get_backend()

    def exchange(self, send, recv, send_bytes, recv_bytes):
        """send / recv: uint8 tensors; chunk p of send goes to rank p, chunk p of recv comes
        from rank p (byte counts per rank)."""
        ops, so, ro = [], 0, 0
        for p in range(self.size):
            if recv_bytes[p]:
                ops.append(self.dist.P2POp(self.dist.irecv, recv[ro:ro + recv_bytes[p]], p))
            ro += recv_bytes[p]
        for p in range(self.size):
            if send_bytes[p]:
                ops.append(self.dist.P2POp(self.dist.isend, send[so:so + send_bytes[p]], p))
            so += send_bytes[p]
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        if send.is_cuda:
            torch.cuda.synchronize()

    def allreduce(self, arr: np.ndarray, op: int):
        t = torch.from_numpy(arr.copy())
        if self.backend == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM if op == 0 else self.dist.ReduceOp.MAX)
        arr[:] = t.cpu().numpy()


class LoopbackGroup:
    """nranks ranks in one process (one host thread each) sharing one device."""

    def __init__(self, nranks: int, timeout: float = 120.0):
        self.n = nranks
        self.bar = threading.Barrier(nranks, timeout=timeout)
        self.slots = [None] * nranks

    def transport(self, rank: int):
        return _LoopbackTransport(self, rank)


class _LoopbackTransport:
    def __init__(self, group: LoopbackGroup, rank: int):
        self.g, self.rank, self.size = group, rank, group.n

    def exchange(self, send, recv, send_bytes, recv_bytes):
        g, r = self.g, self.rank
        g.slots[r] = (send, list(send_bytes))
        g.bar.wait()
        ro = 0
        for p in range(self.size):
            n = recv_bytes[p]
            if n:
                psend, pcounts = g.slots[p]
                off = sum(pcounts[:r])
                if pcounts[r] != n:
                    raise RuntimeError(f"rank {r} expects {n} bytes from {p}, which sends {pcounts[r]}")
                recv[ro:ro + n].copy_(psend[off:off + n])
            ro += n
        torch.cuda.synchronize()
        g.bar.wait()

    def allreduce(self, arr: np.ndarray, op: int):
        g = self.g
        g.slots[self.rank] = arr.copy()
        g.bar.wait()
        vals = np.stack(g.slots[:self.size])
        out = vals.sum(axis=0) if op == 0 else vals.max(axis=0)
        g.bar.wait()
        arr[:] = out


class PartitionedContext:
    """The local context of `rank` for a mesh split into `nranks` parts, with its
    communicator registered.  .ctx is an api.Context usable with every api call; states
    are local [nv][Np][E_local] tensors (owned elements first)."""

    def __init__(self, mesh: dict, phys, levels, rank: int, nranks: int, transport, owner=None):
        self.rank, self.nranks = rank, nranks
        self.owner = PT.partition(mesh, nranks) if owner is None else np.asarray(owner)
        self.locals = [PT.local_problem(mesh, self.owner, r) for r in range(nranks)]
        self.plan = PT.exchange_plan(self.owner, self.locals)[rank]
        self.loc = self.locals[rank]
        self.ctx = api.fr_create(self.loc["mesh"], phys, levels)
        d = mesh["d"]
        nv, np0 = d + 2, (levels[0] + 1) ** d
        eb = nv * np0 * 8
        self.n_owned = self.loc["n_owned"]
        nsend = int(sum(self.plan["send_counts"]))
        nrecv = self.loc["mesh"]["E"] - self.n_owned
        self.send_buf = torch.empty(max(1, nsend) * eb, dtype=torch.uint8, device="cuda")
        self.recv_buf = torch.empty(max(1, nrecv) * eb, dtype=torch.uint8, device="cuda")
        self.send_idx = np.ascontiguousarray(
            np.concatenate(self.plan["send"]) if nsend else np.zeros(1), dtype=np.int32)
        self.transport = transport
        self.error = None
        sc, rc = self.plan["send_counts"], self.plan["recv_counts"]

        def halo(user, level, precision, elem_bytes, stream):
            try:
                self.transport.exchange(self.send_buf, self.recv_buf, [c * elem_bytes for c in sc],
                                        [c * elem_bytes for c in rc])
                return 0
            except Exception:                                   # reported through the status code
                self.error = traceback.format_exc()
                return -1

        def allreduce(user, buf, n, op):
            try:
                arr = np.ctypeslib.as_array(buf, shape=(n,))
                self.transport.allreduce(arr, op)
                return 0
            except Exception:
                self.error = traceback.format_exc()
                return -1

        self._cb = (N.HaloFn(halo), N.AllreduceFn(allreduce))   # kept alive with the context
        comm = N.Comm(self.n_owned, int(mesh["E"]), nsend, self.send_idx.ctypes.data_as(N.PI), C.c_void_p(self.send_buf.data_ptr()),
                      C.c_void_p(self.recv_buf.data_ptr()), self._cb[0], self._cb[1], None)
        N.check(N.load().fr_set_comm(self.ctx.handle, C.byref(comm)), "fr_set_comm")

    def local_state(self, q_global) -> torch.Tensor:
        return torch.from_numpy(PT.scatter_state(np.asarray(q_global), self.loc)).cuda()

    def owned(self, x):
        return x[:, :, :self.n_owned]
