"""Partitioned single-mesh RHS: one part of the mesh per GPU, two halo exchanges per RHS.

The fused RHS needs neighbour data only at the boundaries of the paper's kernel groups (Sec. 2.2
and its kernel-grouping figure): the face solution U^(f) before con_u, and the face data of
comm_flux (the own-normal viscous flux; in the low-Mach form also the float-float mass flux) before
it. Part r of nparts owns a contiguous range of the global element order; the library packs the
face data its peers need into a send buffer and unpacks theirs into its halo slots
(fr_halo_pack / fr_halo_unpack). This module only moves those buffers between parts:

* ``dist_exchange``: one rank per part over torch.distributed (NCCL on CUDA tensors, gloo on CPU
  tensors) with paired send/recv per peer;
* ``local_exchange``: several parts in one process (device-to-device copies), for tests on one GPU.

Buffer layout (the library's): peer by peer in increasing rank, nvar x count values, var-major.
"""
from __future__ import annotations

from typing import Callable, Sequence


def segments(counts: Sequence[int], nvar: int, part: int):
    """(peer, first value, number of values) of every non-empty peer segment of a halo buffer."""
    out, off = [], 0
    for q, c in enumerate(counts):
        if q != part and c > 0:
            out.append((q, nvar * off, nvar * c))
        off += c
    return out


def dist_exchange(send, recv, counts: Sequence[int], nvar: int, part: int, group=None) -> None:
    """Sends the segment of peer q of `send` to rank q and receives rank q's segment for this part
    into the same place of `recv`, for every peer, over the default (or given) process group."""
    import torch.distributed as dist
    ops = []
    for q, s, n in segments(counts, nvar, part):
        ops.append(dist.P2POp(dist.isend, send[s:s + n], q, group))
        ops.append(dist.P2POp(dist.irecv, recv[s:s + n], q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def local_exchange(sends: Sequence, recvs: Sequence, counts: Sequence[Sequence[int]], nvar: int) -> None:
    """Exchange between parts held in one process: part r's segment for peer q receives part q's
    segment for peer r (counts[r] is part r's per-peer count list)."""
    seg = [{q: (s, n) for q, s, n in segments(counts[r], nvar, r)} for r in range(len(sends))]
    for r in range(len(sends)):
        for q, (s, n) in seg[r].items():
            a, b = seg[q][r]
            assert b == n, "peers disagree on the number of exchanged points"
            recvs[r][s:s + n].copy_(sends[q][a:a + b])


class PartRHS:
    """Halo buffers of one part and its RHS as phases with exchanges between them."""

    def __init__(self, mesh_handle, device=None):
        import torch
        self.m = mesh_handle
        info = mesh_handle.halo_info()
        self.part, self.nparts = info["part"], info["nparts"]
        self.counts = info["counts"]
        self.nvar = info["nvar"]
        nh = sum(self.counts)
        dt = mesh_handle.dtype
        dev = device if device is not None else "cuda"
        self.send = [torch.zeros(max(1, v * nh), dtype=dt, device=dev) for v in self.nvar]
        self.recv = [torch.zeros(max(1, v * nh), dtype=dt, device=dev) for v in self.nvar]

    def rhs(self, U, R, exchange: Callable[[int], None], stream=None) -> None:
        """R = R(U) on this part: phase A, exchange 0, phase B, exchange 1, phase C. `exchange(what)`
        moves this part's send[what] to its peers and their data into recv[what]."""
        m = self.m
        m.rhs_phase(0, U, R, stream)
        m.halo_pack(0, self.send[0], stream)
        exchange(0)
        m.halo_unpack(0, self.recv[0], stream)
        m.rhs_phase(1, U, R, stream)
        m.halo_pack(1, self.send[1], stream)
        exchange(1)
        m.halo_unpack(1, self.recv[1], stream)
        m.rhs_phase(2, U, R, stream)

    def rk4_step(self, U, dt: float, exchange: Callable[[int], None], stream=None) -> None:
        """One classical RK4 step of this part's FP64 master state U: per stage phase A, exchange 0,
        phase B, exchange 1, phase C with the stage update (fr_rk4_stage)."""
        m = self.m
        for st in range(4):
            m.rk4_stage(st, 0, U, dt, stream)
            m.halo_pack(0, self.send[0], stream)
            exchange(0)
            m.halo_unpack(0, self.recv[0], stream)
            m.rk4_stage(st, 1, U, dt, stream)
            m.halo_pack(1, self.send[1], stream)
            exchange(1)
            m.halo_unpack(1, self.recv[1], stream)
            m.rk4_stage(st, 2, U, dt, stream)
