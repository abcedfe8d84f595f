"""Distributed training of one decomposition over several ranks (one GPU
each), as Algorithm 1 runs it over processes: every rank trains its own
subdomains, and the values at the interfaces it shares with other ranks are
exchanged once per step (the paper's Isend / Irecv of interface values).

    part = partition(pb, world)                    # xpinn_partition
    ds = DistSolver(pb, part, rank, transport)     # the rank's handle
    losses = ds.step()                              # begin, exchange, end

The library does every computation; this module only cuts the problem
description by rank and moves the exchanged rows between ranks:
TorchTransport sends them with torch.distributed (NCCL for CUDA tensors, gloo
for host tensors); the rows are the other side's solution vector and
exchanged quantity (flux or residual) at the interface points, exactly what
the single-GPU step reads from its own exchange buffer.  No kernel is ever
given another rank's memory and there is no collective: only point-to-point
messages between ranks that share an interface.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import problems as P


def partition(pb: P.Problem, n_parts: int) -> np.ndarray:
    """part[q] in [0, n_parts): subdomains to ranks, balancing the points
    (residual, data and interface points of each subdomain) and cutting few
    interface points (xpinn_partition)."""
    from . import xpinn as X
    lib = X.load()
    w = np.zeros(pb.n_sub, np.float64)
    for q, sd in enumerate(pb.subs):
        w[q] = sd.res_xy.shape[0] + sum(d.xy.shape[0] for d in sd.data if d is not None)
    eq = np.array([it.q for it in pb.ifaces], np.int32)
    eqp = np.array([it.qp for it in pb.ifaces], np.int32)
    ew = np.array([it.xy.shape[0] for it in pb.ifaces], np.float64)
    for it in pb.ifaces:
        w[it.q] += it.xy.shape[0]
        w[it.qp] += it.xy.shape[0]
    part = np.zeros(pb.n_sub, np.int32)
    X._check(lib.xpinn_partition(pb.n_sub, w.ctypes.data, len(eq), eq.ctypes.data if len(eq) else None,
                                 eqp.ctypes.data if len(eq) else None, ew.ctypes.data if len(eq) else None,
                                 n_parts, part.ctypes.data))
    return part


@dataclasses.dataclass
class RankPlan:
    """One rank's part of the decomposition."""
    problem: P.Problem        # its subdomains and interfaces (remote ones marked)
    local: list               # handle subdomain i is global subdomain local[i]
    remote: list              # per remote interface, in the problem's order: (global interface, peer rank, points)
    nv: int                   # floats per point and side in the exchanged rows


def rank_problem(pb: P.Problem, part, rank: int) -> RankPlan:
    """The description of rank `rank`'s subdomains.  An interface with both
    sides on the rank keeps both (renumbered); one with a single side there
    keeps that side as q and is marked remote; the others are dropped.
    Interfaces keep the global order, so two ranks list the interfaces they
    share in the same order."""
    part = np.asarray(part)
    local = [q for q in range(pb.n_sub) if part[q] == rank]
    if not local:
        raise ValueError(f"rank {rank} has no subdomain")
    idx = {q: i for i, q in enumerate(local)}
    ifaces, remote = [], []
    for e, it in enumerate(pb.ifaces):
        a, b = part[it.q] == rank, part[it.qp] == rank
        if a and b:
            ifaces.append(dataclasses.replace(it, q=idx[it.q], qp=idx[it.qp], remote=False))
        elif a or b:
            mine, other = (it.q, it.qp) if a else (it.qp, it.q)
            ifaces.append(dataclasses.replace(it, q=idx[mine], qp=0, remote=True))
            remote.append((e, int(part[other]), int(it.xy.shape[0])))
    prob = dataclasses.replace(pb, name=f"{pb.name}_rank{rank}", subs=[pb.subs[q] for q in local], ifaces=ifaces,
                               subs_per_model=0)
    n_out = sum(n.widths[-1] for n in pb.subs[0].nets)
    nv = n_out + (3 if pb.pde == P.PDE_NS else 1)
    return RankPlan(prob, local, remote, nv)


def exchange_plan(plan: RankPlan):
    """Per peer rank, the slices of the packed remote-values vector (in the
    rank problem's interface order) that go to it and come back from it, in
    global interface order (the same order on both ranks)."""
    out, off = {}, 0
    for e, peer, n in plan.remote:
        out.setdefault(peer, []).append((e, off, off + n * plan.nv))
        off += n * plan.nv
    return out, off


class TorchTransport:
    """Point-to-point exchange of the interface rows with torch.distributed:
    every pair of ranks sharing interfaces swaps one message each way per
    step, posted as non-blocking sends and receives."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def exchange(self, plan: RankPlan, send):
        """send: this rank's packed remote values (CPU or CUDA tensor).
        Returns the tensor of the other sides' values, packed the same way."""
        import torch
        peers, total = exchange_plan(plan)
        recv = torch.empty_like(send)
        ops, bufs = [], []
        for peer in sorted(peers):
            sl = peers[peer]
            s_buf = torch.cat([send[a:b] for _, a, b in sl]).contiguous()
            r_buf = torch.empty_like(s_buf)
            bufs.append((sl, r_buf))
            ops.append(self.dist.isend(s_buf, peer, group=self.group))
            ops.append(self.dist.irecv(r_buf, peer, group=self.group))
        for op in ops:
            op.wait()
        for sl, r_buf in bufs:
            o = 0
            for _, a, b in sl:
                recv[a:b] = r_buf[o:o + (b - a)]
                o += b - a
        return recv


class DistSolver:
    """One rank's handle of a distributed decomposition: step() runs a
    training step of Algorithm 1 with the exchange of interface values
    between ranks in the middle."""

    def __init__(self, pb: P.Problem, part, rank: int, transport, device_exchange=True):
        from . import xpinn as X
        self.plan = rank_problem(pb, part, rank)
        self.solver = X.Solver(self.plan.problem)
        self.transport = transport
        self.device_exchange = device_exchange
        _, self.n_remote = exchange_plan(self.plan)

    def step(self, losses=None):
        import torch
        s = self.solver
        s.step_begin()
        if self.n_remote:
            if self.device_exchange:
                send = torch.empty(self.n_remote, dtype=torch.float32, device="cuda")
                s.remote_values(send)
                torch.cuda.synchronize()
            else:
                send = torch.from_numpy(s.remote_values())
            recv = self.transport.exchange(self.plan, send)
            s.set_remote_values(recv)
        if losses is None:
            losses = np.empty((s.n_sub, P.N_TERMS), np.float32)
        s.step_end(losses)
        return losses

    def close(self):
        self.solver.close()
