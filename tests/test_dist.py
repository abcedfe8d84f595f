"""Distributed training across ranks (Algorithm 1's exchange of interface
values between processes):

* the partitioner balances the points and cuts few interface points on the
  workloads' grids (CPU, the library's host code);
* every rank's description keeps its own subdomains, and an interface shared
  by two ranks appears on both, with the same points, marked remote (CPU);
* two gloo ranks exchange the packed interface rows through the transport
  the distributed solver uses, each receiving exactly the other's rows for
  the interfaces they share (CPU, world size 2);
* two ranks run in one process on one GPU, their rows swapped through the
  host: every loss term and every parameter after a training step equals the
  single-handle step on the whole decomposition within the parity tolerances
  (the same arithmetic, items cut and summed in other orders).
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2104_10013_gb300 import dist as D
from paper_2104_10013_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cut_and_balance(pb, part, n_parts):
    cut = sum(it.xy.shape[0] for it in pb.ifaces if part[it.q] != part[it.qp])
    w = np.zeros(n_parts)
    for q, sd in enumerate(pb.subs):
        w[part[q]] += sd.res_xy.shape[0]
    return cut, w


@pytest.fixture(scope="module")
def built():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()


@pytest.mark.parametrize("n_parts", [2, 4, 8])
def test_partition_of_the_kovasznay_grid(built, n_parts):
    """8 x 8 equal subdomains: parts within 10% of an even share; the cut is
    that of straight cuts into equal blocks (the minimum for parts of equal
    size: every part of 64 / n cells has a perimeter of at least that of the
    most compact block)."""
    pb = P.kovasznay_cpinn(n_res=100, n_iface=8, n_bc=4)
    part = D.partition(pb, n_parts)
    assert sorted(set(part.tolist())) == list(range(n_parts))
    cut, w = cut_and_balance(pb, part, n_parts)
    assert w.max() <= 1.1 * w.mean() + 1e-9
    # straight cuts: 2 parts -> 8 interfaces, 4 -> 16, 8 -> 32 (blocks of 4 x 2), 8 points each
    ideal = {2: 8, 4: 16, 8: 32}[n_parts] * 8
    assert cut <= ideal, (cut, ideal)


def test_partition_of_the_uneven_poisson_grid(built):
    pb = P.poisson_xpinn()
    part = D.partition(pb, 4)
    cut, w = cut_and_balance(pb, part, 4)
    total_iface = sum(it.xy.shape[0] for it in pb.ifaces)
    assert sorted(set(part.tolist())) == [0, 1, 2, 3]
    assert cut < 0.6 * total_iface
    assert np.array_equal(part, D.partition(pb, 4))            # deterministic


def test_rank_problems_cover_the_decomposition(built):
    pb = P.poisson_xpinn(n_res_range=(300, 600), n_iface=16, n_bc=10)
    part = D.partition(pb, 3)
    plans = [D.rank_problem(pb, part, r) for r in range(3)]
    assert sorted(q for p in plans for q in p.local) == list(range(pb.n_sub))
    for e, it in enumerate(pb.ifaces):
        ra, rb = part[it.q], part[it.qp]
        if ra == rb:
            assert sum(1 for p in plans for f in p.problem.ifaces if not f.remote
                       and f.xy is it.xy) == 1
        else:
            for r, peer in ((ra, rb), (rb, ra)):
                assert (e, peer, it.xy.shape[0]) in plans[r].remote
                f = [f for f in plans[r].problem.ifaces if f.xy is it.xy]
                assert len(f) == 1 and f[0].remote


def _gloo_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2104_10013_gb300 import dist as Dm
    from paper_2104_10013_gb300 import problems as Pm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        pb = Pm.poisson_xpinn(n_res_range=(300, 600), n_iface=16, n_bc=10)
        part = np.array([0] * 8 + [1] * 8, np.int32)                 # a fixed split: no library needed here
        plan = Dm.rank_problem(pb, part, rank)
        _, n = Dm.exchange_plan(plan)
        # this rank's "side" of interface e, point i, float j: 1000 e + 10 i + j + 0.5 rank
        send = torch.zeros(n)
        off = 0
        for e, peer, npts in plan.remote:
            for i in range(npts):
                for j in range(plan.nv):
                    send[off + i * plan.nv + j] = 1000 * e + 10 * i + j + 0.5 * rank
            off += npts * plan.nv
        recv = Dm.TorchTransport().exchange(plan, send)
        ok = True
        off = 0
        for e, peer, npts in plan.remote:
            for i in range(npts):
                for j in range(plan.nv):
                    ok &= float(recv[off + i * plan.nv + j]) == 1000 * e + 10 * i + j + 0.5 * peer
            off += npts * plan.nv
        q.put((rank, ok, n))
    finally:
        dist.destroy_process_group()


def test_gloo_exchange_swaps_each_ranks_rows():
    import multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in res) and all(n > 0 for _, _, n in res)


class _InProcess:
    """The exchange of two ranks living in one process (test only)."""

    def __init__(self, plans, sends):
        self.plans, self.sends = plans, sends

    def recv_for(self, rank):
        plan = self.plans[rank]
        out = np.empty_like(self.sends[rank])
        off = 0
        for e, peer, n in plan.remote:
            pp = self.plans[peer]
            po = 0
            for e2, _, n2 in pp.remote:
                if e2 == e:
                    break
                po += n2 * pp.nv
            out[off:off + n * plan.nv] = self.sends[peer][po:po + n * plan.nv]
            off += n * plan.nv
        return out


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["poisson_xpinn", "kovasznay_cpinn"])
def test_two_ranks_on_one_gpu_match_the_single_handle_step(built, name):
    from paper_2104_10013_gb300 import xpinn as X
    from tests.test_parity import RTOL_JET, assert_scaled
    pb = {"poisson_xpinn": lambda: P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40),
          "kovasznay_cpinn": lambda: P.kovasznay_cpinn(nx=3, ny=3, n_res=1500, n_iface=96, n_bc=80)}[name]()
    part = D.partition(pb, 2)
    plans = [D.rank_problem(pb, part, r) for r in range(2)]
    solvers = [X.Solver(p.problem) for p in plans]
    whole = X.Solver(pb)
    for step in range(2):
        ref = whole.step(1)[0]
        for s in solvers:
            s.step_begin()
        sends = [s.remote_values() for s in solvers]
        ex = _InProcess(plans, sends)
        for r, s in enumerate(solvers):
            s.set_remote_values(ex.recv_for(r))
        got = np.zeros_like(ref)
        for r, s in enumerate(solvers):
            l = np.empty((s.n_sub, P.N_TERMS), np.float32)
            s.step_end(l)
            got[plans[r].local] = l
        assert_scaled(got, ref, RTOL_JET if step == 0 else 1e-4, f"{name} step {step} losses", axis=0)
    th = whole.get_params()
    offs = np.cumsum([0] + [sd.n_params for sd in pb.subs])
    for r, s in enumerate(solvers):
        mine = np.concatenate([th[offs[q]:offs[q + 1]] for q in plans[r].local])
        start = np.concatenate([pb.packed_params()[offs[q]:offs[q + 1]] for q in plans[r].local])
        assert np.linalg.norm(s.get_params() - mine) <= 1e-3 * np.linalg.norm(mine - start)
    for s in solvers + [whole]:
        s.close()
