"""Multi-rank host logic on CPU (gloo, world size 2): the interface exchange of a
distributed Q^T reproduces the assembled operator, the per-element dot of
Algorithm 1 sums to p^T A p across ranks, and the bench's whole-job time is the
maximum over ranks.  On the GPU the solves run as independent replicas, one per rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    from oracle.element import element_matrices
    from oracle.mesh import box_mesh
    from oracle.problems import BakeoffProblem
    from oracle.quadrature import bp_rule
    from paper_2004_06722_gb300.partition import build_plan, exchange_sum, partition_slabs
    from synth import uniform_pm1

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dims, N = (2, 2, 4), 3
    coords, l2g = box_mesh(*dims, N, 0.05)
    parts = partition_slabs(*dims, world)
    plan = build_plan([l2g[p] for p in parts])
    prob = BakeoffProblem(5, *dims, N, amp=0.05)
    u = uniform_pm1(5, np.arange(prob.n_global)) * prob.free
    idx = {int(g): i for i, g in enumerate(plan.nodes[rank])}
    partial = np.zeros(len(plan.nodes[rank]))
    rule = bp_rule(5, N)
    dot = 0.0
    for e in parts[rank]:
        A = element_matrices(coords[e], N, rule, want=("A",))["A"]
        ue = u[l2g[e]]
        we = A @ ue
        dot += float(ue @ we)
        for a, g in enumerate(l2g[e]):
            partial[idx[int(g)]] += we[a]
    full = exchange_sum(partial, rank, plan, dist)
    ref = prob.A @ u
    err = float(np.max(np.abs(full - ref[plan.nodes[rank]])) / np.max(np.abs(ref)))
    t = torch.tensor([dot], dtype=torch.float64)
    dist.all_reduce(t)
    dot_err = abs(float(t.item()) - float(u @ ref)) / abs(float(u @ ref))
    tmax = bench.max_over_ranks(1.0 + rank, world, dist, torch.device("cpu"))
    owned_total = torch.tensor([len(plan.owned[rank])], dtype=torch.int64)
    dist.all_reduce(owned_total)
    q.put((rank, err, dot_err, tmax, int(owned_total.item()), prob.n_global, len(plan.interface)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_exchange_matches_assembled_operator():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, dot_err, tmax, owned_total, n_global, n_if in out:
        assert err < 1e-13, (rank, err)
        assert dot_err < 1e-13
        assert tmax == 2.0                     # the slower rank's time
        assert owned_total == n_global          # every node owned exactly once
        assert n_if == (3 * 2 + 1) * (3 * 2 + 1)  # one shared node layer between the two z-slabs


def test_single_rank_plan():
    from oracle.mesh import box_mesh
    from paper_2004_06722_gb300.partition import build_plan, partition_slabs
    coords, l2g = box_mesh(2, 1, 3, 2, 0.0)
    parts = partition_slabs(2, 1, 3, 1)
    plan = build_plan([l2g[p] for p in parts])
    assert len(plan.interface) == 0 and len(plan.owned[0]) == len(plan.nodes[0])
    with pytest.raises(ValueError):
        partition_slabs(2, 1, 3, 4)
