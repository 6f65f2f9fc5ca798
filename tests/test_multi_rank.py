"""The multi-process path on the CPU (gloo, world size 2): every rank gets its own
problem (different seeds and orbitals, the same sizes), the job time is the
maximum over ranks, and the job throughput counts the units of all ranks. No
data-path collective exists; only this timing reduction crosses ranks."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_2208_07731_gb300 import ranks as R
    from paper_2208_07731_gb300 import workload as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, wsz, local = R.env()
    base = W.small_workload(n=6, L=5.0, n_orb=2, n_mu=4, iters=1, ecut=4.0, seed=3)
    w = R.rank_workload(base, r)
    phi, _ = W.make_pair(w)
    elapsed = 0.25 + 0.5 * r                     # a per-rank step time
    job = R.max_over_ranks(elapsed)
    sums = [None] * wsz
    dist.all_gather_object(sums, (w.seed, float(np.abs(phi.numpy()).sum())))
    out.put((r, wsz, local, w.n, w.n_mu, job, R.job_throughput(1, wsz, job), sums))
    dist.destroy_process_group()


def test_two_ranks_own_problems_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, n, n_mu, job, thr, sums) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert (n, n_mu) == (6, 4)                # same sizes on every rank
        assert job == 0.75                        # the slowest rank's time
        assert thr == 2 / 0.75                    # both ranks' units over the job time
        (s0, a0), (s1, a1) = sums
        assert s0 != s1 and a0 != a1              # independent problems


def test_single_process_defaults():
    from paper_2208_07731_gb300 import ranks as R
    assert R.max_over_ranks(1.5) == 1.5
    assert R.job_throughput(3, 1, 0.5) == 6.0
