"""The multi-GPU form of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank runs its own integral (Philox counter word 3 = rank: independent
samples, no data exchange); the job's time is the slowest rank's and its
evaluations are all ranks' (bench.reduce_over_ranks).  Checked here with the
oracle standing in for the GPU path: the ranks' first samples differ, and the
reduction returns the maximum time and the summed evaluations on every rank.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    import oracle
    from paper_2009_05112_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = bench.rank_problem(inputs.three_peaks_d4(n_ev=1000, n_g=50), rank)
    o = oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                         alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                         prm=prob.prm, integral_id=prob.integral_id)
    x, _, _, _ = o.eval_sample(0, 0, 0)
    o.iterate()
    evals = int(o.offsets[-1])
    total_ms = 10.0 * (rank + 1)  # a stand-in for the rank's device time
    t_max, e_all = bench.reduce_over_ranks(total_ms, evals, dist, "cpu")
    out.put((rank, list(x), evals, t_max, e_all, prob.integral_id))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    (r0, x0, e0, t0, a0, id0), (r1, x1, e1, t1, a1, id1) = got
    assert (id0, id1) == (0, 1)
    assert x0 != x1                       # independent Philox streams
    assert t0 == t1 == 20.0               # the slowest rank's time, on every rank
    assert a0 == a1 == float(e0 + e1)     # all ranks' evaluations
