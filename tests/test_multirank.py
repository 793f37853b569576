"""World-size-2 gloo run (CPU) of the replica-sharded host logic used by
bench.py under torchrun: per-rank ensembles are distinct draws, and the
whole-job figures are the sum of units and the max of the timed region."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2101_01160_gb300 import inputs, sharding

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = sharding.world()
    Ns, phis, Ts = inputs.ensemble_params(16, seed=7 + sharding.seed_offset(r))
    units = float(Ns.sum()) * 400            # this rank's particle-steps
    ms = 100.0 + 10.0 * r                    # this rank's timed region
    tot, tmax = sharding.aggregate(dist, units, ms)
    q.put((r, ws, local, units, tot, tmax, Ns.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, l0, u0, t0, m0, n0), (r1, ws1, l1, u1, t1, m1, n1) = res
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2 and (l0, l1) == (0, 1)
    assert n0 != n1                           # distinct ensembles per rank
    assert t0 == t1 == u0 + u1                # units summed over ranks
    assert m0 == m1 == 110.0                  # max of the timed region


def test_single_process_aggregate_is_identity():
    from paper_2101_01160_gb300 import sharding

    assert sharding.aggregate(None, 5.0, 2.0) == (5.0, 2.0)
