"""World-size-2 gloo run (CPU) of the replica-sharded host logic used by
bench.py under torchrun: per-rank ensembles are distinct draws, the
whole-job figures are the sum of units and the max of the timed region, and
the measurements of one state point sampled on both ranks combine into the
measured equilibrium of the union of their windows."""

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
    # one state point's measurements on this rank: counts per class,
    # overflow, particle-windows, moment sums (synthetic, per-rank seed)
    import numpy as np

    rng = np.random.default_rng(100 + r)
    hist = rng.integers(0, 5000, 81)
    ovf = int(rng.integers(0, 50))
    samples = int(hist.sum()) + ovf
    mom = rng.uniform(0.5, 2.0, 2) * samples
    comb = sharding.combine_measurements(dist, hist, ovf, samples, mom)
    q.put((r, ws, local, units, tot, tmax, Ns.tolist(), (hist, ovf, samples, mom), comb))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, l0, u0, t0, m0, n0, own0, c0), (r1, ws1, l1, u1, t1, m1, n1, own1, c1) = res
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2 and (l0, l1) == (0, 1)
    assert n0 != n1                           # distinct ensembles per rank
    assert t0 == t1 == u0 + u1                # units summed over ranks
    assert m0 == m1 == 110.0                  # max of the timed region
    # combined measurements: exact integer sums, identical on both ranks
    import numpy as np

    H = own0[0] + own1[0]
    S = own0[2] + own1[2]
    for c in (c0, c1):
        assert np.array_equal(c[0], H) and c[1] == own0[1] + own1[1] and c[2] == S
        assert np.array_equal(c[4], H / S) and c[4].sum() + c[1] / S == pytest.approx(1.0, abs=1e-12)
        assert c[5] == (own0[3][0] + own1[3][0]) / (2 * S)
    assert np.array_equal(c0[3], c1[3])


def test_single_process_aggregate_is_identity():
    from paper_2101_01160_gb300 import sharding

    assert sharding.aggregate(None, 5.0, 2.0) == (5.0, 2.0)


def test_single_process_combine_is_normalisation():
    import numpy as np

    from paper_2101_01160_gb300 import sharding

    h = np.array([3, 5, 2], np.int64)
    out = sharding.combine_measurements(None, h, 1, 11, [4.0, 8.0])
    assert np.array_equal(out[0], h) and out[2] == 11 and np.array_equal(out[4], h / 11.0)
    assert out[5] == 4.0 / 22 and out[6] == 8.0 / 22
