"""The N>1 path on CPU: two gloo ranks shard independent units and agree on
the maximum per-rank time; each rank's oracle result on its own units equals a
single-process run over all units (the path needs no data exchange)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2511_12051_gb300 import dist as pdist


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            seen = [u for r in range(world) for u in pdist.shard(n, r, world)]
            assert seen == list(range(n))
            sizes = [len(pdist.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_units, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2511_12051_gb300 import synth
    phases = {}
    for u in pdist.shard(n_units, rank, world):
        spec = synth.config_spec(0, H=12, W=14, seed=pdist.unit_seed(5, u))
        ch = oracle.OracleChain(12, 14, (3, 5, 1, 1), K_max=2)
        phases[u] = ch.step(synth.generate(spec).numpy())["phase_real"]
    t = pdist.max_over_ranks(10.0 + rank)
    pdist.barrier()
    out.put((rank, t, phases))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, world, n_units = _free_port(), 2, 5
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_units, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(t == 10.0 + world - 1 for _, t, _ in res)
    merged = {}
    for _, _, ph in res:
        merged.update(ph)
    assert sorted(merged) == list(range(n_units))
    import oracle
    from paper_2511_12051_gb300 import synth
    for u in range(n_units):
        spec = synth.config_spec(0, H=12, W=14, seed=pdist.unit_seed(5, u))
        ch = oracle.OracleChain(12, 14, (3, 5, 1, 1), K_max=2)
        want = ch.step(synth.generate(spec).numpy())["phase_real"]
        assert np.array_equal(merged[u], want)
