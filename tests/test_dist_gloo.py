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


# One burst split into spatial tiles (plk_tile_plan) over two gloo ranks: each
# rank runs the oracle chain on its tiles' crops and keeps the owned parts; the
# stitched burst equals the oracle chain run on the whole burst at every step.
TILE_CASE = dict(H=40, W=66, win=(5, 11, 1, 1), tiles=(2, 3), T=20, M=10, K_max=2)


def _tile_worker(rank, world, port, tiles, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2511_12051_gb300 import synth
    c = TILE_CASE
    z = synth.generate(synth.config_spec(0, N=c["T"], H=c["H"], W=c["W"], seed=33)).numpy()
    mine = {}
    for i in pdist.shard(len(tiles), rank, world):
        sl = pdist.tile_slices(tiles[i])
        crop = np.ascontiguousarray(z[(slice(None),) + sl["crop"]])
        ch = oracle.OracleChain(crop.shape[1], crop.shape[2], c["win"], K_max=c["K_max"], kappa_dtype=np.complex64)
        steps = []
        for s in synth.ministack_slices(c["T"], c["M"]):
            o = ch.step(crop[s])
            steps.append((o["phase_real"][(Ellipsis,) + sl["cells"]], o["tcoh"][sl["cells"]],
                          ch.ring[-1][sl["pixels"]]))
        mine[i] = steps
    t = pdist.max_over_ranks(1.0 + rank)
    pdist.barrier()
    out.put((rank, t, mine))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_burst_into_tiles():
    from paper_2511_12051_gb300 import build, plk
    import oracle
    from paper_2511_12051_gb300 import synth
    build.build()
    c = TILE_CASE
    n_steps = len(synth.ministack_slices(c["T"], c["M"]))
    tiles = plk.tile_plan(c["H"], c["W"], c["win"], *c["tiles"], n_steps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, world = _free_port(), 2
    procs = [ctx.Process(target=_tile_worker, args=(r, world, port, tiles, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(t == float(world) for _, t, _ in res)
    got = {}
    for _, _, mine in res:
        got.update(mine)
    assert sorted(got) == list(range(len(tiles)))
    z = synth.generate(synth.config_spec(0, N=c["T"], H=c["H"], W=c["W"], seed=33)).numpy()
    ch = oracle.OracleChain(c["H"], c["W"], c["win"], K_max=c["K_max"], kappa_dtype=np.complex64)
    for s, sl_t in enumerate(synth.ministack_slices(c["T"], c["M"])):
        o = ch.step(z[sl_t])
        phase = np.full_like(o["phase_real"], np.inf)
        kappa = np.full_like(ch.ring[-1], np.inf)
        for i, t in enumerate(tiles):
            sl = pdist.tile_slices(t)
            ph, tc, ka = got[i][s]
            phase[(Ellipsis,) + sl["burst_cells"]] = ph
            assert np.array_equal(tc, o["tcoh"][sl["burst_cells"]], equal_nan=True)
            kappa[sl["burst_pixels"]] = ka
        assert np.array_equal(phase, o["phase_real"], equal_nan=True)
        assert np.array_equal(kappa, ch.ring[-1])
