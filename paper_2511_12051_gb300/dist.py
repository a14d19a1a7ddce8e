"""Multi-GPU plumbing for independent work units (bursts, stacks or spatial
tiles of one burst).

The phase-linking path shards without any data exchange: each rank processes
its own units and the only collectives are timing ones (a barrier and the
maximum of the per-rank times).  Works with NCCL on GPUs and gloo on CPU.
Spatial tiles come from plk_tile_plan (plk.tile_plan): each tile's crop holds
its owned cells' windows for the planned number of mini-stack steps, so a rank
runs an ordinary state on the crop and keeps the owned part.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_info() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous block of unit indices for `rank` (sizes differ by at most 1)."""
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def unit_seed(base_seed: int, unit: int) -> int:
    """Seed of work unit `unit`, independent of how units are spread over ranks."""
    return int(base_seed) + 7919 * int(unit)


def max_over_ranks(value: float, device: torch.device | str = "cpu") -> float:
    """Maximum of `value` over all ranks (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def tile_slices(t: dict) -> dict:
    """Index tuples of a plk_tile_plan tile: 'crop' (rows, columns of the burst
    the tile loads), 'cells' / 'burst_cells' (its owned output cells in the
    crop's and in the burst's output grid), 'pixels' / 'burst_pixels' (its owned
    full-resolution pixels in the crop and in the burst)."""
    return {
        "crop": (slice(t["y0"], t["y0"] + t["h"]), slice(t["x0"], t["x0"] + t["w"])),
        "cells": (slice(t["cy0"], t["cy0"] + t["oh"]), slice(t["cx0"], t["cx0"] + t["ow"])),
        "burst_cells": (slice(t["oy0"], t["oy0"] + t["oh"]), slice(t["ox0"], t["ox0"] + t["ow"])),
        "pixels": (slice(t["py0"] - t["y0"], t["py0"] - t["y0"] + t["ph"]),
                   slice(t["px0"] - t["x0"], t["px0"] - t["x0"] + t["pw"])),
        "burst_pixels": (slice(t["py0"], t["py0"] + t["ph"]), slice(t["px0"], t["px0"] + t["pw"])),
    }
