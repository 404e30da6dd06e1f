"""Row-block partition of the tile triangle, checked with CPU ranks (gloo,
world size 2 and 3): the ranks' ranges tile the triangle exactly, the work is
balanced, and the ranks' oracle pieces reassemble the full matrix."""
import os
import socket

import numpy as np
import pytest

from paper_1410_4803_gb300 import partition


def test_default_tile_is_the_tensor_core_block():
    assert partition.TILE == 128 and partition.TILE_POPC == 64
    # a rank boundary falls on a 128-sample block edge
    for world in (2, 3, 8):
        for rank in range(world):
            r0, r1 = partition.pair_rows(20000, rank, world)
            assert r0 % 128 == 0 and (r1 % 128 == 0 or r1 == 20000)


@pytest.mark.parametrize("n", [1, 63, 64, 65, 127, 128, 129, 500, 4096, 20000])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("tile", [partition.TILE, partition.TILE_POPC])
def test_ranges_cover_triangle(n, world, tile):
    T = partition.n_tiles(n, tile)
    ranges = partition.partition_tiles(n, world, tile)
    assert ranges[0][0] == 0 and ranges[-1][1] == T * (T + 1) // 2
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    work = [b - a for a, b in ranges]
    if T >= 4 * world:
        # contiguous whole rows: each boundary is within half a row of its target
        total = T * (T + 1) // 2
        assert max(abs(w - total / world) for w in work) <= T


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, m, seed, q):
    import torch
    import torch.distributed as dist

    import oracle
    from helpers import pack_codes, random_codes
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(seed)
    codes = random_codes(rng, n, m)
    packed = pack_codes(codes)
    G = oracle.unpack(packed, n, m)
    r0, r1 = partition.pair_rows(n, rank, world, tile=8)
    rows = np.arange(r0, r1, dtype=np.int64)
    piece, _ = oracle.ibs_block(G, G, rows=rows, threads=1)
    # keep the pairs i <= j of the owned rows
    mine = []
    for k, i in enumerate(rows):
        mine.append(piece[k, i:].reshape(-1, 4))
    mine = np.concatenate(mine) if mine else np.zeros((0, 4), np.int32)
    gathered = [None] * world
    dist.all_gather_object(gathered, (r0, r1, mine))
    if rank == 0:
        full, _ = oracle.ibs_triangle(packed, n, m)
        assembled = np.concatenate([g[2] for g in sorted(gathered, key=lambda g: g[0])])
        q.put(bool(assembled.shape == full.shape and (assembled == full).all()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_reassemble_full_matrix(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, 45, 300, 3, q)) for r in range(world)]
    for p in procs:
        p.start()
    ok = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok
