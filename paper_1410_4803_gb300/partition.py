"""Row-block partition of the triangular tile schedule across ranks.

The paper splits a sample x sample matrix across processes with
`--parallel k K`, each run computing 1/K of the matrix and the pieces being
concatenated ("Multicore and cluster parallelism", "Memory efficiency").  The
GPU equivalent: the pair tiles of the upper triangle, in row-major order, are
cut into contiguous ranges of whole tile rows with near-equal work (row I
holds T - I tiles).  Each rank needs the planes of its rows and of all
columns to its right; the ranks' outputs are disjoint, so no reduction is
needed.  This module is host logic only.

The default tile is the tensor-core kernels' 128-sample block (the operand
planes' block), so a rank's range never splits a block; the integer (POPC)
form works on 64-sample blocks and takes ``tile=TILE_POPC``.
"""
from __future__ import annotations

TILE = 128      # sample block of the tensor-core operand planes (default form)
TILE_POPC = 64  # sample block of the integer form's bit planes


def n_tiles(n: int, tile: int = TILE) -> int:
    return -(-n // tile)


def row_start(I: int, T: int) -> int:
    """Linear index of tile (I, I) in the row-major upper triangle of T x T tiles."""
    return I * T - I * (I - 1) // 2


def partition_rows(n: int, world: int, tile: int = TILE):
    """[(I0, I1)] per rank: contiguous tile-row ranges with near-equal tile
    counts.  Each boundary is the row edge whose cumulative tile count is
    closest to rank r's share r * total / world."""
    T = n_tiles(n, tile)
    total = T * (T + 1) // 2
    cum = [0]
    for I in range(T):
        cum.append(cum[-1] + T - I)
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        best = min(range(bounds[-1], T + 1), key=lambda e: abs(cum[e] - target))
        bounds.append(best)
    bounds.append(T)
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def partition_tiles(n: int, world: int, tile: int = TILE):
    """[(tile_begin, tile_end)] linear tile ranges of each rank."""
    T = n_tiles(n, tile)
    return [(row_start(a, T), row_start(b, T)) for a, b in partition_rows(n, world, tile)]


def pair_rows(n: int, rank: int, world: int, tile: int = TILE):
    """Sample rows [r0, r1) whose pairs (i <= j) rank `rank` owns."""
    a, b = partition_rows(n, world, tile)[rank]
    return min(n, a * tile), min(n, b * tile)
