#!/usr/bin/env python3
"""Write tests/golden/structured_rows.txt: oracle counts of 512 fixed samples of
the structured cohort (n = 20,000 samples x m = 500,000 variants, seed 2)
against all 20,000 samples, one SHA-256 per row.

Calls only ``oracle/`` (and the shared input generator): the expected values
are the plain CPU rule of the paper's section "Improvements in PLINK 1.9 /
Bitwise parallelism" (per marker: skip when either call is missing, equal
codes -> IBS2, both bits differ -> IBS0, else IBS1).  About 5.1e12
comparisons; run once (about 75 minutes on 8 cores).

Row i's record hashes the int32 little-endian bytes of counts[i][j] =
(IBS0, IBS1, IBS2, N) for j = 0 .. n-1 (a full row of the symmetric matrix),
and of the float64 distances (IBS1 + 2 IBS0) / (2 N) the oracle returns, and
lists the four column sums.  The input's SHA-256 is recorded too, so a
machine whose generator produced other bytes is detected before any
comparison.

    python tests/golden/make_structured_rows.py [--threads T]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "structured_rows.txt")


def structured_rows(n: int = 20_000, n_base: int = 19_750) -> np.ndarray:
    """The 512 rows: 262 base samples evenly spread, then every injected
    offspring (200) and duplicate (50), which sit after the base samples."""
    base = np.unique(np.linspace(0, n_base - 1, 262).astype(np.int64))
    rel = np.arange(n_base, n, dtype=np.int64)
    return np.concatenate([base, rel])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--batch", type=int, default=16)
    args = ap.parse_args()
    import oracle
    from paper_1410_4803_gb300 import synth

    t0 = time.time()
    w = synth.structured_config3()
    in_sha = hashlib.sha256(w.packed.tobytes()).hexdigest()
    rows = structured_rows(w.n)
    assert rows.size == 512
    G = oracle.unpack(w.packed, w.n, w.m)
    del w.packed
    partial = OUT + ".partial"
    done = {}
    if os.path.exists(partial):
        for ln in open(partial):
            f = ln.split()
            if len(f) == 8 and f[0] == in_sha:
                done[int(f[1])] = " ".join(f[1:])
    print(f"input {in_sha}, {len(done)} rows already done, {time.time() - t0:.0f} s", flush=True)
    todo = [r for r in rows if int(r) not in done]
    with open(partial, "a") as fp:
        for b0 in range(0, len(todo), args.batch):
            sel = np.asarray(todo[b0:b0 + args.batch], dtype=np.int64)
            t = time.time()
            counts, dist = oracle.ibs_block(G, G, rows=sel, threads=args.threads)
            for k, r in enumerate(sel):
                c = np.ascontiguousarray(counts[k]).astype("<i4")
                d = np.ascontiguousarray(dist[k]).astype("<f8")
                sums = c.astype(np.int64).sum(axis=0)
                rec = (f"{int(r)} {hashlib.sha256(c.tobytes()).hexdigest()} "
                       f"{hashlib.sha256(d.tobytes()).hexdigest()} {sums[0]} {sums[1]} {sums[2]} {sums[3]}")
                done[int(r)] = rec
                fp.write(f"{in_sha} {rec}\n")
            fp.flush()
            print(f"{len(done)}/{rows.size} rows, batch {time.time() - t:.0f} s", flush=True)
    with open(OUT, "w") as fo:
        fo.write("# Oracle rows of the structured cohort: n = 20,000 samples x m = 500,000 variants, seed 2\n")
        fo.write("# (Balding-Nichols, five subpopulations, F = 0.05; 200 parent-offspring pairs, 50 duplicates;\n")
        fo.write("# 1% missing).  Written by tests/golden/make_structured_rows.py, which calls only oracle/.\n")
        fo.write("# Rule: paper, section \"Improvements in PLINK 1.9 / Bitwise parallelism\", the per-marker loop.\n")
        fo.write("# Per row i: sha256 of int32 LE counts[i][0..n-1][IBS0, IBS1, IBS2, N], sha256 of the float64\n")
        fo.write("# LE distances (IBS1 + 2 IBS0) / (2N) (NaN where N = 0), and the four column sums.\n")
        fo.write(f"input_sha256 {in_sha}\n")
        fo.write("n 20000\nm 500000\n")
        for r in rows:
            fo.write("row " + done[int(r)] + "\n")
    os.unlink(partial)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
