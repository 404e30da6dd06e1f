"""The two-SM pair kernel (tcgen05 cta_group::2) through ibs_compute, forced
on for every size with IBS_TC_PAIR=1: bit-exact counts and distances within
1e-12 against the oracle.  The switch is read once per process, so each case
runs in a child process.  Also the default choice (ibs_compute_kernel): the
pair kernel for 65,536 or more variants, the one-SM kernel otherwise.
Shapes: two blocks with a ragged marker tail, a lone diagonal tile per column
pair, garbage in the padding bits, every tile split over K (fewer pair items
than clusters), and whole waves plus an unsplit tail; every ring variant.
The K-lockstep of full waves with 16-chunk segments (lag 2 and 3), so that its
bounded waits run many times per item."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import oracle
from helpers import assert_dist_close, gpu_compute, pack_codes, random_codes
from paper_1410_4803_gb300 import ibs
ctx = ibs.ibs_init(0, flags=ibs.IBS_KERNEL_TC | ibs.IBS_TC_FP4)
rng = np.random.default_rng({seed})
for n, m, miss, garbage in {shapes!r}:
    assert ibs.ibs_compute_kernel(ctx, n, m) == "tc-pair", (n, m)
    codes = random_codes(rng, n, m, miss=miss)
    packed = pack_codes(codes, garbage_rng=np.random.default_rng(7) if garbage else None)
    want_c, want_d = oracle.ibs_triangle(packed, n, m)
    got_c, got_d = gpu_compute(ctx, packed, n, m)
    bad = np.flatnonzero((got_c != want_c).any(axis=1))
    assert bad.size == 0, f"n={{n}} m={{m}}: {{bad.size}} pairs differ, first {{bad[:4]}}"
    assert_dist_close(got_d, want_d)
    print(f"ok n={{n}} m={{m}}")
ibs.ibs_shutdown(ctx)
"""

SHAPES = {
    "3,3": [(129, 65, 0.05, False), (256, 1, 0.0, False), (300, 1000, 0.3, True), (1500, 4000, 0.02, False),
            (2200, 700, 0.02, True)],
    "2,4": [(257, 1025, 0.05, True), (1100, 777, 0.1, False)],
    "4,2": [(257, 1025, 0.05, False), (700, 3001, 0.02, True)],
    "1,8": [(200, 130, 0.05, False), (640, 2000, 0.02, False)],
}


@pytest.mark.parametrize("ring", sorted(SHAPES))
def test_pair_kernel_matches_oracle(ring):
    code = CHILD.format(tests=os.path.join(ROOT, "tests"), root=ROOT, seed=11, shapes=SHAPES[ring])
    env = dict(os.environ, IBS_TC_PAIR="1", IBS_TC_PAIR_RING=ring)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok n=") == len(SHAPES[ring])


CHOICE = r"""
import sys
sys.path.insert(0, {root!r})
from paper_1410_4803_gb300 import ibs
want = {want!r}
for flags, n, m, kern in want:
    ctx = ibs.ibs_init(0, flags=flags)
    got = ibs.ibs_compute_kernel(ctx, n, m)
    ibs.ibs_shutdown(ctx)
    assert got == kern, (flags, n, m, got, kern)
print("ok")
"""


@pytest.mark.parametrize("mode", ["auto", "off"])
def test_default_kernel_choice(mode):
    from paper_1410_4803_gb300 import ibs
    tc4, tc8 = ibs.IBS_KERNEL_TC | ibs.IBS_TC_FP4, ibs.IBS_KERNEL_TC | ibs.IBS_TC_FP8
    long_k = "tc-pair" if mode == "auto" else "tc-persistent"
    want = [(tc4, 4096, 100_000, long_k), (tc4, 20_000, 500_000, long_k), (tc4, 300, 65_536, long_k),
            (tc4, 300, 65_472, "tc-persistent"), (tc4, 4096, 30_000, "tc-persistent"),
            (tc4, 128, 500_000, "tc-persistent"),
            (tc8, 20_000, 500_000, "tc-persistent"), (tc4 | ibs.IBS_OUT_SQUARE, 20_000, 500_000, "tc-tile"),
            (ibs.IBS_KERNEL_CSA, 20_000, 500_000, "popc-csa")]
    env = {k: v for k, v in os.environ.items() if k not in ("IBS_TC_PAIR", "IBS_TC_TILE_KERNEL")}
    if mode == "off":
        env["IBS_TC_PAIR"] = "0"
    r = subprocess.run([sys.executable, "-c", CHOICE.format(root=ROOT, want=want)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


# K-lockstep of full waves with short segments, so that the bounded waits run
# many times per item: shapes with at least one full wave of pair items (76
# clusters; 2,200 samples = 18 blocks = 90 pair items) and hundreds of chunks,
# plus a shape whose items are all in the split tail (no lockstep).
SYNC_SHAPES = [(2200, 20_000, 0.02, True), (2500, 9_001, 0.05, False), (700, 30_000, 0.02, False)]


@pytest.mark.parametrize("sync", ["16,2", "16,3"])
def test_pair_kernel_lockstep_matches_oracle(sync):
    code = CHILD.format(tests=os.path.join(ROOT, "tests"), root=ROOT, seed=12, shapes=SYNC_SHAPES)
    env = dict(os.environ, IBS_TC_PAIR="1", IBS_TC_PAIR_SYNC=sync)
    env.pop("IBS_TC_PAIR_RING", None)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok n=") == len(SYNC_SHAPES)
