"""Batched path (ibs_compute_batch): many subsets of a pool over uneven
variant windows in one persistent launch under a CUDA graph.  Each subset's
result must equal the plain path on that subset alone and the oracle."""
import numpy as np
import pytest

import oracle
from helpers import assert_dist_close, pack_codes

pytestmark = pytest.mark.gpu


def _subset_packed(pool_codes, idx, vb, vl):
    return pack_codes(pool_codes[idx][:, vb:vb + vl])


@pytest.fixture(scope="module")
def pool():
    from paper_1410_4803_gb300 import synth
    w = synth.batch_pool(pool_n=1500, pool_m=30000, seed=11)
    codes = oracle.unpack(w.packed, w.n, w.m)
    return w, codes


def _make_subsets(rng, pool_n, pool_m):
    spec = [(1, 1), (2, 31), (63, 33), (64, 385), (65, 1000), (130, 4097), (700, 20000), (257, 383),
            (5, 29999), (400, 12345), (129, 64), (900, 7000)]
    subs = []
    for n, vl in spec:
        idx = rng.choice(pool_n, size=n, replace=False).astype(np.int64)
        if rng.random() < 0.5:
            idx = np.sort(idx)
        vb = int(rng.integers(0, pool_m - vl + 1))
        subs.append((idx, vb, vl))
    return subs


def _run_batch(ctx, w, subs, dev_packed):
    import torch
    from paper_1410_4803_gb300 import ibs
    args, outs = [], []
    for idx, vb, vl in subs:
        n = idx.size
        P = n * (n + 1) // 2
        c = torch.full((P, 4), -7, dtype=torch.int32, device="cuda")
        d = torch.empty(P, dtype=torch.float64, device="cuda")
        it = torch.from_numpy(idx).cuda()
        args.append((it, vb, vl, c, d))
        outs.append((c, d, it))
    ibs.ibs_compute_batch(ctx, dev_packed, w.n, w.m, args)
    ibs.ibs_synchronize(ctx)
    return [(c.cpu().numpy(), d.cpu().numpy()) for c, d, _ in outs]


def test_batch_matches_plain_and_oracle(pool, tmp_path):
    import torch
    from paper_1410_4803_gb300 import ibs
    w, codes = pool
    rng = np.random.default_rng(5)
    subs = _make_subsets(rng, w.n, w.m)
    dev_packed = torch.from_numpy(w.packed).cuda()
    ctx = ibs.ibs_init(0, autotune_cache_path=str(tmp_path / "tune.jsonl"))
    plain = ibs.ibs_init(0)
    try:
        first = _run_batch(ctx, w, subs, dev_packed)
        second = _run_batch(ctx, w, subs, dev_packed)  # graph replay with new output buffers
        for (idx, vb, vl), (c1, d1), (c2, d2) in zip(subs, first, second):
            n = idx.size
            assert (c1 == c2).all()
            sp = _subset_packed(codes, idx, vb, vl)
            pc, pd = ibs.compute(plain, torch.from_numpy(sp).cuda(), n, vl)
            ibs.ibs_synchronize(plain)
            assert (c1 == pc.cpu().numpy()).all(), f"batch != plain for n={n} window={vb}+{vl}"
            G = oracle.unpack_subset(w.packed, w.n, w.m, idx, vb, vl)
            oc, od, _ = oracle.ibs_triangle_from_codes(G)
            assert (c1 == oc).all(), f"batch != oracle for n={n} window={vb}+{vl}"
            assert_dist_close(d1, od)
        info = ibs.ibs_batch_plan_info(ctx)
        assert info["items"] > 0 and info["grid"] > 0
        assert info["mode"] in (3, 4)  # tensor-core form by default, as ibs_compute
        assert (tmp_path / "tune.jsonl").exists()
    finally:
        ibs.ibs_shutdown(plain)
        ibs.ibs_shutdown(ctx)


def _flags(ibs, names):
    f = 0
    for nm in names.split("|"):
        f |= getattr(ibs, nm)
    return f


@pytest.mark.parametrize("flags_name", ["IBS_KERNEL_PLAIN", "IBS_KERNEL_CSA", "IBS_KERNEL_TC|IBS_TC_FP8",
                                        "IBS_KERNEL_TC|IBS_TC_FP4"])
def test_batch_forced_modes(pool, flags_name):
    import torch
    from paper_1410_4803_gb300 import ibs
    w, codes = pool
    rng = np.random.default_rng(6)
    subs = _make_subsets(rng, w.n, w.m)[:6]
    ctx = ibs.ibs_init(0, flags=_flags(ibs, flags_name))
    try:
        res = _run_batch(ctx, w, subs, torch.from_numpy(w.packed).cuda())
        for (idx, vb, vl), (c, d) in zip(subs, res):
            G = oracle.unpack_subset(w.packed, w.n, w.m, idx, vb, vl)
            oc, od, _ = oracle.ibs_triangle_from_codes(G)
            assert (c == oc).all()
    finally:
        ibs.ibs_shutdown(ctx)


@pytest.mark.parametrize("flags_name", ["IBS_KERNEL_CSA", "IBS_KERNEL_TC|IBS_TC_FP8", "IBS_KERNEL_TC|IBS_TC_FP4"])
def test_batch_split_items(pool, flags_name):
    """One subset of few tiles and many chunks: the autotuner splits the
    marker axis into items that add into a partial triangle, and a finalize
    launch writes the counts."""
    import torch
    from paper_1410_4803_gb300 import ibs
    w, _ = pool
    rng = np.random.default_rng(8)
    subs = [(np.sort(rng.choice(w.n, size=150, replace=False)).astype(np.int64), 17, 29000)]
    ctx = ibs.ibs_init(0, flags=_flags(ibs, flags_name))
    try:
        (c, d), = _run_batch(ctx, w, subs, torch.from_numpy(w.packed).cuda())
        # tensor-core modes may also pick the per-subset launches (policy 2),
        # which split this subset's few tiles over K as ibs_compute does
        assert ibs.ibs_batch_plan_info(ctx)["split_policy"] in ((1, 2, 3) if "TC" in flags_name else (1,))
        idx, vb, vl = subs[0]
        G = oracle.unpack_subset(w.packed, w.n, w.m, idx, vb, vl)
        oc, od, _ = oracle.ibs_triangle_from_codes(G)
        assert (c == oc).all()
        assert_dist_close(d, od)
    finally:
        ibs.ibs_shutdown(ctx)


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("fmt", ["IBS_TC_FP8", "IBS_TC_FP4"])
def test_batch_each_policy(pool, policy, fmt, monkeypatch):
    """Every split policy of the tensor-core batch, fixed by IBS_BATCH_POLICY:
    0 whole tiles in one launch per stage, 1 K-split large subsets, 2 one
    launch per subset over its own work list (small subsets and tail waves
    split over K, split tiles finalised from the subset descriptors), 3 and 4
    (E2M1 only) one launch of the two-SM kernel over every subset's pair items
    with the gather fused in, 5 (E2M1 only) policy 2's launches with each
    two-SM launch's epilogue warps gathering the following subsets (here every
    window is under the two-SM size, so each subset gets its own gather
    launch; the fused form is tested in a child below).  Counts equal the
    oracle for all twelve subsets, twice (graph replay)."""
    import torch
    from paper_1410_4803_gb300 import ibs
    if policy >= 3 and fmt != "IBS_TC_FP4":
        pytest.skip("the two-SM kernel takes E2M1 operands only")
    monkeypatch.setenv("IBS_BATCH_POLICY", str(policy))
    w, codes = pool
    rng = np.random.default_rng(9)
    subs = _make_subsets(rng, w.n, w.m)
    ctx = ibs.ibs_init(0, flags=_flags(ibs, "IBS_KERNEL_TC|" + fmt))
    try:
        dev = torch.from_numpy(w.packed).cuda()
        first = _run_batch(ctx, w, subs, dev)
        second = _run_batch(ctx, w, subs, dev)
        assert ibs.ibs_batch_plan_info(ctx)["split_policy"] == policy
        for (idx, vb, vl), (c1, d1), (c2, d2) in zip(subs, first, second):
            G = oracle.unpack_subset(w.packed, w.n, w.m, idx, vb, vl)
            oc, od, _ = oracle.ibs_triangle_from_codes(G)
            assert (c1 == oc).all(), f"policy {policy}: n={idx.size} window={vb}+{vl}"
            assert (c2 == oc).all()
            assert_dist_close(d1, od)
            np.testing.assert_array_equal(d1, d2)
    finally:
        ibs.ibs_shutdown(ctx)


def test_batch_out_of_range_index_is_reported(pool):
    """A corrupted sample index is not read: the kernel treats that sample as
    all-missing and ibs_synchronize reports IBS_EINVAL."""
    import torch
    from paper_1410_4803_gb300 import ibs
    w, _ = pool
    ctx = ibs.ibs_init(0)
    try:
        idx = torch.tensor([0, 5, w.n + 100], dtype=torch.int64, device="cuda")
        c = torch.empty((6, 4), dtype=torch.int32, device="cuda")
        ibs.ibs_compute_batch(ctx, torch.from_numpy(w.packed).cuda(), w.n, w.m, [(idx, 0, 500, c, None)])
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_synchronize(ctx)
        assert ei.value.status == ibs.IBS_EINVAL
        got = c.cpu().numpy()
        # pairs with the bad sample have N = 0
        assert got[oracle.tri_index(0, 2, 3), 3] == 0 and got[oracle.tri_index(2, 2, 3), 3] == 0
    finally:
        ibs.ibs_shutdown(ctx)


def test_batch_validation_errors(pool):
    import torch
    from paper_1410_4803_gb300 import ibs
    w, _ = pool
    ctx = ibs.ibs_init(0)
    try:
        idx = torch.arange(10, dtype=torch.int64, device="cuda")
        c = torch.empty((55, 4), dtype=torch.int32, device="cuda")
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_compute_batch(ctx, torch.from_numpy(w.packed).cuda(), w.n, w.m, [(idx, w.m - 10, 20, c, None)])
        assert ei.value.status == ibs.IBS_EINVAL
    finally:
        ibs.ibs_shutdown(ctx)


def test_batch_windows_move_between_calls(pool):
    """Same subset shapes (n, window length) on two calls, but the windows
    start elsewhere on the second: the cached plan is reused and the gather's
    CTA map (ordered by pool variant) is rebuilt; both calls equal the oracle."""
    import torch
    from paper_1410_4803_gb300 import ibs
    w, _ = pool
    rng = np.random.default_rng(12)
    subs = _make_subsets(rng, w.n, w.m)[:8]
    moved = []
    for idx, vb, vl in subs:
        vb2 = int(rng.integers(0, w.m - vl + 1))
        moved.append((idx, vb2, vl))
    ctx = ibs.ibs_init(0)
    try:
        dev = torch.from_numpy(w.packed).cuda()
        for case in (subs, moved, subs):
            res = _run_batch(ctx, w, case, dev)
            for (idx, vb, vl), (c, d) in zip(case, res):
                G = oracle.unpack_subset(w.packed, w.n, w.m, idx, vb, vl)
                oc, od, _ = oracle.ibs_triangle_from_codes(G)
                assert (c == oc).all(), f"n={idx.size} window={vb}+{vl}"
                assert_dist_close(d, od)
    finally:
        ibs.ibs_shutdown(ctx)


POLICY5_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import torch
import oracle
from helpers import assert_dist_close
from test_gpu_batch import _flags, _make_subsets, _run_batch
from paper_1410_4803_gb300 import ibs, synth
w = synth.batch_pool(pool_n=1500, pool_m=30000, seed=11)
subs = _make_subsets(np.random.default_rng(9), w.n, w.m)
ctx = ibs.ibs_init(0, flags=_flags(ibs, "IBS_KERNEL_TC|IBS_TC_FP4"))
dev = torch.from_numpy(w.packed).cuda()
first = _run_batch(ctx, w, subs, dev)
second = _run_batch(ctx, w, subs, dev)
assert ibs.ibs_batch_plan_info(ctx)["split_policy"] == 5
launches = ibs.ibs_last_launch_info(ctx)["launches"]
for (idx, vb, vl), (c1, d1), (c2, d2) in zip(subs, first, second):
    G = oracle.unpack_subset(w.packed, w.n, w.m, idx, vb, vl)
    oc, od, _ = oracle.ibs_triangle_from_codes(G)
    assert (c1 == oc).all(), f"n={{idx.size}} window={{vb}}+{{vl}}"
    assert (c2 == oc).all()
    assert_dist_close(d1, od)
    np.testing.assert_array_equal(d1, d2)
ibs.ibs_shutdown(ctx)
print("ok", launches)
"""


def test_batch_policy5_fused_gather():
    """Policy 5 with the two-SM kernel forced on for every subset of two or
    more blocks (IBS_TC_PAIR=1, read once per process: a child): the order
    mixes two-SM subsets, whose epilogue warps gather the planes of the
    subsets after them, and one-SM subsets (n <= 128), which the preceding
    two-SM launch gathers; the first subset gets a gather launch of its own.
    Counts equal the oracle for all twelve subsets, twice (graph replay)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = POLICY5_CHILD.format(tests=os.path.join(root, "tests"), root=root)
    env = dict(os.environ, IBS_TC_PAIR="1", IBS_BATCH_POLICY="5")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout, r.stdout
