"""Parity at the full sizes of the batched, served and structured workloads.

- Batched: 64 cohort subsets of uneven size drawn from a 30,000-sample pool
  over uneven variant windows of a 600,000-variant matrix (the batch the bench
  times).  Every subset of the batched call equals the plain path run on that
  subset's own packed matrix, counts bit for bit and distances exactly; sampled
  pairs of eight subsets equal the oracle.
- Served: the resident 100,000 x 200,000 panel with three requests of
  different sizes in flight together.  Sampled query rows equal the oracle
  against every panel sample, and each request's top-16 equals the oracle's
  ranking rule applied to the oracle's distances.
- Structured: the n = 20,000 x m = 500,000 cohort against 512 rows of oracle
  counts hashed once by tests/golden/make_structured_rows.py (every injected
  offspring and duplicate among them).

The inputs come from the shared generator on the device (the same bytes as
on the host, see test_gpu_synth.py); nothing here reads the reference.
"""
import hashlib
import os

import numpy as np
import pytest

from helpers import assert_dist_close

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _subset_packed(pool, idx, vb, vl):
    """Packed .bed matrix of one subset gathered from the device pool (test harness)."""
    import torch
    rows = pool[vb:vb + vl]
    byte = rows.index_select(1, idx // 4)
    code = (byte >> (2 * (idx % 4)).to(torch.uint8)) & 3
    pad = (-idx.numel()) % 4
    if pad:
        code = torch.nn.functional.pad(code, (0, pad), value=1)
    code = code.view(vl, -1, 4)
    return (code[..., 0] | (code[..., 1] << 2) | (code[..., 2] << 4) | (code[..., 3] << 6)).contiguous()


def test_batch_full_pool_every_subset_equals_plain_and_oracle_pairs():
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs, synth
    torch.cuda.set_device(0)
    w = synth.batch_pool(device=0)
    subs = synth.batch_subsets()
    assert len(subs) == 64 and w.n == 30_000 and w.m == 600_000
    pool = w.packed
    args, outs = [], []
    for s in subs:
        idx = torch.from_numpy(s.sample_idx).cuda()
        P = s.n * (s.n + 1) // 2
        c = torch.empty((P, 4), dtype=torch.int32, device="cuda")
        d = torch.empty(P, dtype=torch.float64, device="cuda")
        args.append((idx, s.var_begin, s.var_len, c, d))
        outs.append((c, d))
    ctx_b = ibs.ibs_init(0)
    ctx_p = ibs.ibs_init(0)
    try:
        ibs.ibs_compute_batch(ctx_b, pool, w.n, w.m, args)
        ibs.ibs_synchronize(ctx_b)
        for k, s in enumerate(subs):
            packed = _subset_packed(pool, args[k][0], s.var_begin, s.var_len)
            pc, pd = ibs.compute(ctx_p, packed, s.n, s.var_len)
            ibs.ibs_synchronize(ctx_p)
            assert torch.equal(outs[k][0], pc), f"subset {k}: counts differ from the plain path"
            bd = torch.nan_to_num(outs[k][1], nan=-1.0)
            assert torch.equal(bd, torch.nan_to_num(pd, nan=-1.0)), f"subset {k}: distances differ"
            del packed, pc, pd
    finally:
        ibs.ibs_shutdown(ctx_b)
        ibs.ibs_shutdown(ctx_p)
    host = pool.cpu().numpy()
    rng = np.random.default_rng(44)
    for k in rng.choice(len(subs), 8, replace=False):
        s = subs[k]
        rows = np.sort(rng.choice(s.n, min(s.n, 24), replace=False))
        G = oracle.unpack_subset(host, w.n, w.m, s.sample_idx[rows], s.var_begin, s.var_len)
        want_c, want_d = oracle.ibs_block(G, G)
        iu = np.triu_indices(rows.size)
        tri = oracle.tri_index(rows[iu[0]], rows[iu[1]], s.n)
        got_c = outs[k][0][torch.from_numpy(tri).cuda()].cpu().numpy()
        got_d = outs[k][1][torch.from_numpy(tri).cuda()].cpu().numpy()
        assert (got_c == want_c[iu]).all(), f"subset {k}: oracle pairs differ"
        assert_dist_close(got_d, want_d[iu])


def test_serving_full_panel_mixed_requests_against_oracle():
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs, synth
    torch.cuda.set_device(0)
    panel = synth.serving_panel(device=0)
    n, m = panel.n, panel.m
    assert n == 100_000 and m == 200_000
    k = 16
    sizes = [1, 37, 300]
    reqs = []
    for i, q in enumerate(sizes):
        qp, _ = synth.serving_queries(panel, q, request_id=900 + i)
        reqs.append((q, qp, torch.empty((q, n, 4), dtype=torch.int32).pin_memory(),
                     torch.empty((q, k), dtype=torch.int32).pin_memory(),
                     torch.empty((q, k), dtype=torch.float64).pin_memory()))
    ctx = ibs.ibs_init(0)
    try:
        ibs.ibs_panel_load(ctx, panel.packed, n, m)
        host_panel = panel.packed.cpu().numpy()
        panel.packed = None
        ids = [ibs.ibs_query(ctx, qp, q, k, oc, oi, od) for q, qp, oc, oi, od in reqs]  # all in flight together
        for rid in ids:
            ibs.ibs_wait(ctx, rid, timeout_ms=600_000)
    finally:
        ibs.ibs_shutdown(ctx)
    # oracle: the first and last query row of each request against every panel
    # sample; panel columns unpacked once, in slices, to bound host memory
    picks = [np.unique(np.array([0, q - 1], dtype=np.int64)) for q, *_ in reqs]
    GQ = np.concatenate([oracle.unpack_subset(qp, q, m, r, 0, m) for (q, qp, *_), r in zip(reqs, picks)])
    want_c = np.empty((GQ.shape[0], n, 4), dtype=np.int32)
    want_d = np.empty((GQ.shape[0], n), dtype=np.float64)
    step = 12_500
    for c0 in range(0, n, step):
        cols = np.arange(c0, min(n, c0 + step), dtype=np.int64)
        GP = oracle.unpack_subset(host_panel, n, m, cols, 0, m)
        cc, dd = oracle.ibs_block(GQ, GP)
        want_c[:, c0:c0 + cols.size] = cc
        want_d[:, c0:c0 + cols.size] = dd
    t = 0
    for (q, qp, oc, oi, od), rows in zip(reqs, picks):
        for r in rows:
            assert (oc.numpy()[r] == want_c[t]).all(), f"q={q} row {r}: counts differ from the oracle"
            idx, dist = oracle.topk(want_d[t], k)
            assert (oi.numpy()[r] == idx).all(), f"q={q} row {r}: top-k indices differ"
            assert_dist_close(od.numpy()[r], dist)
            t += 1


def _golden():
    path = os.path.join(HERE, "golden", "structured_rows.txt")
    if not os.path.exists(path):
        pytest.skip("tests/golden/structured_rows.txt not written yet (make_structured_rows.py)")
    meta, rows = {}, []
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        if f[0] == "row":
            rows.append((int(f[1]), f[2], f[3], tuple(int(x) for x in f[4:8])))
        else:
            meta[f[0]] = f[1]
    return meta, rows


def test_structured_cohort_512_rows_match_oracle_hashes():
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs, synth
    meta, rows = _golden()
    torch.cuda.set_device(0)
    w = synth.structured_config3(device=0)
    n, m = w.n, w.m
    assert (n, m) == (int(meta["n"]), int(meta["m"]))
    assert hashlib.sha256(w.packed.cpu().numpy().tobytes()).hexdigest() == meta["input_sha256"], \
        "the generator produced other input bytes on this machine"
    ctx = ibs.ibs_init(0)
    try:
        counts, dist = ibs.compute(ctx, w.packed, n, m)
        ibs.ibs_synchronize(ctx)
        kernel = ibs.ibs_compute_kernel(ctx, n, m)
    finally:
        ibs.ibs_shutdown(ctx)
    del w
    j = np.arange(n, dtype=np.int64)
    for i, c_sha, d_sha, sums in rows:
        lo, hi = np.minimum(i, j), np.maximum(i, j)
        idx = torch.from_numpy(lo * n - lo * (lo - 1) // 2 + (hi - lo)).cuda()
        c = counts.index_select(0, idx).cpu().numpy().astype("<i4")
        d = dist.index_select(0, idx).cpu().numpy()
        assert tuple(int(x) for x in c.astype(np.int64).sum(axis=0)) == sums, f"row {i} ({kernel}): column sums differ"
        assert hashlib.sha256(c.tobytes()).hexdigest() == c_sha, f"row {i} ({kernel}): counts differ"
        want_d = oracle.dist_from_counts(c)
        assert hashlib.sha256(want_d.astype("<f8").tobytes()).hexdigest() == d_sha
        assert_dist_close(d, want_d)
