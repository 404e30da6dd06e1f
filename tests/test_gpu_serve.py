"""Serving engine: resident panel, continuous batching, admission, top-k.
Each request's result must be the same alone (ibs_query_sync) and in the mix,
and equal to the oracle."""
import threading
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def panel():
    from paper_1410_4803_gb300 import synth
    # 10,040 panel samples = 157 blocks of 64 (79 of 128), more than one step covers for a 2,048-row request
    w = synth.serving_panel(n_base_per_pop=2000, n_pop=5, m=16000, n_offspring=30, n_dup=10, seed=21)
    G = oracle.unpack(w.packed, w.n, w.m)
    return w, G


def _pinned(shape, dtype):
    import torch
    return torch.empty(shape, dtype=dtype).pin_memory()


@pytest.mark.parametrize("kernel", ["tensor-core", "popc"])
def test_serving_mix_equals_alone_and_oracle(panel, kernel):
    """Both pair-kernel families: the tensor-core form (FP4 operand planes,
    128-sample blocks) and the carry-save POPC kernel (bit planes, 64-sample
    blocks)."""
    import torch
    from paper_1410_4803_gb300 import ibs, synth
    w, Gp = panel
    ctx = ibs.ibs_init(0, flags=ibs.IBS_KERNEL_TC if kernel == "tensor-core" else ibs.IBS_KERNEL_CSA)
    try:
        ibs.ibs_panel_load(ctx, torch.from_numpy(w.packed).cuda(), w.n, w.m)
        # The first request is large enough that its work spans several engine
        # steps (a step holds about 16 waves of 64 x 64 tiles, or 8 waves of
        # the tensor-core form's 128 x 128 tiles), so the small requests
        # submitted right after it join while it is still running.
        sizes = [2048, 1, 64, 65, 3, 150, 17, 128, 2, 90, 33, 7, 129]
        k = 16
        reqs = []
        for r, q in enumerate(sizes):
            qp, qs = synth.serving_queries(w, q, request_id=r, related_frac=0.3, seed=21)
            reqs.append((q, qp, qs))
        # all output buffers exist before anything is submitted
        results = [(_pinned((q, w.n, 4), torch.int32), _pinned((q, k), torch.int32), _pinned((q, k), torch.float64))
                   for q, _, _ in reqs]
        ids = [None] * len(reqs)
        errors = []
        # the large request first, then half of the others at once from this
        # thread (they join while it is still on the GPU: the engine takes
        # several steps over it), the rest from three threads at the same time
        ids[0] = ibs.ibs_query(ctx, reqs[0][1], reqs[0][0], k, *results[0])

        def submit(slot_list):
            try:
                for i in slot_list:
                    q, qp, _ = reqs[i]
                    ids[i] = ibs.ibs_query(ctx, qp, q, k, *results[i])
            except Exception as e:  # pragma: no cover
                errors.append(e)

        rest = list(range(1, len(reqs)))
        submit(rest[::2])
        threads = [threading.Thread(target=submit, args=(rest[1::2][j::3],)) for j in range(3)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for i in range(len(reqs)):
            ibs.ibs_wait(ctx, ids[i], timeout_ms=120000)
        stats = ibs.ibs_serve_stats_get(ctx)
        assert stats["requests_done"] == len(reqs)
        assert stats["peak_rows"] > max(sizes), "requests never shared a step"
        assert stats["steps"] > 1
        for i, (q, qp, _) in enumerate(reqs):
            oc, oi, od = (x.numpy() for x in results[i])
            if q > 256:  # the oracle checks a sample of the large request's rows
                rows = np.linspace(0, q - 1, 48).astype(np.int64)
            else:
                rows = np.arange(q)
            # alone, through the unbatched path
            ac = _pinned((q, w.n, 4), torch.int32)
            ai = _pinned((q, k), torch.int32)
            ad = _pinned((q, k), torch.float64)
            ibs.ibs_query_sync(ctx, qp, q, k, ac, ai, ad)
            assert (oc == ac.numpy()).all(), f"request {i}: counts differ alone vs mixed"
            assert (oi == ai.numpy()).all()
            np.testing.assert_array_equal(od, ad.numpy())
            # oracle
            Gq = oracle.unpack(qp, q, w.m)
            wc, wd = oracle.ibs_block(Gq, Gp, rows=rows)
            assert (oc[rows] == wc).all(), f"request {i}: counts differ from the oracle"
            for t, r in enumerate(rows):
                ti, td = oracle.topk(wd[t], k)
                assert (oi[r] == ti).all(), f"request {i} row {r}: top-k indices differ"
                fin = ~np.isnan(td)
                assert (np.isnan(od[r]) == ~fin).all()
                assert np.allclose(od[r][fin], td[fin], rtol=1e-12, atol=0)
    finally:
        ibs.ibs_shutdown(ctx)


def test_serving_device_outputs_and_relatives(panel):
    import torch
    from paper_1410_4803_gb300 import ibs, synth
    w, Gp = panel
    ctx = ibs.ibs_init(0)
    try:
        ibs.ibs_panel_load(ctx, w.packed, w.n, w.m)  # host panel
        q, k = 40, 5
        qp, qs = synth.serving_queries(w, q, request_id=99, related_frac=1.0, seed=21)
        oc = torch.empty((q, w.n, 4), dtype=torch.int32, device="cuda")
        oi = torch.empty((q, k), dtype=torch.int32, device="cuda")
        od = torch.empty((q, k), dtype=torch.float64, device="cuda")
        rid = ibs.ibs_query(ctx, torch.from_numpy(qp).cuda(), q, k, oc, oi, od)
        ibs.ibs_wait(ctx, rid, timeout_ms=60000)
        oi = oi.cpu().numpy()
        gid = {int(g): i for i, g in enumerate(w.samples.gid)}
        oc = oc.cpu().numpy()
        for r in range(q):
            src = gid[int(qs.src_gid[r])]
            if qs.kind[r] == synth.DUPLICATE:
                # the source is the nearest panel sample (or second, behind a panel duplicate of it)
                assert src in oi[r, :2].tolist()
            if qs.kind[r] == synth.OFFSPRING:
                assert oc[r, src, 0] == 0  # a parent and child share an allele at every marker
    finally:
        ibs.ibs_shutdown(ctx)


def test_serving_k_larger_than_panel_and_admission():
    import torch
    from paper_1410_4803_gb300 import ibs
    from helpers import pack_codes, random_codes
    rng = np.random.default_rng(1)
    n_panel, m = 10, 700
    pcodes = random_codes(rng, n_panel, m)
    pcodes[3] = 1  # all-missing panel sample: NaN distance, ranked last
    pp = pack_codes(pcodes)
    # The engine's fixed buffers (panel planes, step planes for 4,096 rows,
    # step tables) take ~1.8 MB with bit planes and ~6.2 MB with FP4 operand
    # planes; the budget leaves room for a small request beside them but not
    # for a 4,096-row one.
    probe = ibs.ibs_init(0)
    tc = ibs.ibs_kernel_info(probe)["family"] == "tensor-core"
    ibs.ibs_shutdown(probe)
    ctx = ibs.ibs_init(0, workspace_bytes=(8 << 20) if tc else (4 << 20))
    try:
        ibs.ibs_panel_load(ctx, pp, n_panel, m)
        qc = random_codes(rng, 3, m)
        qp = pack_codes(qc)
        k = 16
        oi = _pinned((3, k), torch.int32)
        od = _pinned((3, k), torch.float64)
        rid = ibs.ibs_query(ctx, qp, 3, k, None, oi, od)
        ibs.ibs_wait(ctx, rid, timeout_ms=60000)
        _, wd = oracle.ibs_block(qc, pcodes)
        for r in range(3):
            ti, td = oracle.topk(wd[r], k)
            assert (oi.numpy()[r] == ti).all()
            assert (oi.numpy()[r, n_panel:] == -1).all() and np.isnan(od.numpy()[r, n_panel - 1:]).all()
        # a request needing ~2.9 MB (bit planes) or ~7.2 MB (FP4 planes) can never fit beside the
        # engine's buffers and is refused at once
        big = 4096
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_query(ctx, np.zeros((m, big // 4), np.uint8), big, k, _pinned((big, n_panel, 4), torch.int32),
                          _pinned((big, k), torch.int32), _pinned((big, k), torch.float64))
        assert ei.value.status in (ibs.IBS_EBUSY, ibs.IBS_EINVAL)
        # pageable output buffers are refused
        with pytest.raises(ibs.IbsError):
            ibs.ibs_query(ctx, qp, 3, k, None, np.zeros((3, k), np.int32), np.zeros((3, k)))
    finally:
        ibs.ibs_shutdown(ctx)


def test_shutdown_cancels_pending(panel):
    import torch
    from paper_1410_4803_gb300 import ibs, synth
    w, _ = panel
    ctx = ibs.ibs_init(0)
    ibs.ibs_panel_load(ctx, w.packed, w.n, w.m)
    q = 512
    qp, _ = synth.serving_queries(w, q, request_id=7, seed=21)
    statuses = []
    rids = []
    for _ in range(6):
        rids.append(ibs.ibs_query(ctx, qp, q, 4, None, _pinned((q, 4), torch.int32), _pinned((q, 4), torch.float64)))

    def waiter(rid):
        try:
            ibs.ibs_wait(ctx, rid, timeout_ms=120000)
            statuses.append(ibs.IBS_OK)
        except ibs.IbsError as e:
            statuses.append(e.status)

    ts = [threading.Thread(target=waiter, args=(r,)) for r in rids]
    for t in ts:
        t.start()
    time.sleep(0.5)
    ibs.ibs_shutdown(ctx)
    for t in ts:
        t.join(timeout=60)
    assert len(statuses) == len(rids)
    assert all(s in (ibs.IBS_OK, ibs.IBS_ECANCELLED) for s in statuses)


SERVE_TWO_SM = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import oracle
from helpers import pack_codes, random_codes
from paper_1410_4803_gb300 import ibs
rng = np.random.default_rng(5)
n_panel, m, k = 5999, 2100, 8  # 47 panel blocks (ragged), 33 chunks (ragged), padding garbage
pcodes = random_codes(rng, n_panel, m, miss=0.03)
pp = pack_codes(pcodes, garbage_rng=np.random.default_rng(3))
ctx = ibs.ibs_init(0, flags=ibs.IBS_KERNEL_TC | ibs.IBS_TC_FP4)
ibs.ibs_panel_load(ctx, torch.from_numpy(pp).cuda(), n_panel, m)
# 4,096 rows in all: odd and even numbers of 128-row blocks, a lone row, a
# request that spans several steps
sizes = [2900, 1, 130, 300, 129, 64, 77, 495]
reqs = []
for i, q in enumerate(sizes):
    qc = random_codes(np.random.default_rng(100 + i), q, m, miss=0.03)
    reqs.append((q, qc, pack_codes(qc, garbage_rng=np.random.default_rng(200 + i))))
outs = [(torch.empty((q, n_panel, 4), dtype=torch.int32).pin_memory(), torch.empty((q, k), dtype=torch.int32).pin_memory(),
         torch.empty((q, k), dtype=torch.float64).pin_memory()) for q, _, _ in reqs]
ids = [ibs.ibs_query(ctx, qp, q, k, *o) for (q, _, qp), o in zip(reqs, outs)]
for rid in ids:
    ibs.ibs_wait(ctx, rid, timeout_ms=120000)
st = ibs.ibs_serve_stats_get(ctx)
assert st["requests_done"] == len(sizes), st
for i, ((q, qc, qp), (oc, oi, od)) in enumerate(zip(reqs, outs)):
    ac = torch.empty((q, n_panel, 4), dtype=torch.int32).pin_memory()
    ai = torch.empty((q, k), dtype=torch.int32).pin_memory()
    ad = torch.empty((q, k), dtype=torch.float64).pin_memory()
    ibs.ibs_query_sync(ctx, qp, q, k, ac, ai, ad)
    assert (oc.numpy() == ac.numpy()).all(), f"request {{i}}: engine and unbatched counts differ"
    assert (oi.numpy() == ai.numpy()).all()
    rows = np.arange(q) if q <= 512 else np.linspace(0, q - 1, 64).astype(np.int64)
    wc, wd = oracle.ibs_block(qc, pcodes, rows=rows)
    bad = np.flatnonzero((oc.numpy()[rows] != wc).any(axis=(1, 2)))
    assert bad.size == 0, f"request {{i}} (q={{q}}): rows {{rows[bad[:4]]}} differ from the oracle"
    for t, r in enumerate(rows):
        ti, td = oracle.topk(wd[t], k)
        assert (oi.numpy()[r] == ti).all(), f"request {{i}} row {{r}}: top-k differs"
        fin = ~np.isnan(td)
        assert (np.isnan(od.numpy()[r]) == ~fin).all()
        assert np.allclose(od.numpy()[r][fin], td[fin], rtol=1e-12, atol=0)
    print(f"ok q={{q}}")
ibs.ibs_shutdown(ctx)
"""


def test_serving_two_sm_kernel_matches_oracle():
    """The engine's steps and the unbatched path on the two-SM kernel (forced
    on for this small panel with IBS_TC_PAIR=1; the switch is read once per
    process, so the case runs in a child): items of two query blocks x one
    panel block, a lone last block when the step's block count is odd, steps
    of one block on the one-SM kernel, counts columns copied to host memory
    step by step."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = SERVE_TWO_SM.format(tests=os.path.join(root, "tests"), root=root)
    env = dict(os.environ, IBS_TC_PAIR="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok q=") == 8, r.stdout


def test_serving_requests_at_the_row_limit():
    """Three 4,096-row requests submitted at once: each fills the engine's
    4,096 admission slots, so they are admitted one after another while the
    others wait.  Every result equals the unbatched path and the oracle."""
    import torch
    from paper_1410_4803_gb300 import ibs
    from helpers import pack_codes, random_codes
    rng = np.random.default_rng(31)
    n_panel, m, q, k = 300, 700, 4096, 4
    pcodes = random_codes(rng, n_panel, m)
    ctx = ibs.ibs_init(0)
    try:
        ibs.ibs_panel_load(ctx, pack_codes(pcodes), n_panel, m)
        reqs = []
        for i in range(3):
            qc = random_codes(np.random.default_rng(40 + i), q, m)
            out = (_pinned((q, n_panel, 4), torch.int32), _pinned((q, k), torch.int32), _pinned((q, k), torch.float64))
            reqs.append((qc, pack_codes(qc), out))
        ids = [ibs.ibs_query(ctx, qp, q, k, *out) for _, qp, out in reqs]
        for rid in ids:
            ibs.ibs_wait(ctx, rid, timeout_ms=120000)
        for qc, qp, (oc, oi, od) in reqs:
            ac, ai, ad = _pinned((q, n_panel, 4), torch.int32), _pinned((q, k), torch.int32), _pinned((q, k), torch.float64)
            ibs.ibs_query_sync(ctx, qp, q, k, ac, ai, ad)
            assert (oc.numpy() == ac.numpy()).all()
            assert (oi.numpy() == ai.numpy()).all()
            rows = np.arange(0, q, 97)
            wc, _ = oracle.ibs_block(qc, pcodes, rows=rows)
            assert (oc.numpy()[rows] == wc).all()
    finally:
        ibs.ibs_shutdown(ctx)
