"""The allocation-free entry point, ibs_compute_noalloc.

It serves callers that cannot allocate device memory at the moment they need
IBS counts: work recorded into a CUDA graph (allocation is not allowed while a
stream is being captured), applications whose memory pool has reserved the
whole GPU, and latency-bound services that allocate only once at start-up.
It keeps its bit-plane scratch in a fixed array inside the library instead.

The test calls it through the C ABI twice in a row, on two different inputs,
and compares each result with the regular entry point, ibs_compute, and with
the CPU oracle: counts bit for bit and distances within 1e-12 relative error.
The second input is smaller than the first, so stale scratch contents from the
first call would show up as wrong counts.  Both are small triangles whose
marker axis is split (partial counts in the scratch after the planes); the
third wants a split but its partial counts do not fit beside its planes, so it
runs unsplit.  After each call the status query (ibs_noalloc_status) must
report that no bounded device wait expired.
"""
import numpy as np
import pytest

from helpers import assert_dist_close, pack_codes, random_codes

pytestmark = pytest.mark.gpu


def _noalloc(packed_np, n, m):
    import torch
    from paper_1410_4803_gb300 import ibs
    torch.cuda.set_device(0)
    packed = torch.from_numpy(np.ascontiguousarray(packed_np)).cuda()
    P = n * (n + 1) // 2
    counts = torch.empty((P, 4), dtype=torch.int32, device="cuda")
    dist = torch.empty(P, dtype=torch.float64, device="cuda")
    ibs.ibs_compute_noalloc(packed, n, m, counts, dist)
    ibs.ibs_noalloc_status()  # raises IbsError(IBS_ETIMEOUT) if a device wait expired
    torch.cuda.synchronize()
    return counts.cpu().numpy(), dist.cpu().numpy()


def _regular(packed_np, n, m):
    import torch
    from paper_1410_4803_gb300 import ibs
    ctx = ibs.ibs_init(0)
    try:
        packed = torch.from_numpy(np.ascontiguousarray(packed_np)).cuda()
        counts, dist = ibs.compute(ctx, packed, n, m)
        ibs.ibs_synchronize(ctx)
        return counts.cpu().numpy(), dist.cpu().numpy()
    finally:
        ibs.ibs_shutdown(ctx)


def test_noalloc_matches_ibs_compute_on_two_calls():
    import oracle
    rng = np.random.default_rng(2024)
    # 16 blocks (5 splits), 6 blocks (14 splits, the second call smaller than the
    # first), 32 blocks with 41 MB of planes + 32 MB of partial counts (unsplit)
    cases = [(1000, 20000), (333, 5001), (2000, 40000)]
    for n, m in cases:
        packed = pack_codes(random_codes(rng, n, m, miss=0.04), garbage_rng=rng)
        got_c, got_d = _noalloc(packed, n, m)
        want_c, want_d = _regular(packed, n, m)
        assert (got_c == want_c).all(), f"counts differ from ibs_compute for n={n} m={m}"
        assert_dist_close(got_d, want_d)
        ora_c, ora_d = oracle.ibs_triangle(packed, n, m)
        assert (got_c == ora_c).all(), f"counts differ from the oracle for n={n} m={m}"
        assert_dist_close(got_d, ora_d)


def test_noalloc_rejects_host_buffers_before_any_work():
    import torch
    from paper_1410_4803_gb300 import ibs
    torch.cuda.set_device(0)
    n, m = 64, 100
    host_packed = np.zeros((m, n // 4), dtype=np.uint8)
    counts = torch.empty((n * (n + 1) // 2, 4), dtype=torch.int32, device="cuda")
    host_counts = np.empty((n * (n + 1) // 2, 4), dtype=np.int32)
    dev_packed = torch.zeros((m, n // 4), dtype=torch.uint8, device="cuda")
    for args in ((host_packed, counts), (dev_packed, host_counts)):
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_compute_noalloc(args[0], n, m, args[1], None)
        assert ei.value.status == ibs.IBS_EINVAL
    ibs.ibs_noalloc_status()


def test_noalloc_rejects_inputs_beyond_its_scratch():
    import torch
    from paper_1410_4803_gb300 import ibs
    torch.cuda.set_device(0)
    n, m = 4096, 40000  # planes need about 80 MiB, more than the 64 MiB scratch
    packed = torch.zeros((m, n // 4), dtype=torch.uint8, device="cuda")
    counts = torch.empty((n * (n + 1) // 2, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(ibs.IbsError) as ei:
        ibs.ibs_compute_noalloc(packed, n, m, counts, None)
    assert ei.value.status == ibs.IBS_EINVAL
