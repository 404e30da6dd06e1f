"""A bounded device-side wait that runs out: error status, no trap, usable context.

Failure handling of the pair kernels: every wait on a pipeline barrier is
bounded by %globaltimer; when one runs out the kernel records IBS_ETIMEOUT in
the context's status word, stops issuing work, waits (with the full bound)
for the copies and MMAs it already issued, frees its tensor memory and
returns.  The test sets a 1 ns bound through the test hook, so the first
wait that is not already over (an operand stage, the accumulators) runs out,
in the one-SM persistent kernel and in the two-SM kernel (whose waiter warp
then stops waiting but keeps releasing its MMA warp until the work list
ends); ibs_synchronize must then
report IBS_ETIMEOUT, and the next call on the same context with the default
bound must be bit-exact against the oracle.  The failure is made on the
device with a short limit only: nothing faults, traps or hangs.
"""
import numpy as np
import pytest

from helpers import assert_dist_close, pack_codes, random_codes

pytestmark = pytest.mark.gpu


def _run(ctx, packed_dev, n, m):
    from paper_1410_4803_gb300 import ibs
    counts, dist = ibs.compute(ctx, packed_dev, n, m)
    return counts, dist


@pytest.mark.parametrize("n,m,kernel", [(200, 60_000, "tc-persistent"), (300, 200_000, "tc-pair")])
def test_short_wait_limit_reports_timeout_and_context_recovers(n, m, kernel):
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs
    rng = np.random.default_rng(77)
    codes = random_codes(rng, n, m, miss=0.03)
    packed = pack_codes(codes, garbage_rng=rng)
    ctx = ibs.ibs_init(0)
    try:
        assert ibs.ibs_compute_kernel(ctx, n, m) == kernel
        dev = torch.from_numpy(packed).cuda()
        ibs.ibs_test_set_wait_limit(ctx, 1)  # 1 ns: the first wait that is not already over runs out
        _run(ctx, dev, n, m)
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_synchronize(ctx)
        assert ei.value.status == ibs.IBS_ETIMEOUT
        # the default bound again: the same context computes exact counts
        ibs.ibs_test_set_wait_limit(ctx, 0)
        counts, dist = _run(ctx, dev, n, m)
        ibs.ibs_synchronize(ctx)
        got_c, got_d = counts.cpu().numpy(), dist.cpu().numpy()
    finally:
        ibs.ibs_shutdown(ctx)
    want_c, want_d = oracle.ibs_triangle(packed, n, m)
    assert (got_c == want_c).all()
    assert_dist_close(got_d, want_d)


def test_wait_limit_argument_checks():
    from paper_1410_4803_gb300 import ibs
    ctx = ibs.ibs_init(0)
    try:
        for bad in (-1, 3_000_000_000):
            with pytest.raises(ibs.IbsError) as ei:
                ibs.ibs_test_set_wait_limit(ctx, bad)
            assert ei.value.status == ibs.IBS_EINVAL
    finally:
        ibs.ibs_shutdown(ctx)
