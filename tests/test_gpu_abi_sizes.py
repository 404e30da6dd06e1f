"""ibs_compute_sz: the caller's buffer sizes are checked before any work.
Exact sizes give the same counts and distances as ibs_compute; one byte less
in any buffer is refused with IBS_EINVAL and leaves the outputs untouched."""
import numpy as np
import pytest

import oracle
from helpers import pack_codes, random_codes

pytestmark = pytest.mark.gpu


def test_sizes_checked_and_results_equal():
    import torch
    from paper_1410_4803_gb300 import ibs
    rng = np.random.default_rng(41)
    n, m = 133, 700
    codes = random_codes(rng, n, m, miss=0.05)
    packed = torch.from_numpy(pack_codes(codes)).cuda()
    P = n * (n + 1) // 2
    ctx = ibs.ibs_init(0)
    try:
        c_ref = torch.empty((P, 4), dtype=torch.int32, device="cuda")
        d_ref = torch.empty(P, dtype=torch.float64, device="cuda")
        ibs.ibs_compute(ctx, packed, n, m, c_ref, d_ref)
        c = torch.full((P, 4), -5, dtype=torch.int32, device="cuda")
        d = torch.full((P,), -5.0, dtype=torch.float64, device="cuda")
        pb, cb, db = packed.numel(), P * 16, P * 8
        assert pb == m * ((n + 3) // 4)
        for bad in [(pb - 1, cb, db), (pb, cb - 1, db), (pb, cb, db - 1)]:
            with pytest.raises(ibs.IbsError):
                ibs.ibs_compute_sz(ctx, packed, bad[0], n, m, c, bad[1], d, bad[2])
        ibs.ibs_synchronize(ctx)
        assert (c == -5).all() and (d == -5.0).all()
        ibs.ibs_compute_sz(ctx, packed, pb, n, m, c, cb, d, db)
        # without distances, the distance size is not checked
        c2 = torch.empty_like(c)
        ibs.ibs_compute_sz(ctx, packed, pb, n, m, c2, cb, None, 0)
        ibs.ibs_synchronize(ctx)
        assert torch.equal(c, c_ref) and torch.equal(c2, c_ref)
        assert torch.equal(d, d_ref)
        oc, _, _ = oracle.ibs_triangle_from_codes(codes)
        assert (c.cpu().numpy() == oc).all()
    finally:
        ibs.ibs_shutdown(ctx)
