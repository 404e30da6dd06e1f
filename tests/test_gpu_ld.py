"""GPU LD correlation (ibs_ld_r through the C ABI) against the oracle: N exact,
r within 1e-12 relative with NaN in the same places, on shapes around the
128-marker block, 64-marker half-block and 64-sample chunk edges, windows
shorter and longer than a block, degenerate markers, and a larger case."""
import numpy as np
import pytest

import oracle
from helpers import assert_dist_close, pack_codes, random_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1410_4803_gb300 import ibs
    c = ibs.ibs_init(0)
    yield c
    ibs.ibs_shutdown(c)


def _gpu_ld(ctx, codes, window, garbage_seed=None):
    import torch
    from paper_1410_4803_gb300 import ibs
    n, m = codes.shape
    rng = np.random.default_rng(garbage_seed) if garbage_seed is not None else None
    packed = torch.from_numpy(pack_codes(codes, garbage_rng=rng)).cuda()
    r, cnt = ibs.ld_r(ctx, packed, n, m, window)
    ibs.ibs_synchronize(ctx)
    return r.cpu().numpy(), cnt.cpu().numpy()


def _check(ctx, codes, window, garbage_seed=None):
    got_r, got_n = _gpu_ld(ctx, codes, window, garbage_seed)
    want_r, want_n = oracle.ld_r(codes, window)
    assert (got_n == want_n).all(), f"N differs at {np.argwhere(got_n != want_n)[:5]}"
    assert_dist_close(got_r, want_r)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 63, 64, 65, 130])
def test_edge_shapes(ctx, n):
    rng = np.random.default_rng(500 + n)
    for m in [1, 2, 63, 64, 65, 127, 128, 129, 200]:
        for window in [1, 3, 64, 65, 200]:
            _check(ctx, random_codes(rng, n, m, miss=0.08), window, garbage_seed=n * 31 + m)


def test_degenerate_markers(ctx):
    rng = np.random.default_rng(7)
    n, m = 150, 140
    codes = random_codes(rng, n, m)
    codes[:, 5] = codes[:, 4]                                   # duplicate: r = 1
    codes[:, 7] = np.where(codes[:, 6] == 0, 3, np.where(codes[:, 6] == 3, 0, codes[:, 6]))  # relabelled
    codes[:, 10] = 2                                            # all het: variance 0, NaN
    codes[:, 11] = 3                                            # monomorphic hom: NaN
    codes[:, 12] = 1                                            # all missing: N = 0
    codes[3, :] = 1                                             # one sample missing everywhere
    got_r, got_n = _gpu_ld(ctx, codes, 9)
    want_r, want_n = oracle.ld_r(codes, 9)
    assert (got_n == want_n).all()
    assert_dist_close(got_r, want_r)
    assert abs(got_r[4, 0] - 1.0) < 1e-12 and abs(got_r[6, 0] - 1.0) < 1e-12
    assert np.isnan(got_r[10, 0]) and np.isnan(got_r[11, 0]) and got_n[12, 0] == 0


def test_larger_case(ctx):
    """n = 4,100 samples (65 chunks, ragged), m = 1,500 markers, window 300."""
    rng = np.random.default_rng(8)
    codes = random_codes(rng, 4100, 1500, miss=0.02)
    _check(ctx, codes, 300)


def test_repeat_and_rejects(ctx):
    import torch
    from paper_1410_4803_gb300 import ibs
    rng = np.random.default_rng(9)
    codes = random_codes(rng, 70, 90)
    a = _gpu_ld(ctx, codes, 20)
    b = _gpu_ld(ctx, codes, 20)
    np.testing.assert_array_equal(a[0], b[0])
    packed = torch.from_numpy(pack_codes(codes)).cuda()
    out = torch.empty((90, 20), dtype=torch.float64, device="cuda")
    for n, m, w in [(70, 90, 0), (0, 90, 5), (1 << 24, 90, 5)]:
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_ld_r(ctx, packed, n, m, w, out)
        assert ei.value.status == ibs.IBS_EINVAL
