"""GPU complete-linkage clustering (ibs_cluster_complete through the C ABI)
against the oracle on the same distance triangle: identical merges (ids,
heights, sizes) on tie-free distances, on IBS distances with many ties, with
NaN distances, and at a few thousand samples."""
import numpy as np
import pytest

import oracle
from helpers import pack_codes, random_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1410_4803_gb300 import ibs
    c = ibs.ibs_init(0)
    yield c
    ibs.ibs_shutdown(c)


def _tri(D):
    n = D.shape[0]
    iu = np.triu_indices(n)
    return np.ascontiguousarray(D[iu])


def _gpu(ctx, tri, n):
    import torch
    from paper_1410_4803_gb300 import ibs
    z = ibs.cluster_complete(ctx, torch.from_numpy(tri).cuda(), n)
    ibs.ibs_synchronize(ctx)
    return z.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 33, 500, 1100])
def test_tie_free_distances(ctx, n):
    rng = np.random.default_rng(40 + n)
    A = rng.random((n, n))
    D = (A + A.T) / 2
    np.fill_diagonal(D, 0)
    tri = _tri(D)
    np.testing.assert_array_equal(_gpu(ctx, tri, n), oracle.complete_linkage(tri, n))


def test_ibs_distances_with_ties_and_nan(ctx):
    import torch
    from paper_1410_4803_gb300 import ibs
    rng = np.random.default_rng(41)
    n, m = 300, 400
    codes = random_codes(rng, n, m)
    codes[:, :150] = 3              # few informative markers: many equal distances
    codes[7] = 1                    # all-missing sample: NaN distances
    codes[20] = codes[19]           # a duplicate pair: distance 0
    counts, dist = ibs.compute(ctx, torch.from_numpy(pack_codes(codes)).cuda(), n, m)
    ibs.ibs_synchronize(ctx)
    tri = dist.cpu().numpy()
    got = _gpu(ctx, tri, n)
    want = oracle.complete_linkage(tri, n)
    np.testing.assert_array_equal(got, want)
    assert np.isinf(got[-1, 2])
    assert got[0, 2] == 0.0 and {int(got[0, 0]), int(got[0, 1])} == {19, 20}


def test_larger_matrix(ctx):
    rng = np.random.default_rng(42)
    n = 2500
    D = np.round(rng.random((n, n)), 3)   # ties
    D = np.maximum(D, D.T)
    np.fill_diagonal(D, 0)
    tri = _tri(D)
    np.testing.assert_array_equal(_gpu(ctx, tri, n), oracle.complete_linkage(tri, n))


def test_rejects(ctx):
    import torch
    from paper_1410_4803_gb300 import ibs
    d = torch.zeros(6, dtype=torch.float64, device="cuda")
    z = torch.empty((2, 4), dtype=torch.float64, device="cuda")
    for n in [0, (1 << 17) + 1]:
        with pytest.raises(ibs.IbsError) as ei:
            ibs.ibs_cluster_complete(ctx, d, n, z)
        assert ei.value.status == ibs.IBS_EINVAL
