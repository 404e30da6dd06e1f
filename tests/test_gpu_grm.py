"""GPU genomic relationship matrix (ibs_grm through the C ABI) against the
oracle.  The tolerance is the bound stated with ibs_grm, computed per pair:
with z the standardised genotypes (0 where a call is missing or the marker
unused), S = sum |z_j z_k| and T = sum (|z_j| + |z_k|) over the markers both
samples share,
  |A_gpu - A| <= (27 * 2^-22 * S + 2^-25 * T) / N_jk
(FP16 hi/lo split: 3 * 2^-22 per product; 24 FP32 MMA accumulations per
128-marker segment at 2^-22 each; the segments are summed in float-float), and
NaN exactly where no marker is shared.  Cases: shapes around the 128-sample
block, the 16-marker chunk and the 128-marker segment; missing calls;
monomorphic and all-missing markers; samples without calls; a larger case; and
the full-size workload (4,096 samples x 100,000 markers) on sampled rows."""
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


def _gpu_grm(ctx, codes, garbage_seed=None):
    import torch
    from paper_1410_4803_gb300 import ibs
    n, m = codes.shape
    rng = np.random.default_rng(garbage_seed) if garbage_seed is not None else None
    packed = torch.from_numpy(pack_codes(codes, garbage_rng=rng)).cuda()
    out = ibs.grm(ctx, packed, n, m)
    ibs.ibs_synchronize(ctx)
    return out.cpu().numpy()


def _standardised(codes):
    """z and V' of the formula, in float64 (for the tolerance only)."""
    x = np.where(codes == 0, 2.0, np.where(codes == 2, 1.0, 0.0))
    present = codes != 1
    calls = present.sum(axis=0)
    p = np.where(calls > 0, (x * present).sum(axis=0) / np.maximum(2 * calls, 1), 0.0)
    used = (p > 0) & (p < 1)
    keep = present & used
    z = np.where(keep, (x - 2 * p) / np.sqrt(np.where(used, 2 * p * (1 - p), 1.0)), 0.0)
    return z, keep.astype(np.float64)


def _bound(codes, rows=None, step=8192):
    """Per-pair bound (rows x all samples, or all x all), summed over marker
    ranges so that the full-size case stays within a few GB of host memory."""
    n, m = codes.shape
    r = np.arange(n) if rows is None else np.asarray(rows)
    S = np.zeros((r.size, n))
    T = np.zeros((r.size, n))
    N = np.zeros((r.size, n))
    for i0 in range(0, m, step):
        z, v = _standardised(codes[:, i0:i0 + step])
        a = np.abs(z)
        S += a[r] @ a.T
        T += a[r] @ v.T + v[r] @ a.T
        N += v[r] @ v.T
    with np.errstate(invalid="ignore", divide="ignore"):
        return (27 * 2.0 ** -22 * S + 2.0 ** -25 * T) / N, N


def _assert_within(got, want, bound):
    nan = np.isnan(want)
    assert (np.isnan(got) == nan).all(), f"NaN pattern differs at {np.argwhere(np.isnan(got) != nan)[:5]}"
    err = np.abs(got[~nan] - want[~nan])
    tol = bound[~nan] + 1e-13 * np.abs(want[~nan])
    bad = err > tol
    assert not bad.any(), f"{bad.sum()} entries outside the bound; worst excess {(err - tol).max():.3e}"
    return float(err.max()) if err.size else 0.0


def _check(ctx, codes, garbage_seed=None):
    n = codes.shape[0]
    got = _gpu_grm(ctx, codes, garbage_seed)
    want = oracle.grm(codes)
    bound, _ = _bound(codes)
    return _assert_within(got, want, bound[np.triu_indices(n)])


@pytest.mark.parametrize("n", [1, 2, 127, 128, 129, 300])
def test_edge_shapes(ctx, n):
    rng = np.random.default_rng(700 + n)
    for m in [1, 15, 16, 17, 127, 128, 129, 300]:
        _check(ctx, random_codes(rng, n, m, miss=0.06), garbage_seed=n * 13 + m)


def test_segments_and_ragged_tail(ctx):
    """Several 128-marker segments and a ragged last chunk (m = 1,000 = 62.5
    chunks), over three sample blocks with a ragged one."""
    rng = np.random.default_rng(71)
    err = _check(ctx, random_codes(rng, 333, 1000, miss=0.04))
    assert err < 1e-5


def test_degenerate_markers_and_samples(ctx):
    rng = np.random.default_rng(72)
    n, m = 140, 260
    codes = random_codes(rng, n, m, miss=0.05)
    codes[:, 3] = 3                      # monomorphic hom A2: left out
    codes[:, 4] = 0                      # monomorphic hom A1: left out
    codes[:, 5] = 1                      # no calls: left out
    codes[:, 6] = 2                      # all het: p = 1/2, used
    codes[9, :] = 1                      # a sample without calls: NaN row and column
    codes[20, :] = 1
    codes[20, 10] = 0                    # samples 20 and 21 share no marker
    codes[21, :] = 1
    codes[21, 11] = 3
    got = _gpu_grm(ctx, codes)
    want = oracle.grm(codes)
    bound, _ = _bound(codes)
    _assert_within(got, want, bound[np.triu_indices(n)])
    assert np.isnan(got[oracle.tri_index(9, 9, n)])
    assert np.isnan(got[oracle.tri_index(20, 21, n)])
    assert np.isfinite(got[oracle.tri_index(20, 20, n)])


def test_all_markers_monomorphic_is_nan(ctx):
    codes = np.full((70, 40), 3, np.uint8)
    codes[::3] = 1
    assert np.isnan(_gpu_grm(ctx, codes)).all()


def test_larger_case(ctx):
    """600 samples (5 blocks, ragged) x 20,000 markers (157 segments)."""
    rng = np.random.default_rng(73)
    err = _check(ctx, random_codes(rng, 600, 20000, miss=0.02))
    assert err < 1e-5


def test_repeat_is_deterministic_and_rejects(ctx):
    import torch
    from paper_1410_4803_gb300 import ibs
    rng = np.random.default_rng(74)
    codes = random_codes(rng, 150, 500)
    a = _gpu_grm(ctx, codes)
    b = _gpu_grm(ctx, codes)
    np.testing.assert_array_equal(a, b)
    packed = torch.from_numpy(pack_codes(codes)).cuda()
    out = torch.empty(150 * 151 // 2, dtype=torch.float64, device="cuda")
    for n, m in [(0, 500), (150, 0), (150, 1 << 24)]:
        with pytest.raises(ibs.IbsError):
            ibs.ibs_grm(ctx, packed, n, m, out)
    with pytest.raises(ibs.IbsError):
        ibs.ibs_grm(ctx, packed.cpu(), 150, 500, out)


def test_fullsize_sampled_rows(ctx):
    """The benchmarked workload (the plain genotypes: 4,096 samples x 100,000
    markers, MAF ~ U(0.01, 0.5), 2% missing plus 0.5% of markers at 30%):
    sampled rows, every column, against the oracle's row sampler."""
    import torch
    from paper_1410_4803_gb300 import ibs, synth
    w = synth.plain_config2()
    n, m = w.n, w.m
    out = ibs.grm(ctx, torch.from_numpy(w.packed).cuda(), n, m)
    ibs.ibs_synchronize(ctx)
    got = out.cpu().numpy()
    codes = oracle.unpack(w.packed, n, m)
    rows = np.array([0, 1, 127, 128, 2047, 3000, 4095])
    want = oracle.grm_rows(codes, rows)
    bound, _ = _bound(codes, rows)
    k = np.arange(n)
    got_rows = np.stack([got[oracle.tri_index(np.minimum(j, k), np.maximum(j, k), n)] for j in rows])
    err = _assert_within(got_rows, want, bound)
    assert err < 1e-5
