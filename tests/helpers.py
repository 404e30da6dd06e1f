"""Shared test helpers: packing codes, device upload, GPU calls through the C ABI."""
import numpy as np


def pack_codes(codes: np.ndarray, garbage_rng=None) -> np.ndarray:
    """codes [n][m] (0..3) -> variant-major packed bytes [m][ceil(n/4)]."""
    n, m = codes.shape
    nb = (n + 3) // 4
    out = np.zeros((m, nb), dtype=np.uint8)
    for s in range(n):
        out[:, s // 4] |= (codes[s].astype(np.uint8) << (2 * (s % 4))).astype(np.uint8)
    if garbage_rng is not None and n % 4:
        mask = (0xFF << (2 * (n % 4))) & 0xFF
        out[:, nb - 1] |= (garbage_rng.integers(0, 256, m).astype(np.uint8) & mask)
    return out


def random_codes(rng, n, m, miss=0.03):
    p = rng.uniform(0.02, 0.5, m)
    d = (rng.random((n, m)) < p).astype(np.int64) + (rng.random((n, m)) < p).astype(np.int64)
    codes = np.array([0, 2, 3], dtype=np.uint8)[d]
    codes[rng.random((n, m)) < miss] = 1
    return codes


def gpu_compute(ctx, packed_np, n, m, square=False, stream=None):
    import torch
    from paper_1410_4803_gb300 import ibs
    packed = torch.from_numpy(np.ascontiguousarray(packed_np)).cuda()
    counts, dist = ibs.compute(ctx, packed, n, m, square=square, stream=stream)
    ibs.ibs_synchronize(ctx, stream)
    return counts.cpu().numpy(), dist.cpu().numpy()


def assert_dist_close(got, want, rtol=1e-12):
    """Distances: NaN exactly where expected, else within rtol relative error."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape
    nan_g, nan_w = np.isnan(got), np.isnan(want)
    assert (nan_g == nan_w).all(), "NaN pattern differs"
    ok = ~nan_w
    denom = np.maximum(np.abs(want[ok]), 1e-300)
    rel = np.abs(got[ok] - want[ok]) / denom
    assert rel.size == 0 or rel.max() <= rtol, f"max relative error {rel.max()}"
