"""Parity at the workloads' full sizes, in the launch configuration the bench
times (one ibs_compute per matrix).  The oracle checks sampled outputs one by
one; properties that hold for every pair are checked on the whole output on
the device."""
import numpy as np
import pytest

import oracle
from helpers import assert_dist_close

pytestmark = pytest.mark.gpu


_CONFIG3 = []


def _config3():
    from paper_1410_4803_gb300 import synth
    if not _CONFIG3:
        _CONFIG3.append(synth.structured_config3())
    return _CONFIG3[0]


def _whole_output_invariants(counts, n, nonmiss):
    """IBS0+IBS1+IBS2 = N, all counts >= 0, diagonal = (0, 0, N_i, N_i)."""
    import torch
    c = counts
    assert bool((c[:, 0] + c[:, 1] + c[:, 2] == c[:, 3]).all())
    assert bool((c >= 0).all())
    i = torch.arange(n, device=c.device, dtype=torch.int64)
    diag = c[i * n - i * (i - 1) // 2]
    nm = torch.from_numpy(nonmiss.astype(np.int32)).to(c.device)
    assert bool((diag[:, 0] == 0).all() and (diag[:, 1] == 0).all())
    assert bool((diag[:, 2] == nm).all() and (diag[:, 3] == nm).all())


_FLAGS = {"popc": "IBS_KERNEL_CSA", "tc8": ("IBS_KERNEL_TC", "IBS_TC_FP8"), "tc4": ("IBS_KERNEL_TC", "IBS_TC_FP4")}


def _flags(ibs, kernel):
    f = _FLAGS[kernel]
    return getattr(ibs, f) if isinstance(f, str) else getattr(ibs, f[0]) | getattr(ibs, f[1])


@pytest.mark.parametrize("kernel", ["popc", "tc8", "tc4"])
def test_plain_n4096_m100000_sampled_rows(kernel):
    import torch
    from paper_1410_4803_gb300 import ibs, synth
    w = synth.plain_config2()
    n, m = w.n, w.m
    ctx = ibs.ibs_init(0, flags=_flags(ibs, kernel))
    try:
        counts, dist = ibs.compute(ctx, torch.from_numpy(w.packed).cuda(), n, m)
        ibs.ibs_synchronize(ctx)
        G = oracle.unpack(w.packed, n, m)
        _whole_output_invariants(counts, n, (G != 1).sum(axis=1))
        rows = np.array([0, 1, 63, 64, 65, 2047, 2048, 4031, 4094, 4095] +
                        list(np.random.default_rng(1).choice(n, 14, replace=False)))
        wc, wd = oracle.ibs_block(G, G, rows=rows)
        c_host = counts.cpu().numpy()
        d_host = dist.cpu().numpy()
        for t, i in enumerate(rows):
            j = np.arange(i, n)
            p = oracle.tri_index(i, j, n)
            assert (c_host[p] == wc[t, i:]).all(), f"row {i} differs"
            assert_dist_close(d_host[p], wd[t, i:])
    finally:
        ibs.ibs_shutdown(ctx)


@pytest.mark.parametrize("kernel", ["popc", "tc8", "tc4"])
def test_structured_n20000_m500000_sampled_pairs(kernel):
    """Five subpopulations, injected parent-offspring pairs and duplicates: the
    oracle checks a block of sampled pairs plus every relative pair.  With
    m = 500,000 the counts reach 2^19, so the tensor-core forms' FP32
    accumulation is checked far above 2^14."""
    import torch
    from paper_1410_4803_gb300 import ibs, synth
    w = _config3()
    n, m = w.n, w.m
    ctx = ibs.ibs_init(0, flags=_flags(ibs, kernel))
    try:
        counts, dist = ibs.compute(ctx, torch.from_numpy(w.packed).cuda(), n, m)
        ibs.ibs_synchronize(ctx)
        s = w.samples
        gid = {int(g): i for i, g in enumerate(s.gid)}
        rel = [(gid[int(s.src_gid[t])], int(t)) for t in np.flatnonzero(s.kind != synth.BASE)]
        rng = np.random.default_rng(2)
        pick = np.unique(np.concatenate([rng.choice(n, 40, replace=False), [0, 63, 64, 19999],
                                         [a for a, _ in rel[:20]], [b for _, b in rel[:20]]]))
        G = oracle.unpack_subset(w.packed, n, m, pick, 0, m)
        wc, wd = oracle.ibs_block(G, G)
        pos = {int(v): k for k, v in enumerate(pick)}
        ii, jj = np.triu_indices(pick.size)
        a, b = pick[ii], pick[jj]
        p = torch.from_numpy(oracle.tri_index(a, b, n)).cuda()
        got_c = counts[p].cpu().numpy()
        got_d = dist[p].cpu().numpy()
        assert (got_c == wc[ii, jj]).all()
        assert_dist_close(got_d, wd[ii, jj])
        # every injected relative: parents and offspring never share zero alleles
        pr = torch.from_numpy(oracle.tri_index(np.array([min(x) for x in rel]), np.array([max(x) for x in rel]), n)).cuda()
        rc = counts[pr].cpu().numpy()
        kinds = s.kind[[b for _, b in rel]]
        assert (rc[kinds == synth.OFFSPRING, 0] == 0).all()
        assert (rc[kinds == synth.DUPLICATE, 0] + rc[kinds == synth.DUPLICATE, 1] < 0.003 * m).all()
        del pos
    finally:
        ibs.ibs_shutdown(ctx)


@pytest.mark.parametrize("kernel", ["tc8", "tc4"])
def test_tensor_core_long_marker_range_is_split(kernel):
    """m = 2,200,000 markers: one FP32 accumulation would exceed 2^24 (its
    third accumulator grows by up to 6 per marker), so every tile is split over
    K into pieces of at most 2^21 markers whose counts are added as integers.
    The counts reach 2.2e6 and must equal the oracle on sampled rows."""
    import torch
    from paper_1410_4803_gb300 import ibs
    from helpers import pack_codes, random_codes
    rng = np.random.default_rng(31)
    n, m = 130, 2_200_000
    codes = random_codes(rng, n, m, miss=0.01)
    codes[5] = 3          # hom A2 everywhere: IBS0 = N against sample 6
    codes[6] = 0
    packed = pack_codes(codes)
    ctx = ibs.ibs_init(0, flags=_flags(ibs, kernel))
    try:
        counts, dist = ibs.compute(ctx, torch.from_numpy(packed).cuda(), n, m)
        ibs.ibs_synchronize(ctx)
        assert ibs.ibs_last_launch_info(ctx)["splits"] > 1
        rows = np.array([0, 5, 6, 64, 127, 129])
        wc, wd = oracle.ibs_block(codes, codes, rows=rows)
        c_host, d_host = counts.cpu().numpy(), dist.cpu().numpy()
        for t, i in enumerate(rows):
            j = np.arange(i, n)
            p = oracle.tri_index(i, j, n)
            assert (c_host[p] == wc[t, i:]).all(), f"row {i} differs"
            assert_dist_close(d_host[p], wd[t, i:])
        assert c_host[oracle.tri_index(5, 6, n), 0] == m
    finally:
        ibs.ibs_shutdown(ctx)
