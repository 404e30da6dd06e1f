"""The seeded input generator: known-answer vectors, determinism and the
structure each workload promises (checked with the CPU oracle)."""
import os

import numpy as np

import oracle
from paper_1410_4803_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for ln in open(os.path.join(GOLDEN, "philox_kat.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        v = [int(x, 16) for x in ln.split()]
        out = synth.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_deterministic_and_subsettable():
    model = synth.plain_model(3000, 9, miss=0.02)
    s = synth.Samples.base(50)
    a = synth.generate(model, s, threads=1)
    b = synth.generate(model, s, threads=5)
    assert (a == b).all()
    # a subset of samples and a window of variants generate the same codes
    G = oracle.unpack(a, 50, 3000)
    sub = s.take([3, 17, 49, 0])
    w = synth.generate(model.window(1000, 700), sub)
    Gs = oracle.unpack(w, 4, 700)
    assert (Gs == G[[3, 17, 49, 0]][:, 1000:1700]).all()


def test_plain_rates():
    w = synth.plain_config2(n=512, m=20000)
    G = oracle.unpack(w.packed, w.n, w.m)
    miss = (G == 1).mean()
    # 2% i.i.d. plus 0.5% of variants at 30%: expected 0.02*0.995 + 0.3*0.005
    assert abs(miss - (0.02 * 0.995 + 0.3 * 0.005)) < 0.003
    hi = (G == 1).mean(axis=0) > 0.2
    assert 0.003 < hi.mean() < 0.008
    # A2 frequency per variant is folded to a MAF within [0.01, 0.5]
    nm = G != 1
    dose = np.where(G == 3, 2, np.where(G == 2, 1, 0))
    p = (dose * nm).sum(0) / (2 * nm.sum(0))
    maf = np.minimum(p, 1 - p)
    assert maf.mean() > 0.15 and maf.max() <= 0.6


def test_structured_relatives():
    w = synth.structured_config3(n_base_per_pop=40, m=4000, n_offspring=12, n_dup=6)
    G = oracle.unpack(w.packed, w.n, w.m)
    s = w.samples
    gid_to_idx = {int(g): i for i, g in enumerate(s.gid)}
    off = np.flatnonzero(s.kind == synth.OFFSPRING)
    dup = np.flatnonzero(s.kind == synth.DUPLICATE)
    assert off.size == 12 and dup.size == 6
    for t in off:
        src = gid_to_idx[int(s.src_gid[t])]
        c, _ = oracle.ibs_block(G, G, rows=[src], cols=[t])
        assert c[0, 0, 0] == 0  # a parent and child always share an allele
        assert c[0, 0, 3] > 0
    for t in dup:
        src = gid_to_idx[int(s.src_gid[t])]
        c, d = oracle.ibs_block(G, G, rows=[t], cols=np.arange(w.n))
        # 0.1% discordance: at most a handful of discordant sites of ~3900
        assert c[0, src, 0] + c[0, src, 1] <= 20
        # the duplicate's nearest other sample is its source
        d = d[0].copy()
        d[t] = np.inf
        assert int(np.nanargmin(d)) == src
    # subpopulation structure: within-population pairs are closer on average
    base = np.flatnonzero(s.kind == synth.BASE)
    c, d = oracle.ibs_block(G, G, rows=base[:40], cols=base)
    same = s.pop[base[:40]][:, None] == s.pop[base][None, :]
    offd = ~np.eye(40, base.size, dtype=bool)
    assert d[same & offd].mean() < d[~same].mean()


def test_batch_subsets_shape():
    subs = synth.batch_subsets(pool_n=1000, pool_m=5000, n_subsets=10, n_range=(20, 300), m_range=(100, 2000))
    for sb in subs:
        assert 20 <= sb.n <= 300 and np.unique(sb.sample_idx).size == sb.n
        assert 0 <= sb.var_begin and sb.var_begin + sb.var_len <= 5000


def test_query_sizes_log_uniform():
    q = synth.serving_query_sizes(5000)
    assert q.min() >= 1 and q.max() <= 512
    assert np.median(q) < 64 and (q > 256).mean() > 0.05
