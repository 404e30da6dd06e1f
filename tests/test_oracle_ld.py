"""Pins of the oracle's linkage-disequilibrium correlation (paper, "Bitwise
parallelism", the correlation coefficient r between two markers with missing
calls): a hand-worked example, an independent route through numpy.corrcoef on
the samples where both calls are present, the paper's mean form written out,
and invariants (a duplicated marker, A1/A2 relabelling, monomorphic and
all-missing markers, sample order)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ld_hand_example.txt")


def _read_golden():
    G, slots, window = [], [], None
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "window":
            window = int(t[1])
        elif t[0] == "sample":
            G.append([int(x) for x in t[2:]])
        elif t[0] == "slot":
            slots.append((int(t[1]), int(t[2]), float(t[3]), int(t[4])))
    return np.array(G, dtype=np.uint8), window, slots


def test_hand_example():
    G, window, slots = _read_golden()
    r, cnt = oracle.ld_r(G, window)
    for a, d, want_r, want_n in slots:
        assert cnt[a, d] == want_n
        if np.isnan(want_r):
            assert np.isnan(r[a, d])
        else:
            assert abs(r[a, d] - want_r) <= 1e-15


def _major_x(codes):
    """x of one marker (sample vector): +1 hom major, -1 hom minor, 0 het; NaN missing."""
    a1 = (codes == 0).sum() >= (codes == 3).sum()
    x = np.where(codes == 0, 1.0, np.where(codes == 3, -1.0, 0.0))
    if not a1:
        x = -x
    x[codes == 1] = np.nan
    return x


def _random(rng, n, m, miss=0.05):
    G = rng.choice(np.array([0, 2, 3], dtype=np.uint8), size=(n, m), p=[0.45, 0.35, 0.2])
    G[rng.random((n, m)) < miss] = 1
    return G


def test_matches_numpy_corrcoef_on_common_samples():
    rng = np.random.default_rng(11)
    for n, m in [(7, 5), (40, 12), (301, 9)]:
        G = _random(rng, n, m)
        G[:, 2] = G[:, 1]                    # a duplicated marker
        window = m - 1
        r, cnt = oracle.ld_r(G, window)
        X = np.stack([_major_x(G[:, k]) for k in range(m)], axis=1)
        for a in range(m):
            for d in range(window):
                b = a + 1 + d
                if b >= m:
                    assert np.isnan(r[a, d]) and cnt[a, d] == 0
                    continue
                both = ~np.isnan(X[:, a]) & ~np.isnan(X[:, b])
                assert cnt[a, d] == both.sum()
                x, y = X[both, a], X[both, b]
                if both.sum() == 0 or x.std() == 0 or y.std() == 0:
                    assert np.isnan(r[a, d])
                    continue
                want = np.corrcoef(x, y)[0, 1]
                assert abs(r[a, d] - want) <= 1e-12, (n, m, a, b)


def test_paper_mean_form():
    """The paper writes r with means over S_xy; the oracle's integer form is
    the same value up to rounding."""
    rng = np.random.default_rng(12)
    G = _random(rng, 500, 8)
    r, _ = oracle.ld_r(G, 7)
    X = np.stack([_major_x(G[:, k]) for k in range(8)], axis=1)
    for a in range(8):
        for b in range(a + 1, 8):
            both = ~np.isnan(X[:, a]) & ~np.isnan(X[:, b])
            x, y = X[both, a], X[both, b]
            N = both.sum()
            xb, yb, x2, y2 = x.sum() / N, y.sum() / N, (x * x).sum() / N, (y * y).sum() / N
            want = ((x * y).sum() / N - xb * yb) / np.sqrt((x2 - xb * xb) * (y2 - yb * yb))
            assert abs(r[a, b - a - 1] - want) <= 1e-12


def test_invariants():
    rng = np.random.default_rng(13)
    n, m = 120, 10
    G = _random(rng, n, m)
    G[:, 3] = G[:, 2]                                        # duplicate: r = 1
    G[:, 5] = np.where(G[:, 4] == 0, 3, np.where(G[:, 4] == 3, 0, G[:, 4]))  # A1/A2 relabelled copy
    G[:, 7] = 2                                              # monomorphic (all het): NaN
    G[:, 8] = 1                                              # all missing: N = 0, NaN
    r, cnt = oracle.ld_r(G, m - 1)
    assert abs(r[2, 0] - 1.0) <= 1e-15
    assert abs(r[4, 0] - 1.0) <= 1e-15                       # orientation follows the major allele
    assert np.isnan(r[6, 0]) and np.isnan(r[7, 0]) and np.isnan(r[7, 1])
    assert (cnt[0:8, :] >= 0).all() and cnt[7, 0] == 0 and cnt[0, 7] == 0
    finite = r[~np.isnan(r)]
    assert (np.abs(finite) <= 1.0 + 1e-15).all()
    # relabelling any marker leaves every r unchanged
    G2 = G.copy()
    G2[:, 1] = np.where(G[:, 1] == 0, 3, np.where(G[:, 1] == 3, 0, G[:, 1]))
    r2, _ = oracle.ld_r(G2, m - 1)
    np.testing.assert_allclose(r2, r, rtol=0, atol=1e-15)
    # sample order does not matter
    perm = rng.permutation(n)
    r3, cnt3 = oracle.ld_r(G[perm], m - 1)
    np.testing.assert_allclose(r3, r, rtol=0, atol=1e-14)
    assert (cnt3 == cnt).all()


def test_threads_do_not_change_results():
    rng = np.random.default_rng(14)
    G = _random(rng, 200, 50)
    r1, c1 = oracle.ld_r(G, 10, threads=1)
    r8, c8 = oracle.ld_r(G, 10, threads=8)
    np.testing.assert_array_equal(r1, r8)
    assert (c1 == c8).all()


@pytest.mark.parametrize("window", [0, -1])
def test_rejects_bad_window(window):
    with pytest.raises(ValueError):
        oracle.ld_r(np.zeros((3, 3), np.uint8), window)
