"""Pins of the oracle's genomic relationship matrix (paper, "Partial sum
lookup", the GCTA matrix as a weighted sum of per-marker cases): a
hand-worked example, an independent route through numpy (standardised
genotype matrix with missing calls zeroed, Z Z^T divided by the pair counts),
and invariants (allele relabelling, monomorphic markers ignored, sample
order, thread count, NaN without shared markers)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grm_hand_example.txt")


def test_hand_example():
    G, want = [], {}
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "sample":
            G.append([int(x) for x in t[2:]])
        elif t[0] == "pair":
            want[(int(t[1]), int(t[2]))] = float(t[3])
    G = np.array(G, dtype=np.uint8)
    n = G.shape[0]
    got = oracle.grm(G)
    for (j, k), v in want.items():
        assert abs(got[oracle.tri_index(j, k, n)] - v) <= 1e-15


def _numpy_grm(G):
    x = np.where(G == 0, 2.0, np.where(G == 2, 1.0, 0.0))
    present = G != 1
    calls = present.sum(axis=0)
    p = np.where(calls > 0, (x * present).sum(axis=0) / np.maximum(2 * calls, 1), 0.0)
    used = (p > 0) & (p < 1)
    Z = np.where(present & used, (x - 2 * p) / np.sqrt(np.where(used, 2 * p * (1 - p), 1.0)), 0.0)
    Vp = (present & used).astype(np.float64)
    num, den = Z @ Z.T, Vp @ Vp.T
    with np.errstate(invalid="ignore", divide="ignore"):
        A = np.where(den > 0, num / np.where(den > 0, den, 1.0), np.nan)
    return A[np.triu_indices(G.shape[0])]


def _random(rng, n, m, miss=0.05):
    p = rng.uniform(0.02, 0.5, m)
    d = (rng.random((n, m)) < p).astype(int) + (rng.random((n, m)) < p).astype(int)
    G = np.array([0, 2, 3], dtype=np.uint8)[d]
    G[rng.random((n, m)) < miss] = 1
    return G


def test_matches_numpy_matrix_route():
    rng = np.random.default_rng(31)
    for n, m in [(5, 7), (40, 300), (120, 1000)]:
        G = _random(rng, n, m)
        G[:, 3] = 3                      # monomorphic: left out
        got, want = oracle.grm(G), _numpy_grm(G)
        assert (np.isnan(got) == np.isnan(want)).all()
        f = ~np.isnan(want)
        assert np.abs(got[f] - want[f]).max() <= 1e-12 * max(1.0, np.abs(want[f]).max())


def test_invariants():
    rng = np.random.default_rng(32)
    n, m = 60, 400
    G = _random(rng, n, m)
    A = oracle.grm(G)
    # relabelling A1 <-> A2 at any marker changes nothing
    G2 = G.copy()
    sw = rng.random(m) < 0.5
    G2[:, sw] = np.where(G[:, sw] == 0, 3, np.where(G[:, sw] == 3, 0, G[:, sw]))
    np.testing.assert_allclose(oracle.grm(G2), A, rtol=0, atol=1e-13)
    # adding monomorphic markers (p = 0 or 1) changes nothing
    G3 = np.concatenate([G, np.full((n, 5), 3, np.uint8), np.full((n, 5), 0, np.uint8)], axis=1)
    np.testing.assert_allclose(oracle.grm(G3), A, rtol=0, atol=1e-14)
    # sample order permutes the matrix
    perm = rng.permutation(n)
    Ap = oracle.grm(G[perm])
    full = np.empty((n, n))
    full[np.triu_indices(n)] = A
    full = np.triu(full) + np.triu(full, 1).T
    np.testing.assert_allclose(Ap, full[np.ix_(perm, perm)][np.triu_indices(n)], rtol=0, atol=1e-13)
    # thread count does not change anything
    np.testing.assert_array_equal(oracle.grm(G, threads=1), oracle.grm(G, threads=7))


def test_no_shared_markers_is_nan():
    G = np.array([[0, 1, 2], [1, 0, 2], [3, 3, 0]], dtype=np.uint8)
    A = oracle.grm(G)
    # samples 0 and 1 share only marker 2; marker 1 has calls from samples 1, 2 only
    assert np.isfinite(A).all()
    G[0, 2] = 1
    G[1, 2] = 1
    A = oracle.grm(G)
    assert np.isnan(A[oracle.tri_index(0, 1, 3)])


def test_rows_match_triangle():
    """grm_rows gives the rows of the same symmetric matrix, in any order and
    with repeats, bit for bit (same arithmetic per pair), and rejects rows
    outside [0, n)."""
    rng = np.random.default_rng(33)
    n, m = 45, 260
    G = _random(rng, n, m, miss=0.1)
    G[7, :] = 1                          # a sample without calls: NaN row
    A = oracle.grm(G)
    full = np.empty((n, n))
    full[np.triu_indices(n)] = A
    full = np.triu(full) + np.triu(full, 1).T
    rows = np.array([44, 0, 7, 13, 13, 30])
    got = oracle.grm_rows(G, rows, threads=3)
    np.testing.assert_array_equal(got, full[rows])
    assert np.isnan(got[2]).all()
    with pytest.raises(ValueError):
        oracle.grm_rows(G, [n])
    with pytest.raises(ValueError):
        oracle.grm_rows(G, [-1])
