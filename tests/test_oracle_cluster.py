"""Pins of the oracle's complete-linkage clustering (paper, "Identity-by-state
matrices, complete linkage clustering"): hand-worked examples (one with
ties), scipy's complete linkage on tie-free distances, and brute-force
invariants (every merge height is the largest distance between the merged
clusters' members, heights never decrease, ids and sizes are consistent), and
NaN distances treated as infinite."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cluster_hand_example.txt")


def _tri_from_square(D):
    n = D.shape[0]
    return np.array([D[i, j] for i in range(n) for j in range(i, n)], dtype=np.float64)


def _read_golden():
    ex, cur = {}, None
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "example":
            cur = ex.setdefault(t[1], {"merges": []})
        elif t[0] == "n":
            cur["n"] = int(t[1])
        elif t[0] == "points":
            cur["points"] = None if t[1] == "equal" else [float(x) for x in t[1:]]
        elif t[0] == "merge":
            cur["merges"].append([float(x) for x in t[1:]])
    return ex


@pytest.mark.parametrize("name", ["line", "ties"])
def test_hand_examples(name):
    e = _read_golden()[name]
    n = e["n"]
    if e["points"] is None:
        D = np.ones((n, n)) - np.eye(n)
    else:
        x = np.array(e["points"])
        D = np.abs(x[:, None] - x[None, :])
    Z = oracle.complete_linkage(_tri_from_square(D), n)
    np.testing.assert_array_equal(Z, np.array(e["merges"]))


def _random_square(rng, n):
    A = rng.random((n, n))
    D = (A + A.T) / 2
    np.fill_diagonal(D, 0)
    return D


def test_matches_scipy_on_tie_free_distances():
    hierarchy = pytest.importorskip("scipy.cluster.hierarchy")
    from scipy.spatial.distance import squareform
    rng = np.random.default_rng(21)
    for n in [2, 3, 10, 60, 200]:
        D = _random_square(rng, n)
        Z = oracle.complete_linkage(_tri_from_square(D), n)
        want = hierarchy.linkage(squareform(D, checks=False), method="complete")
        np.testing.assert_array_equal(Z[:, :2], np.sort(want[:, :2], axis=1))
        np.testing.assert_array_equal(Z[:, 2:], want[:, 2:])


def _members(Z, n):
    mem = {i: [i] for i in range(n)}
    for s, (a, b, _, _) in enumerate(Z):
        mem[n + s] = mem.pop(int(a)) + mem.pop(int(b))
    return mem


def test_brute_force_invariants_with_ties():
    rng = np.random.default_rng(22)
    for trial in range(300):
        n = int(rng.integers(2, 10))
        D = rng.integers(0, 4, size=(n, n)).astype(np.float64) / 4.0   # many ties
        D = np.maximum(D, D.T)
        np.fill_diagonal(D, 0)
        Z = oracle.complete_linkage(_tri_from_square(D), n)
        mem = {i: [i] for i in range(n)}
        seen = set()
        prev = -np.inf
        for s, (a, b, h, size) in enumerate(Z):
            a, b = int(a), int(b)
            assert a < b and a not in seen and b not in seen and a in mem and b in mem
            seen |= {a, b}
            A, B = mem.pop(a), mem.pop(b)
            assert h == max(D[i, j] for i in A for j in B)
            # greedy: no other pair of active clusters is closer
            for c1 in mem:
                for c2 in mem:
                    if c1 < c2:
                        assert max(D[i, j] for i in mem[c1] for j in mem[c2]) >= h
            assert size == len(A) + len(B)
            assert h >= prev
            prev = h
            mem[n + s] = A + B
        assert list(mem.values())[0].__len__() == n


def test_nan_distance_is_infinite_and_joins_last():
    rng = np.random.default_rng(23)
    n = 12
    D = _random_square(rng, n)
    D[4, :] = np.nan
    D[:, 4] = np.nan
    D[4, 4] = 0
    Z = oracle.complete_linkage(_tri_from_square(D), n)
    assert np.isinf(Z[-1, 2]) and 4 in (int(Z[-1, 0]), int(Z[-1, 1]))
    assert np.isfinite(Z[:-1, 2]).all()


def test_single_sample_and_bad_size():
    assert oracle.complete_linkage(np.zeros(1), 1).shape == (0, 4)
    with pytest.raises(ValueError):
        oracle.complete_linkage(np.zeros(4), 3)
