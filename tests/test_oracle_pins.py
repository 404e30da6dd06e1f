"""Pins for the CPU oracle: checks against things other than the oracle itself.

- the 16 ordered code pairs against the allele-multiset meaning of identity by
  state and against the paper's seven-case enumeration ("Partial sum lookup");
- a hand-worked example (tests/golden/hand_example.txt);
- brute force by multiset intersection, with its own unpacker, on tiny random
  inputs with garbage in the padding bits;
- invariants: symmetry, IBS0+IBS1+IBS2 = N, diagonal = (0, 0, N_i, N_i),
  N_ij <= min(N_i, N_j), allele-flip invariance, marker-permutation
  invariance, sample-permutation equivariance, additivity over marker blocks;
- an independent library route: one-hot indicator matrices multiplied with
  numpy int64 matmul;
- closed forms for the distance (exact values, NaN at N = 0).
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Alleles carried by each non-missing code (A1 = 1, A2 = 2).
ALLELES = {0: (1, 1), 2: (1, 2), 3: (2, 2)}


def pack_codes(codes: np.ndarray, garbage_rng=None) -> np.ndarray:
    """Test-local packer: codes [n][m] -> variant-major bytes [m][ceil(n/4)]."""
    n, m = codes.shape
    nb = (n + 3) // 4
    out = np.zeros((m, nb), dtype=np.uint8)
    for s in range(n):
        out[:, s // 4] |= (codes[s].astype(np.uint8) << (2 * (s % 4))).astype(np.uint8)
    if garbage_rng is not None and n % 4:
        mask = (0xFF << (2 * (n % 4))) & 0xFF
        out[:, nb - 1] |= (garbage_rng.integers(0, 256, m).astype(np.uint8) & mask)
    return out


def unpack_bits(packed: np.ndarray, n: int) -> np.ndarray:
    """Second, independent unpacker: little-endian bit order via np.unpackbits."""
    bits = np.unpackbits(packed, axis=1, bitorder="little")  # [m][8*nb]
    lo = bits[:, 0::2][:, :n].astype(np.int64)
    hi = bits[:, 1::2][:, :n].astype(np.int64)
    return (lo + 2 * hi).T  # [n][m]


def multiset_ibs(a: int, b: int):
    """IBS state as the size of the multiset intersection of the two genotypes'
    alleles, or None when either call is missing."""
    if a == 1 or b == 1:
        return None
    x, y = list(ALLELES[a]), list(ALLELES[b])
    shared = 0
    for al in x:
        if al in y:
            y.remove(al)
            shared += 1
    return shared


def brute_force(codes: np.ndarray):
    n, m = codes.shape
    res = {}
    for i in range(n):
        for j in range(i, n):
            c = [0, 0, 0, 0]
            for k in range(m):
                s = multiset_ibs(int(codes[i, k]), int(codes[j, k]))
                if s is None:
                    continue
                c[s] += 1
                c[3] += 1
            res[(i, j)] = c
    return res


def test_code_pair_table_matches_multiset_and_seven_cases():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "code_pairs.txt")) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 16
    state_of_case = {1: "IBS2", 4: "IBS2", 6: "IBS2", 2: "IBS1", 5: "IBS1", 3: "IBS0", 7: "skip"}
    for a, b, outcome, case in rows:
        a, b, case = int(a), int(b), int(case)
        assert state_of_case[case] == outcome
        ms = multiset_ibs(a, b)
        assert outcome == ("skip" if ms is None else f"IBS{ms}")
        packed = pack_codes(np.array([[a], [b]], dtype=np.uint8))
        counts, dist = oracle.ibs_triangle(packed, 2, 1)
        c01 = counts[1]
        expect = {"skip": [0, 0, 0, 0], "IBS0": [1, 0, 0, 1], "IBS1": [0, 1, 0, 1], "IBS2": [0, 0, 1, 1]}[outcome]
        assert c01.tolist() == expect, (a, b)
        if outcome == "skip":
            assert np.isnan(dist[1])


def test_hand_example():
    lines = [ln.split() for ln in open(os.path.join(GOLDEN, "hand_example.txt")) if ln.strip() and not ln.startswith("#")]
    n = int([l for l in lines if l[0] == "n"][0][1])
    m = int([l for l in lines if l[0] == "m"][0][1])
    codes = np.array([[int(x) for x in l[2:]] for l in lines if l[0] == "codes"], dtype=np.uint8)
    packed = np.array([int(x, 16) for x in [l for l in lines if l[0] == "packed"][0][1:]], dtype=np.uint8).reshape(m, 1)
    assert (pack_codes(codes) == packed).all()
    counts, dist = oracle.ibs_triangle(packed, n, m)
    for l in [l for l in lines if l[0] == "pair"]:
        i, j = int(l[1]), int(l[2])
        p = int(oracle.tri_index(i, j, n))
        assert counts[p].tolist() == [int(x) for x in l[3:7]]
        assert dist[p] == float(l[7])


@pytest.mark.parametrize("seed", range(0, 400))
def test_random_tiny_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 10))
    m = int(rng.integers(1, 71))
    pmiss = rng.uniform(0, 0.6)
    codes = rng.choice([0, 2, 3], size=(n, m)).astype(np.uint8)
    codes[rng.random((n, m)) < pmiss] = 1
    packed = pack_codes(codes, garbage_rng=rng)
    assert (unpack_bits(packed, n) == codes).all()
    assert (oracle.unpack(packed, n, m) == codes).all()
    counts, dist = oracle.ibs_triangle(packed, n, m, threads=1 + seed % 3)
    bf = brute_force(unpack_bits(packed, n))
    for (i, j), c in bf.items():
        p = int(oracle.tri_index(i, j, n))
        assert counts[p].tolist() == [c[0], c[1], c[2], c[3]], (seed, i, j)
        if c[3] == 0:
            assert np.isnan(dist[p])
        else:
            assert dist[p] == (c[1] + 2 * c[0]) / (2.0 * c[3])


def _random_codes(rng, n, m, miss=0.05):
    p = rng.uniform(0.02, 0.5, m)
    d = (rng.random((n, m)) < p).astype(np.int64) + (rng.random((n, m)) < p).astype(np.int64)
    codes = np.array([0, 2, 3], dtype=np.uint8)[d]
    codes[rng.random((n, m)) < miss] = 1
    return codes


def test_invariants():
    rng = np.random.default_rng(11)
    n, m = 37, 531
    codes = _random_codes(rng, n, m)
    codes[5, :] = 1  # an all-missing sample
    codes[:, 17] = 1  # an all-missing marker
    G = codes
    full, fdist = oracle.ibs_block(G, G)
    # symmetry
    assert (full == full.transpose(1, 0, 2)).all()
    np.testing.assert_array_equal(fdist, fdist.T)
    # sum
    assert (full[..., 0] + full[..., 1] + full[..., 2] == full[..., 3]).all()
    # diagonal
    nonmiss = (codes != 1).sum(axis=1)
    for i in range(n):
        assert full[i, i].tolist() == [0, 0, int(nonmiss[i]), int(nonmiss[i])]
    # N_ij <= min(N_i, N_j)
    assert (full[..., 3] <= np.minimum.outer(nonmiss, nonmiss)).all()
    # the all-missing sample has N = 0 with everyone, distance NaN
    assert (full[5, :, 3] == 0).all() and np.isnan(fdist[5]).all()
    # allele flip at a random marker subset: code 0 <-> 3
    flip = rng.random(m) < 0.5
    fl = codes.copy()
    sel = flip[None, :] & ((codes == 0) | (codes == 3))
    fl[sel] = 3 - fl[sel]
    assert (oracle.ibs_block(fl, fl)[0] == full).all()
    # marker permutation
    perm = rng.permutation(m)
    assert (oracle.ibs_block(codes[:, perm], codes[:, perm])[0] == full).all()
    # sample permutation equivariance
    sp = rng.permutation(n)
    psq = oracle.ibs_block(codes[sp], codes[sp])[0]
    assert (psq == full[sp][:, sp]).all()
    # additivity over marker blocks
    a = oracle.ibs_block(codes[:, :200], codes[:, :200])[0]
    b = oracle.ibs_block(codes[:, 200:], codes[:, 200:])[0]
    assert (a + b == full).all()
    # the triangle entry points agree with the square
    tri, tdist = oracle.ibs_triangle(pack_codes(codes), n, m)
    iu = np.triu_indices(n)
    assert (tri == full[iu]).all()
    np.testing.assert_array_equal(tdist, fdist[iu])


def test_onehot_matmul_library_route():
    """IBS2 = sum_c A_c A_c^T, IBS0 = A0 A3^T + A3 A0^T, N = V V^T with one-hot
    indicators A_c (c in {0, 2, 3}, zero where missing), computed by numpy."""
    rng = np.random.default_rng(5)
    n, m = 300, 2000
    codes = _random_codes(rng, n, m, miss=0.03)
    A = {c: (codes == c).astype(np.int64) for c in (0, 2, 3)}
    V = A[0] + A[2] + A[3]
    ibs2 = A[0] @ A[0].T + A[2] @ A[2].T + A[3] @ A[3].T
    ibs0 = A[0] @ A[3].T + A[3] @ A[0].T
    N = V @ V.T
    ibs1 = N - ibs0 - ibs2
    tri, dist = oracle.ibs_triangle(pack_codes(codes), n, m)
    iu = np.triu_indices(n)
    assert (tri[:, 0] == ibs0[iu]).all()
    assert (tri[:, 1] == ibs1[iu]).all()
    assert (tri[:, 2] == ibs2[iu]).all()
    assert (tri[:, 3] == N[iu]).all()


def test_distance_closed_forms():
    m = 97
    # identical monomorphic samples: IBS2 = m, distance 0
    codes = np.full((2, m), 3, dtype=np.uint8)
    c, d = oracle.ibs_triangle(pack_codes(codes), 2, m)
    assert c[1].tolist() == [0, 0, m, m] and d[1] == 0.0
    # opposite homozygotes everywhere: IBS0 = m, distance 1
    codes = np.stack([np.zeros(m, np.uint8), np.full(m, 3, np.uint8)])
    c, d = oracle.ibs_triangle(pack_codes(codes), 2, m)
    assert c[1].tolist() == [m, 0, 0, m] and d[1] == 1.0
    # hom vs het everywhere: IBS1 = m, distance 1/2
    codes = np.stack([np.zeros(m, np.uint8), np.full(m, 2, np.uint8)])
    c, d = oracle.ibs_triangle(pack_codes(codes), 2, m)
    assert c[1].tolist() == [0, m, 0, m] and d[1] == 0.5
    # one sample entirely missing: N = 0, distance NaN
    codes = np.stack([np.ones(m, np.uint8), np.full(m, 2, np.uint8)])
    c, d = oracle.ibs_triangle(pack_codes(codes), 2, m)
    assert c[1].tolist() == [0, 0, 0, 0] and np.isnan(d[1]) and np.isnan(d[0])


def test_unpack_subset_matches_full_unpack():
    rng = np.random.default_rng(3)
    n, m = 23, 301
    codes = _random_codes(rng, n, m)
    packed = pack_codes(codes, garbage_rng=rng)
    sel = np.array([22, 0, 7, 7, 13])
    G = oracle.unpack_subset(packed, n, m, sel, 40, 200)
    assert (G == codes[sel][:, 40:240]).all()


def test_topk_rule():
    d = np.array([0.3, np.nan, 0.1, 0.3, 0.1, 0.2])
    idx, dist = oracle.topk(d, 8)
    assert idx.tolist() == [2, 4, 5, 0, 3, 1, -1, -1]
    assert np.isnan(dist[5]) and np.isnan(dist[6]) and dist[0] == 0.1
    idx, _ = oracle.topk(d, 2)
    assert idx.tolist() == [2, 4]


def test_dist_from_counts_equals_the_c_oracle_bit_for_bit():
    # the numpy restatement used by the large GPU checks must give exactly the
    # C oracle's doubles, NaN included
    rng = np.random.default_rng(31)
    codes = _random_codes(rng, 37, 300, miss=0.3)
    codes[5] = 1  # a sample with no calls: N = 0 against everyone
    counts, dist = oracle.ibs_triangle(pack_codes(codes), 37, 300)
    got = oracle.dist_from_counts(counts)
    assert np.array_equal(np.isnan(got), np.isnan(dist))
    ok = ~np.isnan(dist)
    assert np.array_equal(got[ok].view(np.uint64), dist[ok].view(np.uint64))
