"""The .bed reader and writer (paper_1410_4803_gb300.bedio): round trip, the
counts from .fam / .bim line counts, and refusal of a bad magic number, a
sample-major file and a size that does not match the counts."""
import numpy as np
import pytest

import oracle
from helpers import pack_codes, random_codes
from paper_1410_4803_gb300 import bedio


def test_round_trip_with_fam_and_bim(tmp_path):
    rng = np.random.default_rng(3)
    n, m = 37, 53
    codes = random_codes(rng, n, m, miss=0.1)
    packed = pack_codes(codes)
    path = str(tmp_path / "cohort.bed")
    bedio.write_bed(path, packed, n)
    (tmp_path / "cohort.fam").write_text("".join(f"F{i} I{i} 0 0 0 -9\n" for i in range(n)))
    (tmp_path / "cohort.bim").write_text("".join(f"1 rs{k} 0 {k + 1} A C\n" for k in range(m)))
    got, gn, gm = bedio.read_bed(path)
    assert (gn, gm) == (n, m)
    np.testing.assert_array_equal(got, packed)
    # the codes read back through the oracle's own unpacker are the ones written
    np.testing.assert_array_equal(oracle.unpack(got, n, m), codes)
    with open(path, "rb") as f:
        assert f.read(3) == b"\x6c\x1b\x01"


def test_counts_given_directly(tmp_path):
    packed = np.arange(3 * 2, dtype=np.uint8).reshape(3, 2)
    path = str(tmp_path / "x.bed")
    bedio.write_bed(path, packed, 6)
    got, n, m = bedio.read_bed(path, n_samples=6, n_variants=3)
    assert (n, m) == (6, 3)
    np.testing.assert_array_equal(got, packed)


def test_refusals(tmp_path):
    path = str(tmp_path / "y.bed")
    body = bytes(range(8))
    for head, msg in [(b"\x00\x00\x01", "magic"), (b"\x6c\x1b\x00", "sample-major"), (b"\x6c\x1b\x07", "mode")]:
        with open(path, "wb") as f:
            f.write(head + body)
        with pytest.raises(ValueError, match=msg):
            bedio.read_bed(path, n_samples=8, n_variants=4)
    with open(path, "wb") as f:
        f.write(b"\x6c\x1b\x01" + body)
    with pytest.raises(ValueError, match="genotype bytes"):
        bedio.read_bed(path, n_samples=9, n_variants=4)  # 3 bytes per row needed
    with pytest.raises(ValueError):
        bedio.write_bed(path, np.zeros((4, 2), np.uint8), 9)
