"""PLINK 1 binary genotype files (.bed) for the library's calls.

A .bed file is three header bytes, 0x6C 0x1B and a mode byte, followed by
the genotype matrix.  Mode 0x01 is variant-major: one row per variant of
ceil(n/4) bytes, sample s in bits 2*(s%4) and 2*(s%4)+1 of byte s//4 - the
layout every entry point of include/ibs.h takes.  Mode 0x00 (sample-major,
PLINK's pre-1.0 layout) is refused rather than transposed.  The sample and
variant counts are not stored in the .bed file; they are the line counts of
the companion .fam and .bim files, or given directly.

This module only moves bytes between files and numpy arrays; it computes
nothing of the method.
"""
from __future__ import annotations

import os

import numpy as np

MAGIC = b"\x6c\x1b"
VARIANT_MAJOR = 0x01
SAMPLE_MAJOR = 0x00


def count_lines(path: str) -> int:
    """Non-empty lines of a text file (.fam: samples, .bim: variants)."""
    with open(path, "rb") as f:
        return sum(1 for line in f if line.strip())


def read_bed(path: str, n_samples: int | None = None, n_variants: int | None = None,
             fam: str | None = None, bim: str | None = None) -> tuple[np.ndarray, int, int]:
    """Read a variant-major .bed file.

    The counts come from n_samples / n_variants, else from the .fam / .bim
    files (by default the .bed path with those suffixes).  Returns
    (packed uint8 [n_variants][ceil(n_samples/4)], n_samples, n_variants).
    Raises ValueError on a bad magic number, a sample-major file, or a file
    size that does not match the counts."""
    stem = path[:-4] if path.endswith(".bed") else path
    if n_samples is None:
        n_samples = count_lines(fam or stem + ".fam")
    if n_variants is None:
        n_variants = count_lines(bim or stem + ".bim")
    if n_samples < 1 or n_variants < 1:
        raise ValueError(f"need at least one sample and one variant (got {n_samples}, {n_variants})")
    row_bytes = (n_samples + 3) // 4
    with open(path, "rb") as f:
        head = f.read(3)
        if len(head) < 3 or head[:2] != MAGIC:
            raise ValueError(f"{path}: not a PLINK 1 .bed file (magic {head[:2].hex()})")
        if head[2] == SAMPLE_MAJOR:
            raise ValueError(f"{path}: sample-major .bed (mode 0x00) is not supported; rewrite it variant-major")
        if head[2] != VARIANT_MAJOR:
            raise ValueError(f"{path}: unknown .bed mode byte 0x{head[2]:02x}")
        body = f.read()
    if len(body) != n_variants * row_bytes:
        raise ValueError(f"{path}: {len(body)} genotype bytes, expected {n_variants} variants x {row_bytes} bytes "
                         f"for {n_samples} samples")
    packed = np.frombuffer(body, dtype=np.uint8).reshape(n_variants, row_bytes).copy()
    return packed, n_samples, n_variants


def write_bed(path: str, packed: np.ndarray, n_samples: int) -> None:
    """Write packed uint8 [n_variants][ceil(n_samples/4)] as a variant-major
    .bed file (no .fam / .bim)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    if packed.ndim != 2 or packed.shape[1] != (n_samples + 3) // 4:
        raise ValueError(f"packed shape {packed.shape} does not match {n_samples} samples")
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(MAGIC + bytes([VARIANT_MAJOR]))
        f.write(packed.tobytes())
    os.replace(tmp, path)
