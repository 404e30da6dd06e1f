"""Plain CPU oracle for all-pairs identity-by-state counts.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never loads, links or calls it, and it shares no code with that library: it
has its own unpacker, its own pair rule and its own distance formula.

What it computes (paper, "Improvements in PLINK 1.9 / Bitwise parallelism",
the per-marker loop PLINK 1.07 used): for every sample pair and every marker,
skip the marker if either call is missing; otherwise count IBS2 when the two
2-bit codes are equal, IBS0 when both bits differ and IBS1 otherwise.  N is
the number of markers not skipped.  The derived distance is
(IBS1 + 2*IBS0) / (2*N) in float64 (NaN when N == 0), the complement of the
IBS similarity the paper's ``--distance ibs`` command prints.

The arithmetic lives in ``ibs_oracle.c`` (plain C, one byte per genotype).
``ld_r`` is the linkage-disequilibrium correlation of marker pairs from the
same file (paper, "Bitwise parallelism", the example of r with missing calls),
``complete_linkage`` the complete-linkage clustering of the samples under
the distance matrix (paper, "Identity-by-state matrices, complete linkage
clustering"), and ``grm`` the GCTA genomic relationship matrix (paper,
"Partial sum lookup").
``topk`` below is the one rule written in Python: rank panel samples by
ascending distance, break ties by ascending index, put NaN (N == 0) last, and
pad with (-1, NaN) when k exceeds the panel size.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibs_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libibs_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``ibs_oracle.c`` with gcc -O2 into ``oracle/_build``.

    The environment variable IBS_ORACLE_LIB names a prebuilt library to use
    instead; the mutation tests use it to run the pins against an oracle with a
    planted mistake."""
    override = os.environ.get("IBS_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, p = ctypes.c_int64, ctypes.c_void_p
            lib.oracle_unpack.argtypes = [p, i64, i64, p]
            lib.oracle_unpack.restype = ctypes.c_int
            lib.oracle_unpack_subset.argtypes = [p, i64, i64, p, i64, i64, i64, p]
            lib.oracle_unpack_subset.restype = ctypes.c_int
            lib.oracle_ibs_block.argtypes = [p, p, i64, p, i64, p, i64, p, p, ctypes.c_int]
            lib.oracle_ibs_block.restype = ctypes.c_int
            lib.oracle_ibs_triangle.argtypes = [p, i64, i64, p, p, ctypes.c_int]
            lib.oracle_ibs_triangle.restype = ctypes.c_int
            lib.oracle_ld_r.argtypes = [p, i64, i64, i64, p, p, ctypes.c_int]
            lib.oracle_ld_r.restype = ctypes.c_int
            lib.oracle_complete_linkage.argtypes = [p, i64, p]
            lib.oracle_complete_linkage.restype = ctypes.c_int
            lib.oracle_grm.argtypes = [p, i64, i64, p, ctypes.c_int]
            lib.oracle_grm.restype = ctypes.c_int
            lib.oracle_grm_rows.argtypes = [p, i64, i64, p, i64, p, ctypes.c_int]
            lib.oracle_grm_rows.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def n_pairs(n: int) -> int:
    """Number of pairs i <= j (upper triangle including the diagonal)."""
    return n * (n + 1) // 2


def tri_index(i, j, n):
    """Row-major index of pair (i, j), i <= j, in the upper triangle incl. diagonal."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * n - i * (i - 1) // 2 + (j - i)


def unpack(packed: np.ndarray, n: int, m: int) -> np.ndarray:
    """One byte per genotype, sample-major [n][m] (codes 0..3)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    if packed.size != m * ((n + 3) // 4):
        raise ValueError("packed buffer size does not match n, m")
    G = np.empty((n, m), dtype=np.uint8)
    if _load().oracle_unpack(_ptr(packed), n, m, _ptr(G)) != 0:
        raise ValueError("oracle_unpack failed")
    return G


def unpack_subset(packed: np.ndarray, n: int, m: int, sel, var_begin: int, var_len: int) -> np.ndarray:
    """Codes of samples ``sel`` over markers [var_begin, var_begin + var_len)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    G = np.empty((sel.size, var_len), dtype=np.uint8)
    if _load().oracle_unpack_subset(_ptr(packed), n, m, _ptr(sel), sel.size, var_begin, var_len, _ptr(G)) != 0:
        raise ValueError("oracle_unpack_subset failed")
    return G


def ibs_block(GA: np.ndarray, GB: np.ndarray, rows=None, cols=None, threads: int = 0):
    """Counts [len(rows)][len(cols)][4] = (IBS0, IBS1, IBS2, N) and distances."""
    GA = np.ascontiguousarray(GA, dtype=np.uint8)
    GB = np.ascontiguousarray(GB, dtype=np.uint8)
    if GA.shape[1] != GB.shape[1]:
        raise ValueError("marker counts differ")
    m = GA.shape[1]
    rows = np.arange(GA.shape[0], dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.arange(GB.shape[0], dtype=np.int64) if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    counts = np.empty((rows.size, cols.size, 4), dtype=np.int32)
    dist = np.empty((rows.size, cols.size), dtype=np.float64)
    used = _load().oracle_ibs_block(_ptr(GA), _ptr(GB), m, _ptr(rows), rows.size, _ptr(cols), cols.size,
                                    _ptr(counts), _ptr(dist), int(threads))
    if used < 0:
        raise ValueError("oracle_ibs_block failed")
    return counts, dist


def ibs_triangle_from_codes(G: np.ndarray, threads: int = 0):
    """Upper triangle incl. diagonal, row-major: counts [P][4], dist [P], threads used."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    n, m = G.shape
    counts = np.empty((n_pairs(n), 4), dtype=np.int32)
    dist = np.empty(n_pairs(n), dtype=np.float64)
    used = _load().oracle_ibs_triangle(_ptr(G), n, m, _ptr(counts), _ptr(dist), int(threads))
    if used < 0:
        raise ValueError("oracle_ibs_triangle failed")
    return counts, dist, used


def ibs_triangle(packed: np.ndarray, n: int, m: int, threads: int = 0):
    """All-pairs counts of a packed variant-major matrix (upper triangle incl. diagonal)."""
    counts, dist, _ = ibs_triangle_from_codes(unpack(packed, n, m), threads)
    return counts, dist


def ibs_rows(packed: np.ndarray, n: int, m: int, rows, threads: int = 0):
    """Counts of the listed samples against every sample: [len(rows)][n][4], dist [len(rows)][n]."""
    G = unpack(packed, n, m)
    return ibs_block(G, G, rows=rows, threads=threads)


def ld_r(G: np.ndarray, window: int, threads: int = 0):
    """LD correlation r of marker pairs (a, a+1 .. a+window) from sample-major
    codes G [n][m] (paper, "Bitwise parallelism", the correlation coefficient
    with missing calls; x = +1 hom major, -1 hom minor, 0 het or missing, means
    over the samples where both calls are present).  Returns (r [m][window]
    float64, N [m][window] int32); slots past the last marker are NaN and 0."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    n, m = G.shape
    r = np.empty((m, window), dtype=np.float64)
    cnt = np.empty((m, window), dtype=np.int32)
    used = _load().oracle_ld_r(_ptr(G), n, m, int(window), _ptr(r), _ptr(cnt), int(threads))
    if used <= 0:
        raise ValueError("oracle_ld_r rejected its arguments")
    return r, cnt


def complete_linkage(tri: np.ndarray, n: int) -> np.ndarray:
    """Complete-linkage clustering (paper, "Identity-by-state matrices,
    complete linkage clustering") of n samples under the distance triangle
    (upper triangle with diagonal, as the library writes it; NaN = +inf).
    Greedy: merge the closest active pair; ties to the smallest (rep A, rep B),
    a cluster's rep being its smallest member.  Returns Z [n-1][4] = (id1, id2,
    height, size), ids in scipy's convention."""
    tri = np.ascontiguousarray(tri, dtype=np.float64)
    if tri.size != n * (n + 1) // 2:
        raise ValueError("triangle size does not match n")
    Z = np.empty((max(n - 1, 0), 4), dtype=np.float64)
    if _load().oracle_complete_linkage(_ptr(tri), n, _ptr(Z)) != 0:
        raise ValueError("oracle_complete_linkage rejected its arguments")
    return Z


def grm(G: np.ndarray, threads: int = 0) -> np.ndarray:
    """GCTA genomic relationship matrix (paper, "Partial sum lookup") of the
    samples of G [n][m]: per marker a table of the increments
    (x_j - 2p)(x_k - 2p) / (2p(1-p)) (x = A1 count, p its frequency over the
    marker's calls), summed over the markers where both calls are present and
    divided by their number; monomorphic markers left out; NaN when none is
    left.  Returns the upper triangle with diagonal (float64)."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    n, m = G.shape
    out = np.empty(n * (n + 1) // 2, dtype=np.float64)
    if _load().oracle_grm(_ptr(G), n, m, _ptr(out), int(threads)) <= 0:
        raise ValueError("oracle_grm rejected its arguments")
    return out


def grm_rows(G: np.ndarray, rows, threads: int = 0) -> np.ndarray:
    """Rows of the full symmetric relationship matrix of grm(): out[r][k] =
    A_{rows[r], k}, with the marker frequencies taken over all samples of G."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    n, m = G.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.size, n), dtype=np.float64)
    if _load().oracle_grm_rows(_ptr(G), n, m, _ptr(rows), rows.size, _ptr(out), int(threads)) <= 0:
        raise ValueError("oracle_grm_rows rejected its arguments")
    return out


def dist_from_counts(counts: np.ndarray) -> np.ndarray:
    """The oracle's distance (IBS1 + 2*IBS0) / (2*N) from count quadruples
    [..., 4] = (IBS0, IBS1, IBS2, N): one IEEE float64 division of exact
    integers, as ibs_oracle.c forms it, NaN where N == 0."""
    c = np.asarray(counts)
    num = c[..., 1].astype(np.float64) + 2.0 * c[..., 0].astype(np.float64)
    den = 2.0 * c[..., 3].astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        d = num / den
    return np.where(c[..., 3] == 0, np.nan, d)


def topk(dist_row: np.ndarray, k: int):
    """k nearest panel samples by distance: ascending distance, ties by ascending
    index, NaN ranked after every finite value, padded with (-1, NaN)."""
    dist_row = np.asarray(dist_row, dtype=np.float64)
    nan = np.isnan(dist_row)
    # np.lexsort sorts by the last key first: NaN flag, then distance, then index.
    order = np.lexsort((np.arange(dist_row.size), np.where(nan, 0.0, dist_row), nan))
    idx = np.full(k, -1, dtype=np.int32)
    dist = np.full(k, np.nan, dtype=np.float64)
    take = min(k, dist_row.size)
    idx[:take] = np.asarray(order[:take], dtype=np.int32)
    dist[:take] = dist_row[idx[:take]]
    return idx, dist
