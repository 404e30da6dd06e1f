"""Seeded synthetic PLINK 1 .bed matrices shaped like the paper's IBS workloads.

The paper times its IBS matrix on datasets that are not distributed with it
(section "Performance comparisons": synth1/synth2 simulations and 1000 Genomes
subsets).  These generators stand in for them with the same kind of data:
biallelic variants in Hardy-Weinberg proportions, uniform minor-allele
frequencies, i.i.d. missing calls, and, for the structured cohorts, a
Balding-Nichols five-subpopulation model with injected parent-offspring pairs
and near-duplicate samples.

This module draws inputs only.  It holds no identity-by-state arithmetic and
is the one module the GPU tests and the CPU oracle's tests share.  Per-variant
parameters come from numpy's PCG64 generator with a fixed seed; per-genotype
draws come from the C generator (Philox4x32-10, counter = (variant, sample)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_bed.c")
_SRC_GPU = os.path.join(_HERE, "synth_bed_gpu.cu")
_BUILD_DIR = os.path.join(os.path.dirname(_HERE), "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libsynth_bed.so")
_LIB_GPU_PATH = os.path.join(_BUILD_DIR, "libsynth_bed_gpu.so")
_lib = None
_lib_gpu = None
_lock = threading.Lock()

BASE, OFFSPRING, DUPLICATE = 0, 1, 2


def build(force: bool = False) -> str:
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_gpu(force: bool = False) -> str:
    """Compile the device-side generator (synth_bed_gpu.cu, sm_103a)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_GPU_PATH) or os.path.getmtime(_LIB_GPU_PATH) < os.path.getmtime(_SRC_GPU):
        import shutil
        nvcc = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
        if not os.path.exists(nvcc):
            nvcc = shutil.which("nvcc") or nvcc
        tmp = _LIB_GPU_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler",
                               "-fPIC", _SRC_GPU, "-o", tmp])
        os.replace(tmp, _LIB_GPU_PATH)
    return _LIB_GPU_PATH


def _load_gpu():
    global _lib_gpu
    with _lock:
        if _lib_gpu is None:
            lib = ctypes.CDLL(build_gpu())
            i64, p = ctypes.c_int64, ctypes.c_void_p
            lib.synth_bed_gpu.argtypes = [i64, ctypes.c_uint64, i64, p, ctypes.c_int32, p, i64, p, p, p, p, p,
                                          ctypes.c_uint64, ctypes.c_int, p, p]
            lib.synth_bed_gpu.restype = ctypes.c_int
            _lib_gpu = lib
    return _lib_gpu


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, p = ctypes.c_int64, ctypes.c_void_p
            lib.synth_bed.argtypes = [i64, ctypes.c_uint64, i64, p, ctypes.c_int32, p, i64, p, p, p, p, p,
                                      ctypes.c_double, ctypes.c_int, p, ctypes.c_int]
            lib.synth_bed.restype = ctypes.c_int
            lib.synth_philox4x32_10.argtypes = [p, p, p]
            lib.synth_philox4x32_10.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def philox4x32_10(counter, key):
    """One Philox4x32-10 block (exposed for known-answer tests)."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _load().synth_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


@dataclass
class Samples:
    """Per-sample descriptors: global id, subpopulation, kind and source."""
    gid: np.ndarray
    pop: np.ndarray
    kind: np.ndarray
    src_gid: np.ndarray
    src_pop: np.ndarray

    @property
    def n(self) -> int:
        return int(self.gid.size)

    def take(self, idx) -> "Samples":
        idx = np.asarray(idx)
        return Samples(self.gid[idx], self.pop[idx], self.kind[idx], self.src_gid[idx], self.src_pop[idx])

    @staticmethod
    def base(n: int, n_pop: int = 1, gid0: int = 0) -> "Samples":
        gid = np.arange(gid0, gid0 + n, dtype=np.int64)
        per = -(-n // n_pop)
        pop = (np.arange(n) // per).astype(np.int32)
        return Samples(gid, pop, np.zeros(n, np.int32), gid.copy(), pop.copy())


@dataclass
class Model:
    """Per-variant parameters: A2 frequency per subpopulation [n_pop][m] and missing rate [m]."""
    p_pop: np.ndarray
    miss_rate: np.ndarray
    seed: int
    var_offset: int = 0
    dup_discord: float = 0.001

    @property
    def m(self) -> int:
        return int(self.miss_rate.size)

    def window(self, begin: int, length: int) -> "Model":
        return Model(np.ascontiguousarray(self.p_pop[:, begin:begin + length]),
                     np.ascontiguousarray(self.miss_rate[begin:begin + length]), self.seed,
                     self.var_offset + begin, self.dup_discord)


def generate(model: Model, samples: Samples, pad_garbage: bool = False, threads: int = 0) -> np.ndarray:
    """Packed variant-major matrix uint8 [m][ceil(n/4)] for `samples` under `model`."""
    m, n = model.m, samples.n
    out = np.empty((m, (n + 3) // 4), dtype=np.uint8)
    p_pop = np.ascontiguousarray(model.p_pop, dtype=np.float64)
    miss = np.ascontiguousarray(model.miss_rate, dtype=np.float64)
    arrs = [np.ascontiguousarray(a, dtype=t) for a, t in
            ((samples.gid, np.int64), (samples.pop, np.int32), (samples.kind, np.int32),
             (samples.src_gid, np.int64), (samples.src_pop, np.int32))]
    rc = _load().synth_bed(m, model.seed, model.var_offset, _ptr(p_pop), p_pop.shape[0], _ptr(miss), n,
                           *[_ptr(a) for a in arrs], float(model.dup_discord), int(pad_garbage), _ptr(out),
                           int(threads))
    if rc != 0:
        raise ValueError("synth_bed rejected its arguments")
    return out


def thresholds(p) -> np.ndarray:
    """32-bit fixed-point thresholds of probabilities, as the C generator forms
    them: floor(p * 2^32), 0 for p <= 0, 2^32 for p >= 1 (uint64)."""
    p = np.asarray(p, dtype=np.float64)
    inner = np.clip(p, 0.0, 1.0) * 4294967296.0
    t = inner.astype(np.uint64)
    t[p <= 0.0] = 0
    t[p >= 1.0] = np.uint64(1) << np.uint64(32)
    return t


def generate_device(model: Model, samples: Samples, pad_garbage: bool = False, device: int = 0, stream=None):
    """generate() on the GPU: the same packed bytes, as a torch uint8 tensor
    [m][ceil(n/4)] on cuda:`device` (enqueued on `stream`, default the
    current stream)."""
    import torch
    dev = torch.device("cuda", device)
    m, n = model.m, samples.n
    out = torch.empty((m, (n + 3) // 4), dtype=torch.uint8, device=dev)
    thr = torch.from_numpy(np.ascontiguousarray(thresholds(model.p_pop))).to(dev)
    miss = torch.from_numpy(np.ascontiguousarray(thresholds(model.miss_rate))).to(dev)
    arrs = [torch.from_numpy(np.ascontiguousarray(a, dtype=t)).to(dev) for a, t in
            ((samples.gid, np.int64), (samples.pop, np.int32), (samples.kind, np.int32),
             (samples.src_gid, np.int64), (samples.src_pop, np.int32))]
    for name, a in (("pop", samples.pop), ("src_pop", samples.src_pop)):
        if np.any(np.asarray(a) < 0) or np.any(np.asarray(a) >= model.p_pop.shape[0]):
            raise ValueError(f"{name} out of range")
    dup = int(thresholds(np.array([model.dup_discord]))[0])
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    with torch.cuda.device(dev):
        rc = _load_gpu().synth_bed_gpu(m, model.seed, model.var_offset, thr.data_ptr(), model.p_pop.shape[0],
                                       miss.data_ptr(), n, *[a.data_ptr() for a in arrs], dup, int(pad_garbage),
                                       out.data_ptr(), st)
    if rc != 0:
        raise ValueError(f"synth_bed_gpu failed ({rc})")
    torch.cuda.current_stream(dev).synchronize() if stream is None else stream.synchronize()
    return out


def _flip(rng, p):
    # Orientation of A2 versus A1 by a coin per variant (IBS is invariant to it).
    return np.where(rng.random(p.size) < 0.5, 1.0 - p, p)


def plain_model(m: int, seed: int, maf=(0.05, 0.5), miss=0.01, hi_miss_frac=0.0, hi_miss_rate=0.3) -> Model:
    """One population, MAF ~ U(maf), i.i.d. missing calls; a fraction of
    variants gets the higher missing rate instead."""
    rng = np.random.default_rng(seed)
    p = _flip(rng, rng.uniform(maf[0], maf[1], m))
    rate = np.full(m, miss)
    if hi_miss_frac > 0:
        rate[rng.random(m) < hi_miss_frac] = hi_miss_rate
    return Model(p[None, :].copy(), rate, seed)


def balding_nichols_model(m: int, seed: int, n_pop=5, fst=0.05, anc=(0.02, 0.5), miss=0.01) -> Model:
    """Ancestral p ~ U(anc); subpopulation p_k ~ Beta(p(1-F)/F, (1-p)(1-F)/F)."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(anc[0], anc[1], m)
    a = p * (1 - fst) / fst
    b = (1 - p) * (1 - fst) / fst
    pk = rng.beta(a[None, :].repeat(n_pop, 0), b[None, :].repeat(n_pop, 0))
    flip = rng.random(m) < 0.5
    pk[:, flip] = 1.0 - pk[:, flip]
    return Model(np.ascontiguousarray(pk), np.full(m, miss), seed)


def structured_samples(n_base: int, n_pop: int, n_offspring: int, n_dup: int, seed: int, gid0: int = 0) -> Samples:
    """Base samples split evenly over subpopulations, then offspring of random
    base samples, then duplicates of other random base samples (appended)."""
    rng = np.random.default_rng(seed + 7919)
    base = Samples.base(n_base, n_pop, gid0)
    srcs = rng.choice(n_base, size=n_offspring + n_dup, replace=False)
    k = n_base + n_offspring + n_dup
    gid = np.arange(gid0, gid0 + k, dtype=np.int64)
    pop = np.concatenate([base.pop, base.pop[srcs]]).astype(np.int32)
    kind = np.concatenate([np.zeros(n_base), np.full(n_offspring, OFFSPRING), np.full(n_dup, DUPLICATE)]).astype(np.int32)
    src_gid = np.concatenate([base.gid, base.gid[srcs]]).astype(np.int64)
    src_pop = pop.copy()
    return Samples(gid, pop, kind, src_gid, src_pop)


@dataclass
class Workload:
    name: str
    packed: np.ndarray
    n: int
    m: int
    samples: Samples
    model: Model
    info: dict = field(default_factory=dict)

    @property
    def comparisons(self) -> int:
        return self.n * (self.n - 1) // 2 * self.m


def _packed(model: Model, s: Samples, pad_garbage: bool = False, device=None):
    """The packed matrix on the host (numpy) or, with `device` an ordinal, on
    that GPU (torch tensor, same bytes)."""
    if device is None:
        return generate(model, s, pad_garbage)
    return generate_device(model, s, pad_garbage, device=device)


def plain_config1(pad_garbage=False, device=None) -> Workload:
    """n=256, m=4,096, MAF ~ U(0.05, 0.5), 1% missing i.i.d., seed 0."""
    model = plain_model(4096, 0, maf=(0.05, 0.5), miss=0.01)
    s = Samples.base(256)
    return Workload("plain n=256 m=4096", _packed(model, s, pad_garbage, device), 256, 4096, s, model)


def plain_config2(n=4096, m=100_000, device=None) -> Workload:
    """n=4,096, m=100,000, MAF ~ U(0.01, 0.5), 2% missing i.i.d. and 0.5% of
    variants at 30% missing, seed 1."""
    model = plain_model(m, 1, maf=(0.01, 0.5), miss=0.02, hi_miss_frac=0.005, hi_miss_rate=0.3)
    s = Samples.base(n)
    return Workload(f"plain n={n} m={m}", _packed(model, s, device=device), n, m, s, model)


def structured_config3(n_base_per_pop=3950, n_pop=5, m=500_000, n_offspring=200, n_dup=50, seed=2,
                       device=None) -> Workload:
    """Balding-Nichols five subpopulations (F=0.05), 200 parent-offspring pairs
    and 50 duplicates at 0.1% discordance, 1% missing; n = 20,000 at full size."""
    model = balding_nichols_model(m, seed, n_pop=n_pop, fst=0.05, anc=(0.02, 0.5), miss=0.01)
    s = structured_samples(n_base_per_pop * n_pop, n_pop, n_offspring, n_dup, seed)
    return Workload(f"structured n={s.n} m={m}", _packed(model, s, device=device), s.n, m, s, model)


@dataclass
class Subset:
    sample_idx: np.ndarray  # int64 indices into the pool
    var_begin: int
    var_len: int

    @property
    def n(self) -> int:
        return int(self.sample_idx.size)

    @property
    def comparisons(self) -> int:
        return self.n * (self.n - 1) // 2 * self.var_len


def batch_subsets(pool_n=30_000, pool_m=600_000, n_subsets=64, n_range=(200, 8000), m_range=(10_000, 200_000),
                  seed=3):
    """Subsets of uneven size drawn without replacement from the pool, each
    over a contiguous variant window of uneven length."""
    rng = np.random.default_rng(seed + 104729)
    subs = []
    for _ in range(n_subsets):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        n = min(n, pool_n)
        idx = np.sort(rng.choice(pool_n, size=n, replace=False)).astype(np.int64)
        vl = int(rng.integers(m_range[0], m_range[1] + 1))
        vl = min(vl, pool_m)
        vb = int(rng.integers(0, pool_m - vl + 1))
        subs.append(Subset(idx, vb, vl))
    return subs


def batch_pool(pool_n=30_000, pool_m=600_000, seed=3, device=None) -> Workload:
    """Pool generated as the plain n=4,096 workload but without the
    high-missingness variants: MAF ~ U(0.01, 0.5), 2% missing."""
    model = plain_model(pool_m, seed, maf=(0.01, 0.5), miss=0.02)
    s = Samples.base(pool_n)
    return Workload(f"pool n={pool_n} m={pool_m}", _packed(model, s, device=device), pool_n, pool_m, s, model)


def serving_panel(n_base_per_pop=19_750, n_pop=5, m=200_000, n_offspring=1000, n_dup=250, seed=4,
                  device=None) -> Workload:
    """Reference panel generated like the structured cohort, scaled."""
    return structured_config3(n_base_per_pop, n_pop, m, n_offspring, n_dup, seed, device=device)


def serving_query_sizes(n_requests: int, seed=4, q_max=512):
    """q = floor(exp(U(0, ln 512))) + 1, clipped to 512 (log-uniform sizes)."""
    rng = np.random.default_rng(seed + 15485863)
    q = np.floor(np.exp(rng.uniform(0.0, np.log(q_max), n_requests))).astype(np.int64) + 1
    return np.minimum(q, q_max)


def serving_queries(panel: Workload, q: int, request_id: int, related_frac=0.1, seed=4):
    """Fresh query samples from the panel's model; about `related_frac` of them
    are offspring or duplicates of panel base samples.  Returns (packed, Samples)."""
    rng = np.random.default_rng(seed * 1_000_003 + request_id)
    gid0 = (1 << 40) + request_id * 4096
    n_pop = panel.model.p_pop.shape[0]
    gid = np.arange(gid0, gid0 + q, dtype=np.int64)
    pop = rng.integers(0, n_pop, q).astype(np.int32)
    kind = np.zeros(q, np.int32)
    src_gid = gid.copy()
    src_pop = pop.copy()
    base_idx = np.flatnonzero(panel.samples.kind == BASE)
    rel = rng.random(q) < related_frac
    for t in np.flatnonzero(rel):
        b = int(rng.choice(base_idx))
        kind[t] = OFFSPRING if rng.random() < 0.5 else DUPLICATE
        src_gid[t] = panel.samples.gid[b]
        src_pop[t] = panel.samples.pop[b]
        pop[t] = src_pop[t]
    s = Samples(gid, pop, kind, src_gid, src_pop)
    return generate(panel.model, s), s
