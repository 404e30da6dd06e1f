"""Python binding of libibs (ctypes).  Argument marshalling only: every step of
the computation runs in the CUDA library; there is no Python or CPU fallback.

The functions carry the C ABI's names (include/ibs.h).  Buffers may be given
as torch tensors, numpy arrays or raw integer addresses.  A stream may be a
torch.cuda.Stream, a raw cudaStream_t integer, or None, which means torch's
current stream on the context's device.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "_build", "libibs.so")
HEADER = os.path.join(ROOT, "include", "ibs.h")

IBS_OK, IBS_EINVAL, IBS_ENOMEM, IBS_ECUDA, IBS_ETIMEOUT, IBS_EBUSY, IBS_ECANCELLED, IBS_ESTATE = range(8)
STATUS_NAMES = ["IBS_OK", "IBS_EINVAL", "IBS_ENOMEM", "IBS_ECUDA", "IBS_ETIMEOUT", "IBS_EBUSY", "IBS_ECANCELLED",
                "IBS_ESTATE"]
IBS_OUT_SQUARE = 0x1
IBS_NO_DIST = 0x2
IBS_KERNEL_PLAIN = 0x10
IBS_KERNEL_CSA = 0x20
IBS_TIMING = 0x40
IBS_KERNEL_TC = 0x80
IBS_TC_FP8 = 0x100
IBS_TC_FP4 = 0x200


class IbsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")


class ibs_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t), ("flags", ctypes.c_int),
                ("autotune_cache_path", ctypes.c_char_p)]


class ibs_subset(ctypes.Structure):
    _fields_ = [("sample_idx", ctypes.c_void_p), ("n", ctypes.c_int64), ("var_begin", ctypes.c_int64),
                ("var_len", ctypes.c_int64), ("out_counts", ctypes.c_void_p), ("out_dist", ctypes.c_void_p)]


class ibs_serve_stats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("peak_rows", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()


def declared_functions():
    """Names of the functions include/ibs.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:ibs_status|const char\*)\s+(ibs_\w+)\s*\(", text, re.M)))


def load():
    """Load libibs.so; raises if it was not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libibs.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                               "python -m paper_1410_4803_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        p, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int
        sig = {
            "ibs_init": [ctypes.POINTER(ibs_config), ctypes.POINTER(p)],
            "ibs_compute": [p, p, i64, i64, p, p, p],
            "ibs_compute_sz": [p, p, ctypes.c_size_t, i64, i64, p, ctypes.c_size_t, p, ctypes.c_size_t, p],
            "ibs_synchronize": [p, p],
            "ibs_compute_batch": [p, p, i64, i64, ctypes.POINTER(ibs_subset), i32, p],
            "ibs_panel_load": [p, p, i64, i64],
            "ibs_query": [p, p, i64, i32, p, p, p, ctypes.POINTER(ctypes.c_uint64)],
            "ibs_query_sync": [p, p, i64, i32, p, p, p],
            "ibs_wait": [p, ctypes.c_uint64, i64],
            "ibs_poll": [p, ctypes.c_uint64],
            "ibs_serve_stats_get": [p, ctypes.POINTER(ibs_serve_stats)],
            "ibs_shutdown": [p],
            "ibs_probe_int_pipes": [p, ctypes.POINTER(ctypes.c_double)],
            "ibs_probe_mma": [p, ctypes.POINTER(ctypes.c_double)],
            "ibs_batch_plan_info": [p, ctypes.POINTER(ctypes.c_int64)],
            "ibs_kernel_info": [p, ctypes.POINTER(ctypes.c_int64)],
            "ibs_compute_kernel": [p, i64, i64, ctypes.POINTER(ctypes.c_int64)],
            "ibs_ld_r": [p, p, i64, i64, i64, p, p, p],
            "ibs_cluster_complete": [p, p, i64, p, p],
            "ibs_grm": [p, p, i64, i64, p, p],
            "ibs_last_launch_info": [p, ctypes.POINTER(ctypes.c_int64)],
            "ibs_kernel_times": [p, ctypes.POINTER(ctypes.c_double)],
            "ibs_compute_noalloc": [p, i64, i64, p, p, p],
            "ibs_noalloc_status": [p],
            "ibs_test_set_wait_limit": [p, i64],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = st
        lib.ibs_last_error.argtypes = []
        lib.ibs_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def ibs_last_error() -> str:
    return load().ibs_last_error().decode(errors="replace")


def _check(status: int, where: str):
    if status != IBS_OK:
        raise IbsError(status, where, ibs_last_error())


def _addr(x):
    """Device/host address of a torch tensor, numpy array or integer (None -> 0)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s, device=None):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream(device).cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


class Context:
    """Owning handle of an ibs_ctx."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        ibs_shutdown(self)

    @property
    def _h(self):
        if self.handle is None:
            raise IbsError(IBS_ESTATE, "Context", "context was shut down")
        return self.handle


def ibs_init(device: int = 0, workspace_bytes: int = 0, flags: int = 0, autotune_cache_path: str | None = None):
    lib = load()
    cfg = ibs_config(device, workspace_bytes, flags,
                     autotune_cache_path.encode() if autotune_cache_path else None)
    h = ctypes.c_void_p()
    _check(lib.ibs_init(ctypes.byref(cfg), ctypes.byref(h)), "ibs_init")
    return Context(h, device)


def ibs_compute(ctx: Context, packed, n_samples: int, n_variants: int, out_counts, out_dist=None, stream=None):
    _check(load().ibs_compute(ctx._h, _addr(packed), n_samples, n_variants, _addr(out_counts), _addr(out_dist),
                              _stream(stream, ctx.device)), "ibs_compute")


def ibs_compute_sz(ctx: Context, packed, packed_bytes: int, n_samples: int, n_variants: int, out_counts,
                   counts_bytes: int, out_dist=None, dist_bytes: int = 0, stream=None):
    """ibs_compute with the buffers' byte sizes checked first (see include/ibs.h)."""
    _check(load().ibs_compute_sz(ctx._h, _addr(packed), packed_bytes, n_samples, n_variants, _addr(out_counts),
                                 counts_bytes, _addr(out_dist), dist_bytes, _stream(stream, ctx.device)),
           "ibs_compute_sz")


def ibs_compute_noalloc(packed, n_samples: int, n_variants: int, out_counts, out_dist=None, stream=None):
    """Allocation-free ibs_compute on the current device (fixed 64 MiB scratch; see include/ibs.h)."""
    _check(load().ibs_compute_noalloc(_addr(packed), n_samples, n_variants, _addr(out_counts), _addr(out_dist),
                                      _stream(stream)), "ibs_compute_noalloc")


def ibs_noalloc_status(stream=None):
    """Wait for `stream` and report a bounded device wait that expired in the
    last ibs_compute_noalloc call on it (IbsError with IBS_ETIMEOUT)."""
    _check(load().ibs_noalloc_status(_stream(stream)), "ibs_noalloc_status")


def ibs_synchronize(ctx: Context, stream=None):
    _check(load().ibs_synchronize(ctx._h, _stream(stream, ctx.device)), "ibs_synchronize")


def ibs_compute_batch(ctx: Context, pool_packed, pool_n: int, pool_m: int, subsets, stream=None):
    """subsets: sequence of (sample_idx, var_begin, var_len, out_counts, out_dist) with device buffers."""
    arr = (ibs_subset * len(subsets))()
    for i, (idx, vb, vl, oc, od) in enumerate(subsets):
        n = idx.numel() if hasattr(idx, "numel") else len(idx)
        arr[i] = ibs_subset(_addr(idx), n, vb, vl, _addr(oc), _addr(od))
    _check(load().ibs_compute_batch(ctx._h, _addr(pool_packed), pool_n, pool_m, arr, len(subsets),
                                    _stream(stream, ctx.device)), "ibs_compute_batch")


def ibs_panel_load(ctx: Context, panel_packed, n_panel: int, n_variants: int):
    _check(load().ibs_panel_load(ctx._h, _addr(panel_packed), n_panel, n_variants), "ibs_panel_load")


def ibs_query(ctx: Context, query_packed, n_query: int, k: int, out_counts, out_topk_idx, out_topk_dist) -> int:
    rid = ctypes.c_uint64()
    _check(load().ibs_query(ctx._h, _addr(query_packed), n_query, k, _addr(out_counts), _addr(out_topk_idx),
                            _addr(out_topk_dist), ctypes.byref(rid)), "ibs_query")
    return rid.value


def ibs_query_sync(ctx: Context, query_packed, n_query: int, k: int, out_counts, out_topk_idx, out_topk_dist):
    _check(load().ibs_query_sync(ctx._h, _addr(query_packed), n_query, k, _addr(out_counts), _addr(out_topk_idx),
                                 _addr(out_topk_dist)), "ibs_query_sync")


def ibs_wait(ctx: Context, req_id: int, timeout_ms: int = -1):
    _check(load().ibs_wait(ctx._h, req_id, timeout_ms), "ibs_wait")


def ibs_poll(ctx: Context, req_id: int) -> bool:
    st = load().ibs_poll(ctx._h, req_id)
    if st == IBS_EBUSY:
        return False
    _check(st, "ibs_poll")
    return True


def ibs_serve_stats_get(ctx: Context) -> dict:
    s = ibs_serve_stats()
    _check(load().ibs_serve_stats_get(ctx._h, ctypes.byref(s)), "ibs_serve_stats_get")
    return {f: getattr(s, f) for f, _ in s._fields_}


def ibs_shutdown(ctx: Context):
    if ctx.handle is not None:
        _check(load().ibs_shutdown(ctx.handle), "ibs_shutdown")
        ctx.handle = None


def ibs_probe_mma(ctx: Context) -> dict:
    out = (ctypes.c_double * 2)()
    _check(load().ibs_probe_mma(ctx._h, out), "ibs_probe_mma")
    return {"e4m3_tflops": out[0], "e2m1_tflops": out[1]}


def ibs_probe_int_pipes(ctx: Context) -> dict:
    out = (ctypes.c_double * 5)()
    _check(load().ibs_probe_int_pipes(ctx._h, out), "ibs_probe_int_pipes")
    return {"popc_per_clk_sm": out[0], "lop3_per_clk_sm": out[1], "iadd3_per_clk_sm": out[2], "sm_mhz": out[3],
            "sms": int(out[4])}


def ibs_last_launch_info(ctx: Context) -> dict:
    out = (ctypes.c_int64 * 3)()
    _check(load().ibs_last_launch_info(ctx._h, out), "ibs_last_launch_info")
    return {"launches": out[0], "tiles": out[1], "splits": out[2]}


def ibs_kernel_times(ctx: Context) -> dict:
    out = (ctypes.c_double * 4)()
    _check(load().ibs_kernel_times(ctx._h, out), "ibs_kernel_times")
    return {"planes_ms": out[0], "pairs_ms": out[1], "finalize_ms": out[2], "calls": int(out[3])}


def ibs_ld_r(ctx: Context, packed, n_samples: int, n_variants: int, window: int, out_r, out_n=None,
             stream=None) -> None:
    _check(load().ibs_ld_r(ctx._h, _addr(packed), n_samples, n_variants, window, _addr(out_r), _addr(out_n),
                           _stream(stream)), "ibs_ld_r")


def ibs_grm(ctx: Context, packed, n_samples: int, n_variants: int, out_grm, stream=None) -> None:
    _check(load().ibs_grm(ctx._h, _addr(packed), n_samples, n_variants, _addr(out_grm), _stream(stream)), "ibs_grm")


def grm(ctx: Context, packed, n_samples: int, n_variants: int, stream=None):
    """Allocate the upper triangle (with diagonal, float64) on the packed
    tensor's device and run ibs_grm."""
    import torch
    out = torch.empty(n_samples * (n_samples + 1) // 2, dtype=torch.float64, device=packed.device)
    ibs_grm(ctx, packed, n_samples, n_variants, out, stream)
    return out


def ibs_cluster_complete(ctx: Context, dist, n_samples: int, out_linkage, stream=None) -> None:
    _check(load().ibs_cluster_complete(ctx._h, _addr(dist), n_samples, _addr(out_linkage), _stream(stream)),
           "ibs_cluster_complete")


def cluster_complete(ctx: Context, dist, n_samples: int, stream=None):
    """Allocate the linkage [n-1][4] on dist's device and run ibs_cluster_complete."""
    import torch
    z = torch.empty((max(n_samples - 1, 0), 4), dtype=torch.float64, device=dist.device)
    ibs_cluster_complete(ctx, dist, n_samples, z, stream)
    return z


def ld_r(ctx: Context, packed, n_samples: int, n_variants: int, window: int, stream=None):
    """Allocate the outputs on the packed tensor's device and run ibs_ld_r:
    returns (r float64 [n_variants][window], N int32 [n_variants][window])."""
    import torch
    dev = packed.device
    r = torch.empty((n_variants, window), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_variants, window), dtype=torch.int32, device=dev)
    ibs_ld_r(ctx, packed, n_samples, n_variants, window, r, cnt, stream)
    return r, cnt


def ibs_kernel_info(ctx: Context) -> dict:
    out = (ctypes.c_int64 * 4)()
    _check(load().ibs_kernel_info(ctx._h, out), "ibs_kernel_info")
    return {"family": ("popc-plain", "popc-csa", "tensor-core")[out[0]], "tc_format": ("e4m3", "e2m1")[out[1]],
            "sms": out[2], "device": out[3]}


COMPUTE_KERNELS = ("popc-plain", "popc-csa", "tc-persistent", "tc-pair", "tc-tile")


def ibs_compute_kernel(ctx: Context, n_samples: int, n_variants: int) -> str:
    """The pair kernel ibs_compute runs on this context for an n x m matrix:
    one of COMPUTE_KERNELS ('tc-pair' is the two-SM cta_group::2 kernel)."""
    out = ctypes.c_int64()
    _check(load().ibs_compute_kernel(ctx._h, n_samples, n_variants, ctypes.byref(out)), "ibs_compute_kernel")
    return COMPUTE_KERNELS[out.value]


def ibs_test_set_wait_limit(ctx: Context, ns: int):
    """Testing hook: bound (ns) of the pipeline waits of ibs_compute's
    persistent pair kernels on this context; 0 restores the 2 s default."""
    _check(load().ibs_test_set_wait_limit(ctx._h, ns), "ibs_test_set_wait_limit")


def ibs_batch_plan_info(ctx: Context) -> dict:
    out = (ctypes.c_int64 * 5)()
    _check(load().ibs_batch_plan_info(ctx._h, out), "ibs_batch_plan_info")
    return {"mode": out[0], "split_policy": out[1], "items": out[2], "grid": out[3], "pair_min_chunks": out[4]}


# ---------------------------------------------------------------------------
# Convenience wrappers over torch tensors (allocation and the calls above).

def n_pairs(n: int) -> int:
    return n * (n + 1) // 2


def compute(ctx: Context, packed, n: int, m: int, with_dist: bool = True, stream=None, square: bool = False):
    """Allocate outputs on packed's device and run ibs_compute; returns (counts, dist)."""
    import torch
    P = n * n if square else n_pairs(n)
    counts = torch.empty((P, 4), dtype=torch.int32, device=packed.device)
    dist = torch.empty(P, dtype=torch.float64, device=packed.device) if with_dist else None
    ibs_compute(ctx, packed, n, m, counts, dist, stream)
    return counts, dist
