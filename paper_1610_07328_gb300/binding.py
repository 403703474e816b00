"""Thin ctypes binding of include/ssh.h (argument marshalling only).

Every function here has the name of the C entry point it calls. Host arrays are
numpy arrays; device arrays are CUDA torch tensors (torch supplies device
memory and the current stream, nothing else). Errors raise SSHError with the
status name and the library's one-line reason. There is no fallback: if the
CUDA library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build_ext

SSH_OK, SSH_EINVAL, SSH_ENOMEM, SSH_ECUDA, SSH_ELENGTH, SSH_EBUSY, SSH_ETIMEOUT, SSH_ENOTSUP = range(8)
SSH_ADD_BORROW = 1
SSH_OPT_LB_PRUNE = 1
SSH_OPT_KERNEL_TIMING = 2
SSH_OPT_HASH_KERNEL = 3
SSH_OPT_CWS_FP64 = 4
SSH_OPT_EXACT_SCAN = 5
SSH_OPT_LB_CASCADE = 6
SSH_OPT_MINHASH = 7

_lib = None
_lock = threading.Lock()


class SSHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


class ssh_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "series_hashed", "sketch_fp64", "cws_fp64", "queries", "candidates", "dtw_computed", "lb_pruned",
        "kernel_launches", "lb2_pruned", "lb2_skipped")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ssh_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("calls", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("units", ctypes.c_double)]


class ssh_server_stats(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int64), ("queries_submitted", ctypes.c_int64), ("queries_done", ctypes.c_int64),
                ("errors", ctypes.c_int64), ("batches", ctypes.c_int64), ("max_inflight", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("inserts_submitted", ctypes.c_int64),
                ("inserts_applied", ctypes.c_int64), ("insert_errors", ctypes.c_int64),
                ("insert_batches", ctypes.c_int64), ("insert_latency_ms_sum", ctypes.c_double),
                ("max_inflight_device", ctypes.c_int64), ("deferred", ctypes.c_int64), ("refused", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "ssh_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ssh_last_error": (ctypes.c_char_p, []),
    "ssh_create": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "ssh_create_srp": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                                      ctypes.POINTER(_P)]),
    "ssh_destroy": (None, [_P]),
    "ssh_get_filter": (ctypes.c_int, [_P, _P]),
    "ssh_index_add": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _I64P]),
    "ssh_index_add_device": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_uint32, _P, _I64P]),
    "ssh_index_add_windows_device": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P,
                                                    _I64P]),
    "ssh_index_clear": (ctypes.c_int, [_P]),
    "ssh_index_size": (ctypes.c_int, [_P, _I64P]),
    "ssh_query": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int, _P, _P]),
    "ssh_query_device": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int, _P, _P, _P]),
    "ssh_group_query_device": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int64, ctypes.c_int, _P, _P, _P, _P]),
    "ssh_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                        ctypes.POINTER(_P)]),
    "ssh_batch_query": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "ssh_batch_stats": (ctypes.c_int, [_P, _I64P, _I64P, _I64P, ctypes.POINTER(ctypes.c_int32)]),
    "ssh_batch_destroy": (None, [_P]),
    "ssh_batch_set_persistent": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ssh_server_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                         ctypes.POINTER(_P)]),
    "ssh_server_create_ex": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(_P)]),
    "ssh_server_now": (ctypes.c_double, [_P]),
    "ssh_server_submit": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "ssh_server_insert": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64]),
    "ssh_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P]),
    "ssh_server_collect": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P, _P, _P]),
    "ssh_server_flush": (ctypes.c_int, [_P, ctypes.c_double]),
    "ssh_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ssh_server_stats)]),
    "ssh_server_destroy": (None, [_P]),
    "ssh_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    "ssh_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ssh_stats)]),
    "ssh_reset_stats": (ctypes.c_int, [_P]),
    "ssh_get_kernel_times": (ctypes.c_int, [_P, ctypes.POINTER(ssh_kernel_time), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "ssh_hash_device": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, _P] + [_P] * 7),
    "ssh_hash_device_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, _P] + [_P] * 7),
    "ssh_dtw_device": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "ssh_dtw_device_tiled": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "ssh_lb_keogh_device": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "ssh_lb_bound_device": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, _P, _P]),
    "ssh_read_device": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32, _P]),
}
EXPORTED = tuple(_SIGS)


def lib_path() -> str:
    return build_ext.LIB


def load(build: bool = True):
    """Load libssh_gb300.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build_ext.build() if build else build_ext.LIB
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_name(s: int) -> str:
    names = ["SSH_OK", "SSH_EINVAL", "SSH_ENOMEM", "SSH_ECUDA", "SSH_ELENGTH", "SSH_EBUSY", "SSH_ETIMEOUT",
             "SSH_ENOTSUP"]
    return names[s] if 0 <= s < len(names) else f"SSH_STATUS_{s}"


def _check(status: int):
    if status != SSH_OK:
        raise SSHError(status, load().ssh_last_error().decode())


def _host_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


# ------------------------------------------------------------ entry points

def ssh_create(W: int, delta: int, n: int, K: int, L: int, band: float, seed: int) -> ctypes.c_void_p:
    h = _P()
    _check(load().ssh_create(W, delta, n, K, L, float(band), int(seed) & (2 ** 64 - 1), ctypes.byref(h)))
    return h


def ssh_create_srp(K: int, L: int, band: float, seed: int) -> ctypes.c_void_p:
    h = _P()
    _check(load().ssh_create_srp(K, L, float(band), int(seed) & (2 ** 64 - 1), ctypes.byref(h)))
    return h


def ssh_destroy(h) -> None:
    if h:
        load().ssh_destroy(h)


def ssh_get_filter(h, W: int) -> np.ndarray:
    out = np.zeros(W, np.float32)
    _check(load().ssh_get_filter(h, _host_ptr(out)))
    return out


def ssh_index_add(h, series: np.ndarray, lengths: np.ndarray) -> int:
    s = np.ascontiguousarray(series, dtype=np.float32).reshape(-1)
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    first = ctypes.c_int64()
    _check(load().ssh_index_add(h, _host_ptr(s), _host_ptr(ln), len(ln), ctypes.byref(first)))
    return first.value


def ssh_index_add_device(h, d_series, lengths: np.ndarray, flags: int = 0, stream=None) -> int:
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    first = ctypes.c_int64()
    _check(load().ssh_index_add_device(h, _dev_ptr(d_series), _host_ptr(ln), len(ln), flags, _stream(stream),
                                       ctypes.byref(first)))
    return first.value


def ssh_index_clear(h) -> None:
    _check(load().ssh_index_clear(h))


def ssh_index_size(h) -> int:
    c = ctypes.c_int64()
    _check(load().ssh_index_size(h, ctypes.byref(c)))
    return c.value


def ssh_query(h, queries: np.ndarray, lengths: np.ndarray, k: int):
    q = np.ascontiguousarray(queries, dtype=np.float32).reshape(-1)
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    nq = len(ln)
    ids = np.zeros((nq, k), np.int64)
    dists = np.zeros((nq, k), np.float32)
    _check(load().ssh_query(h, _host_ptr(q), _host_ptr(ln), nq, k, _host_ptr(ids), _host_ptr(dists)))
    return ids, dists


def ssh_query_device(h, d_queries, lengths: np.ndarray, k: int, d_ids, d_dists, stream=None) -> None:
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    _check(load().ssh_query_device(h, _dev_ptr(d_queries), _host_ptr(ln), len(ln), k, _dev_ptr(d_ids),
                                   _dev_ptr(d_dists), _stream(stream)))


def ssh_group_query_device(handles, d_queries, lengths: np.ndarray, k: int, d_ids, d_dists, d_which=None,
                           stream=None) -> None:
    """Queries of mixed lengths over several indexes (one per length and filter length)."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    _check(load().ssh_group_query_device(ctypes.cast(arr, ctypes.c_void_p), len(handles), _dev_ptr(d_queries),
                                         _host_ptr(ln), len(ln), k, _dev_ptr(d_ids), _dev_ptr(d_dists),
                                         _dev_ptr(d_which), _stream(stream)))


def ssh_batch_create(handles, max_queries: int, k: int, max_pairs: int = 0):
    """A batch plan over the indexes `handles` (see include/ssh.h)."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    out = _P()
    _check(load().ssh_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(handles), max_queries, k, max_pairs,
                                   ctypes.byref(out)))
    return out


def ssh_batch_query(b, d_queries, lengths: np.ndarray, d_ids, d_dists, d_which=None, stream=None) -> None:
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    _check(load().ssh_batch_query(b, _dev_ptr(d_queries), _host_ptr(ln), len(ln), _dev_ptr(d_ids), _dev_ptr(d_dists),
                                  _dev_ptr(d_which), _stream(stream)))


def ssh_batch_stats(b) -> dict:
    pairs, dtw, cap = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    nk = ctypes.c_int32()
    _check(load().ssh_batch_stats(b, ctypes.byref(pairs), ctypes.byref(dtw), ctypes.byref(cap), ctypes.byref(nk)))
    return dict(pairs=pairs.value, dtw=dtw.value, pair_capacity=cap.value, graph_kernels=nk.value)


def ssh_batch_destroy(b) -> None:
    if b:
        load().ssh_batch_destroy(b)


class SSHBatch:
    """Owning wrapper around an ssh_batch plan."""

    def __init__(self, indexes, max_queries: int, k: int, max_pairs: int = 0):
        self.k = k
        self.indexes = list(indexes)  # kept alive for the plan's lifetime
        self.handle = ssh_batch_create([ix.handle for ix in self.indexes], max_queries, k, max_pairs)

    def query(self, d_queries, lengths, d_ids, d_dists, d_which=None, stream=None):
        ssh_batch_query(self.handle, d_queries, lengths, d_ids, d_dists, d_which, stream)

    def stats(self) -> dict:
        return ssh_batch_stats(self.handle)

    def set_persistent(self, on) -> None:
        """The rerank as one persistent launch (True), as per-class kernels (False), or by batch
        size (None, the default: persistent up to 512 queries)."""
        _check(load().ssh_batch_set_persistent(self.handle, -1 if on is None else (1 if on else 0)))

    def close(self):
        if self.handle:
            ssh_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SSHServer:
    """Owning wrapper around an ssh_server (serving loop with continuous batching)."""

    def __init__(self, indexes, k: int, max_batch: int = 256, max_slots: int = 4, reserve_bytes: int = 1 << 30,
                 max_pairs: int = 0):
        self.k = k
        self.indexes = list(indexes)  # kept alive for the server's lifetime
        arr = (ctypes.c_void_p * len(self.indexes))(*[ix.handle.value if isinstance(ix.handle, ctypes.c_void_p)
                                                       else ix.handle for ix in self.indexes])
        out = _P()
        _check(load().ssh_server_create_ex(ctypes.cast(arr, ctypes.c_void_p), len(self.indexes), k, max_batch,
                                           max_slots, reserve_bytes, max_pairs, ctypes.byref(out)))
        self.handle = out

    def now(self) -> float:
        return load().ssh_server_now(self.handle)

    def submit(self, queries: np.ndarray, lengths: np.ndarray, arrival_s: np.ndarray | None = None) -> np.ndarray:
        q = np.ascontiguousarray(queries, dtype=np.float32).reshape(-1)
        ln = np.ascontiguousarray(lengths, dtype=np.int32)
        tickets = np.zeros(len(ln), np.int64)
        arr = None if arrival_s is None else np.ascontiguousarray(arrival_s, dtype=np.float64)
        _check(load().ssh_server_submit(self.handle, _host_ptr(q), _host_ptr(ln), len(ln),
                                        None if arr is None else _host_ptr(arr), _host_ptr(tickets)))
        return tickets

    def insert(self, series: np.ndarray, lengths: np.ndarray) -> None:
        x = np.ascontiguousarray(series, dtype=np.float32).reshape(-1)
        ln = np.ascontiguousarray(lengths, dtype=np.int32)
        _check(load().ssh_server_insert(self.handle, _host_ptr(x), _host_ptr(ln), len(ln)))

    def wait(self, ticket: int, timeout_s: float = 10.0):
        ids = np.zeros(self.k, np.int64)
        dists = np.zeros(self.k, np.float32)
        which = ctypes.c_int32()
        lat = ctypes.c_double()
        _check(load().ssh_server_wait(self.handle, int(ticket), timeout_s, _host_ptr(ids), _host_ptr(dists),
                                      ctypes.byref(which), ctypes.byref(lat)))
        return ids, dists, which.value, lat.value

    def collect(self, max_n: int = 4096, timeout_s: float = 0.01):
        tickets = np.zeros(max_n, np.int64)
        ids = np.zeros((max_n, self.k), np.int64)
        dists = np.zeros((max_n, self.k), np.float32)
        lat = np.zeros(max_n, np.float64)
        status = np.zeros(max_n, np.int32)
        n = ctypes.c_int64()
        _check(load().ssh_server_collect(self.handle, max_n, timeout_s, _host_ptr(tickets), _host_ptr(ids),
                                         _host_ptr(dists), _host_ptr(lat), _host_ptr(status), ctypes.byref(n)))
        c = n.value
        return tickets[:c], ids[:c], dists[:c], lat[:c], status[:c]

    def flush(self, timeout_s: float = 60.0) -> None:
        _check(load().ssh_server_flush(self.handle, timeout_s))

    def stats(self) -> dict:
        st = ssh_server_stats()
        _check(load().ssh_server_get_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.handle:
            load().ssh_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ssh_set_option(h, opt: int, value: int) -> None:
    _check(load().ssh_set_option(h, opt, int(value)))


def ssh_get_stats(h) -> dict:
    st = ssh_stats()
    _check(load().ssh_get_stats(h, ctypes.byref(st)))
    return st.as_dict()


def ssh_reset_stats(h) -> None:
    _check(load().ssh_reset_stats(h))


def ssh_get_kernel_times(h) -> dict:
    """{group: {"launches", "calls", "total_ms", "units"}} since the last reset."""
    cap = 32
    arr = (ssh_kernel_time * cap)()
    n = ctypes.c_int()
    _check(load().ssh_get_kernel_times(h, arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): dict(launches=int(arr[i].launches), calls=int(arr[i].calls),
                                       total_ms=float(arr[i].total_ms), units=float(arr[i].units))
            for i in range(min(n.value, cap))}


def ssh_hash_device(h, d_series, m: int, count: int, d_bits=None, d_sh_ids=None, d_sh_counts=None, d_nnz=None,
                    d_kstar=None, d_tstar=None, d_keys=None, stream=None) -> None:
    _check(load().ssh_hash_device(h, _dev_ptr(d_series), m, count, _stream(stream), _dev_ptr(d_bits),
                                  _dev_ptr(d_sh_ids), _dev_ptr(d_sh_counts), _dev_ptr(d_nnz), _dev_ptr(d_kstar),
                                  _dev_ptr(d_tstar), _dev_ptr(d_keys)))


def ssh_hash_device_noalloc(h, d_series, m: int, count: int, d_bits=None, d_sh_ids=None, d_sh_counts=None,
                            d_nnz=None, d_kstar=None, d_tstar=None, d_keys=None, stream=None) -> None:
    """ssh_hash_device with its scratch in the library's fixed device array (no allocation)."""
    _check(load().ssh_hash_device_noalloc(h, _dev_ptr(d_series), m, count, _stream(stream), _dev_ptr(d_bits),
                                          _dev_ptr(d_sh_ids), _dev_ptr(d_sh_counts), _dev_ptr(d_nnz),
                                          _dev_ptr(d_kstar), _dev_ptr(d_tstar), _dev_ptr(d_keys)))


def ssh_dtw_device(d_a, d_a_idx, d_b, d_b_idx, m: int, rb: int, d_out, stream=None) -> None:
    _check(load().ssh_dtw_device(_dev_ptr(d_a), _dev_ptr(d_a_idx), _dev_ptr(d_b), _dev_ptr(d_b_idx),
                                 d_a_idx.numel(), m, rb, _dev_ptr(d_out), _stream(stream)))


def ssh_dtw_device_tiled(d_a, d_a_idx, d_b, d_b_idx, m: int, rb: int, S: int, variant: int, d_out,
                         stream=None) -> None:
    """ssh_dtw_device with the tiling (S slots per lane, kernel variant) given explicitly."""
    _check(load().ssh_dtw_device_tiled(_dev_ptr(d_a), _dev_ptr(d_a_idx), _dev_ptr(d_b), _dev_ptr(d_b_idx),
                                       d_a_idx.numel(), m, rb, S, variant, _dev_ptr(d_out), _stream(stream)))


def ssh_lb_keogh_device(d_a, d_a_idx, d_b, d_b_idx, m: int, rb: int, d_out, stream=None) -> None:
    _check(load().ssh_lb_keogh_device(_dev_ptr(d_a), _dev_ptr(d_a_idx), _dev_ptr(d_b), _dev_ptr(d_b_idx),
                                      d_a_idx.numel(), m, rb, _dev_ptr(d_out), _stream(stream)))


def ssh_lb_bound_device(d_a, d_a_idx, d_b, d_b_idx, m: int, rb: int, kind: int, d_out, stream=None) -> None:
    """Lower bounds of the banded DTW: kind 0 LB_Keogh, 1 with the LB_Kim endpoints, 2 reversed."""
    _check(load().ssh_lb_bound_device(_dev_ptr(d_a), _dev_ptr(d_a_idx), _dev_ptr(d_b), _dev_ptr(d_b_idx),
                                      d_a_idx.numel(), m, rb, kind, _dev_ptr(d_out), _stream(stream)))


def ssh_read_device(d_buf, passes: int, stream=None) -> None:
    """Enqueue `passes` L1-bypassing reads of the whole of d_buf (a measurement helper)."""
    _check(load().ssh_read_device(_dev_ptr(d_buf), d_buf.numel() * d_buf.element_size(), passes,
                                  _stream(stream)))


# ------------------------------------------------------------ convenience

class SSHIndex:
    """Owning wrapper around an ssh_index handle."""

    def __init__(self, W: int, delta: int, n: int, K: int, L: int, band: float, seed: int = 0):
        self.W, self.delta, self.n, self.K, self.L = W, delta, n, K, L
        self.band, self.seed = band, seed
        self.handle = ssh_create(W, delta, n, K, L, band, seed)

    @classmethod
    def srp(cls, K: int, L: int, band: float, seed: int = 0) -> "SSHIndex":
        """The paper's SRP baseline behind the same index API (ssh_create_srp)."""
        self = cls.__new__(cls)
        self.W, self.delta, self.n, self.K, self.L = 1, 1, 1, K, L
        self.band, self.seed = band, seed
        self.handle = ssh_create_srp(K, L, band, seed)
        return self

    def close(self):
        if self.handle:
            ssh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def filter(self) -> np.ndarray:
        return ssh_get_filter(self.handle, self.W)

    def add(self, series: np.ndarray, lengths=None) -> int:
        series = np.asarray(series, np.float32)
        if lengths is None:
            lengths = np.full(series.shape[0], series.shape[1], np.int32)
        return ssh_index_add(self.handle, series, lengths)

    def add_device(self, d_series, lengths=None, borrow: bool = False, stream=None) -> int:
        if lengths is None:
            lengths = np.full(d_series.shape[0], d_series.shape[1], np.int32)
        return ssh_index_add_device(self.handle, d_series, lengths, SSH_ADD_BORROW if borrow else 0, stream)

    def add_windows_device(self, d_stream, t: int, step: int = 1, stream=None) -> int:
        """Every length-t window of the 1-D device tensor d_stream at offsets 0, step, 2 step, ...
        (borrowed: keep d_stream alive and unchanged); returns the first window's id."""
        first = ctypes.c_int64(0)
        _check(load().ssh_index_add_windows_device(self.handle, _dev_ptr(d_stream), d_stream.numel(), t, step,
                                                   _stream(stream), ctypes.byref(first)))
        return first.value

    def clear(self):
        ssh_index_clear(self.handle)

    def __len__(self):
        return ssh_index_size(self.handle)

    def query(self, queries: np.ndarray, k: int, lengths=None):
        queries = np.asarray(queries, np.float32)
        if lengths is None:
            lengths = np.full(queries.shape[0], queries.shape[1], np.int32)
        return ssh_query(self.handle, queries, lengths, k)

    def query_device(self, d_queries, k: int, d_ids, d_dists, lengths=None, stream=None):
        if lengths is None:
            lengths = np.full(d_queries.shape[0], d_queries.shape[1], np.int32)
        ssh_query_device(self.handle, d_queries, lengths, k, d_ids, d_dists, stream)

    def set_lb_prune(self, on: bool):
        ssh_set_option(self.handle, SSH_OPT_LB_PRUNE, 1 if on else 0)

    def set_hash_kernel(self, generic: bool):
        ssh_set_option(self.handle, SSH_OPT_HASH_KERNEL, 1 if generic else 0)

    def set_cws_fp64(self, on: bool):
        ssh_set_option(self.handle, SSH_OPT_CWS_FP64, 1 if on else 0)

    def set_exact_scan(self, on: bool):
        """Rank every stored series of the query's length (exact top-k, no hashing)."""
        ssh_set_option(self.handle, SSH_OPT_EXACT_SCAN, 1 if on else 0)

    def set_minhash(self, kind: int):
        """0 ICWS (default), 1 densified one-permutation hashing (only on an empty index)."""
        ssh_set_option(self.handle, SSH_OPT_MINHASH, int(kind))

    def set_lb_cascade(self, mode):
        """0 LB_Keogh alone, 1 with the LB_Kim endpoints (default), 2 + reversed LB_Keogh;
        True / False select 2 / 0."""
        mode = {True: 2, False: 0}.get(mode, mode) if isinstance(mode, bool) else int(mode)
        ssh_set_option(self.handle, SSH_OPT_LB_CASCADE, mode)

    def set_kernel_timing(self, on: bool):
        ssh_set_option(self.handle, SSH_OPT_KERNEL_TIMING, 1 if on else 0)

    def kernel_times(self) -> dict:
        return ssh_get_kernel_times(self.handle)

    def stats(self) -> dict:
        return ssh_get_stats(self.handle)

    def reset_stats(self):
        ssh_reset_stats(self.handle)
