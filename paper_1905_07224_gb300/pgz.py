"""Thin ctypes binding of libpgz (include/pgz.h), same names as the C ABI.

Argument marshalling only: every step of the decompression runs in the CUDA
kernels of libpgz.so.  Device buffers are passed as integer addresses (e.g.
``tensor.data_ptr()``), host buffers as numpy arrays or bytes.  Importing this
module raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpgz.so")

PGZ_OK = 0
PGZ_E_ARG, PGZ_E_HEADER, PGZ_E_DATA, PGZ_E_CRC, PGZ_E_ISIZE, PGZ_E_CAPACITY = 1, 2, 3, 4, 5, 6
PGZ_E_NOSYNC, PGZ_E_UNSUPPORTED, PGZ_E_TIMEOUT, PGZ_E_CUDA, PGZ_E_NOMEM, PGZ_E_ABORTED = 7, 8, 9, 10, 11, 12
# int sink(void* user, const uint8_t* bytes, uint64_t n)
PGZ_SINK = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64)
NONE = (1 << 64) - 1

U64 = ctypes.c_uint64
VP = ctypes.c_void_p


class pgz_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", VP), ("chunk_bytes", U64), ("n_chunks", ctypes.c_int),
                ("threads_per_chunk", ctypes.c_int), ("allowed", ctypes.c_uint8 * 32),
                ("confirm_blocks", ctypes.c_int), ("min_block", ctypes.c_uint32), ("max_block", ctypes.c_uint32),
                ("dev_mem_budget", U64), ("spin_cap", U64), ("warps_per_block", ctypes.c_int),
                ("exec_pipelined", ctypes.c_int), ("determined_tail", ctypes.c_int)]


class pgz_stats(ctypes.Structure):
    _fields_ = [("in_bytes", U64), ("out_bytes", U64), ("chunks", U64), ("empty_chunks", U64),
                ("false_syncs", U64), ("retries", U64), ("placeholders", U64), ("symbols", U64),
                ("ms_sync", ctypes.c_float), ("ms_inflate", ctypes.c_float), ("ms_chain", ctypes.c_float),
                ("ms_translate", ctypes.c_float), ("ms_crc", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("determined", U64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pgz_tune_entry(ctypes.Structure):
    _fields_ = [("chunk_bytes", U64), ("warps_per_block", ctypes.c_int), ("exec_pipelined", ctypes.c_int),
                ("status", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pgz_request(ctypes.Structure):
    _fields_ = [("file", ctypes.c_int), ("whole", ctypes.c_int), ("offset", U64), ("length", U64), ("out", VP),
                ("out_cap", U64), ("status", ctypes.c_int), ("out_len", U64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class pgz_job(ctypes.Structure):
    _fields_ = [("gz", VP), ("gz_len", U64), ("out", VP), ("out_cap", U64), ("out_len", U64),
                ("status", ctypes.c_int)]


class pgz_part_state(ctypes.Structure):
    _fields_ = [("lo", U64), ("given", ctypes.c_int32), ("probe", ctypes.c_int32), ("disabled", ctypes.c_int32),
                ("confirm_ext", ctypes.c_int32), ("state", ctypes.c_int32), ("err", ctypes.c_int32),
                ("sync", U64), ("end", U64), ("blocks", ctypes.c_uint32), ("confirmed", ctypes.c_uint32)]


PGZ_PART_FOUND, PGZ_PART_EMPTY, PGZ_PART_DONE, PGZ_PART_ERROR = 1, 2, 3, 4
(PGZ_PART_OK, PGZ_PART_DATA, PGZ_PART_TRUNC, PGZ_PART_DIST, PGZ_PART_OVERFLOW, PGZ_PART_CHAIN, PGZ_PART_CONFIRM,
 PGZ_PART_TRAIL) = range(8)
PGZ_RECOVER_STOP, PGZ_RECOVER_RERUN, PGZ_RECOVER_GROW = 0, 1, 2


class PgzError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {pgz_strerror(status)} ({status})" if what else pgz_strerror(status))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpgz.so is not built ({LIB_PATH}); run paper_1905_07224_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "pgz_config_init": (None, [P(pgz_config)]),
        "pgz_create": (ctypes.c_int, [P(VP), P(pgz_config)]),
        "pgz_destroy": (None, [VP]),
        "pgz_decompress": (ctypes.c_int, [VP, VP, U64, VP, U64, P(U64), P(pgz_stats)]),
        "pgz_decompress_host": (ctypes.c_int, [VP, VP, U64, VP, U64, P(U64), P(pgz_stats)]),
        "pgz_decompress_stream": (ctypes.c_int, [VP, VP, U64, U64, PGZ_SINK, VP, P(U64), P(pgz_stats)]),
        "pgz_set_tuning": (ctypes.c_int, [VP, U64, ctypes.c_int, ctypes.c_int]),
        "pgz_decompress_at": (ctypes.c_int, [VP, VP, U64, U64, VP, VP, ctypes.c_uint8, U64, P(U64), P(U64), P(U64)]),
        "pgz_decompress_batch": (ctypes.c_int, [VP, ctypes.c_int, P(pgz_job), P(pgz_stats)]),
        "pgz_decompress_batch_host": (ctypes.c_int, [VP, ctypes.c_int, P(pgz_job), P(pgz_stats)]),
        "pgz_wave_chunk_bytes": (ctypes.c_int, [VP, P(pgz_job), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                P(U64), P(ctypes.c_int)]),
        "pgz_batch_prepare": (ctypes.c_int, [VP, ctypes.c_int, P(pgz_job), P(VP)]),
        "pgz_batch_run": (ctypes.c_int, [VP, P(pgz_job), P(pgz_stats)]),
        "pgz_batch_free": (None, [VP]),
        "pgz_index_build": (ctypes.c_int, [VP, VP, U64, P(VP)]),
        "pgz_index_info": (ctypes.c_int, [VP, P(U64), P(U64)]),
        "pgz_decompress_range": (ctypes.c_int, [VP, VP, U64, U64, VP]),
        "pgz_index_free": (None, [VP]),
        "pgz_inspect_parts": (ctypes.c_int, [VP, ctypes.c_int, VP, VP, VP, P(ctypes.c_int)]),
        "pgz_inspect_symbols": (ctypes.c_int, [VP, ctypes.c_int, VP, U64, P(U64)]),
        "pgz_inspect_window": (ctypes.c_int, [VP, ctypes.c_int, VP]),
        "pgz_kernel_launches": (U64, [VP]),
        "pgz_decompress_noalloc": (ctypes.c_int, [VP, U64, VP, U64, P(U64), VP]),
        "pgz_autotune": (ctypes.c_int, [VP, P(pgz_job), ctypes.c_int, P(U64), ctypes.c_int, P(ctypes.c_int),
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, P(pgz_tune_entry),
                                        P(pgz_tune_entry)]),
        "pgz_server_create": (ctypes.c_int, [P(VP), P(pgz_config), ctypes.c_int, U64]),
        "pgz_server_add_file": (ctypes.c_int, [VP, VP, U64, P(ctypes.c_int)]),
        "pgz_server_submit": (ctypes.c_int, [VP, P(pgz_request)]),
        "pgz_server_poll": (ctypes.c_int, [VP, P(ctypes.c_int)]),
        "pgz_server_drain": (ctypes.c_int, [VP]),
        "pgz_server_pending": (ctypes.c_int, [VP]),
        "pgz_server_destroy": (None, [VP]),
        "pgz_extract_sequences": (ctypes.c_int, [VP, VP, U64, ctypes.c_uint32, VP, U64, P(U64), P(U64)]),
        "pgz_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "pgz_recover_step": (ctypes.c_int, [ctypes.c_int, P(pgz_part_state), U64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, P(U64), P(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


EXPORTED = ["pgz_config_init", "pgz_create", "pgz_destroy", "pgz_decompress", "pgz_decompress_host",
            "pgz_decompress_at", "pgz_decompress_batch", "pgz_decompress_batch_host", "pgz_batch_prepare", "pgz_batch_run", "pgz_batch_free",
            "pgz_index_build", "pgz_index_info", "pgz_decompress_range", "pgz_index_free", "pgz_inspect_parts",
            "pgz_inspect_symbols", "pgz_inspect_window", "pgz_kernel_launches", "pgz_strerror",
            "pgz_decompress_noalloc", "pgz_autotune", "pgz_server_create", "pgz_server_add_file",
            "pgz_server_submit", "pgz_server_poll", "pgz_server_drain", "pgz_server_pending", "pgz_server_destroy",
            "pgz_extract_sequences", "pgz_decompress_stream", "pgz_set_tuning", "pgz_wave_chunk_bytes",
            "pgz_recover_step"]


def pgz_strerror(status: int) -> str:
    return lib().pgz_strerror(status).decode()


def pgz_config_init(**overrides) -> pgz_config:
    cfg = pgz_config()
    lib().pgz_config_init(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "allowed":
            for i in range(32):
                cfg.allowed[i] = int(v[i])
        else:
            setattr(cfg, k, v)
    return cfg


def pgz_create(cfg: pgz_config) -> int:
    h = VP()
    st = lib().pgz_create(ctypes.byref(h), ctypes.byref(cfg))
    if st:
        raise PgzError(st, "pgz_create")
    return h.value


def pgz_destroy(ctx: int) -> None:
    lib().pgz_destroy(ctx)


def pgz_decompress(ctx: int, gz_ptr: int, gz_len: int, out_ptr: int, out_cap: int, stats: bool = False):
    """(status, out_len, stats dict or None); device addresses."""
    n = U64(0)
    st = pgz_stats() if stats else None
    r = lib().pgz_decompress(ctx, gz_ptr, gz_len, out_ptr, out_cap, ctypes.byref(n),
                             ctypes.byref(st) if st is not None else None)
    return r, n.value, (st.as_dict() if st is not None else None)


def pgz_decompress_host(ctx: int, gz, out: np.ndarray, stats: bool = False):
    """(status, out_len, stats); gz: bytes/uint8 array in host memory, out: uint8 array."""
    a = np.frombuffer(gz, dtype=np.uint8) if isinstance(gz, (bytes, bytearray)) else np.ascontiguousarray(gz)
    n = U64(0)
    st = pgz_stats() if stats else None
    r = lib().pgz_decompress_host(ctx, a.ctypes.data, a.size, out.ctypes.data, out.size, ctypes.byref(n),
                                  ctypes.byref(st) if st is not None else None)
    return r, n.value, (st.as_dict() if st is not None else None)


def pgz_set_tuning(ctx: int, chunk_bytes: int, warps_per_block: int, exec_pipelined: int) -> int:
    """Applies a part size, CTA shape and execution form chosen earlier; returns the status."""
    return lib().pgz_set_tuning(ctx, chunk_bytes, warps_per_block, exec_pipelined)


def pgz_decompress_stream(ctx: int, gz, segment_bytes: int = 0, sink=None, stats: bool = False):
    """(status, out_len, stats, out); gz: bytes/uint8 array in host memory.  sink(memoryview) receives the
    output segment by segment (a truthy return stops the decode); without a sink the output is collected
    and returned as bytes in `out`."""
    a = np.frombuffer(gz, dtype=np.uint8) if isinstance(gz, (bytes, bytearray)) else np.ascontiguousarray(gz)
    parts = []
    raised = []

    def _cb(_user, p, n):
        view = (ctypes.c_uint8 * n).from_address(p)
        if sink is None:
            parts.append(bytes(view))
            return 0
        try:
            return 1 if sink(memoryview(view)) else 0
        except BaseException as exc:                 # stop the decode; re-raised after the call returns
            raised.append(exc)
            return 1

    cb = PGZ_SINK(_cb)
    n = U64(0)
    st = pgz_stats() if stats else None
    r = lib().pgz_decompress_stream(ctx, a.ctypes.data, a.size, segment_bytes, cb, None, ctypes.byref(n),
                                    ctypes.byref(st) if st is not None else None)
    if raised:
        raise raised[0]
    return r, n.value, (st.as_dict() if st is not None else None), (b"".join(parts) if sink is None else None)


def pgz_decompress_at(ctx: int, gz_ptr: int, gz_len: int, start_bit: int, sym_ptr: int | None,
                      byte_ptr: int | None, fill: int, out_cap: int):
    """(status, out_len, block_bit, first_determined); device addresses."""
    n, bb, fd = U64(0), U64(0), U64(0)
    r = lib().pgz_decompress_at(ctx, gz_ptr, gz_len, start_bit, sym_ptr, byte_ptr, fill, out_cap,
                                ctypes.byref(n), ctypes.byref(bb), ctypes.byref(fd))
    return r, n.value, bb.value, fd.value


def _jobs(jobs):
    arr = (pgz_job * len(jobs))()
    for k, (gz_ptr, gz_len, out_ptr, out_cap) in enumerate(jobs):
        arr[k].gz, arr[k].gz_len, arr[k].out, arr[k].out_cap = gz_ptr, gz_len, out_ptr, out_cap
    return arr


def pgz_decompress_batch(ctx: int, jobs, stats: bool = False):
    """jobs: list of (gz_ptr, gz_len, out_ptr, out_cap); returns (status, [(status, out_len)], stats)."""
    arr = _jobs(jobs)
    st = pgz_stats() if stats else None
    r = lib().pgz_decompress_batch(ctx, len(jobs), arr, ctypes.byref(st) if st is not None else None)
    return r, [(arr[k].status, arr[k].out_len) for k in range(len(jobs))], (st.as_dict() if st is not None else None)


def pgz_decompress_batch_host(ctx: int, jobs, stats: bool = False):
    """jobs: list of (gz_ptr, gz_len, out_ptr, out_cap) with HOST addresses; returns (status,
    [(status, out_len)], stats)."""
    arr = _jobs(jobs)
    st = pgz_stats() if stats else None
    r = lib().pgz_decompress_batch_host(ctx, len(jobs), arr, ctypes.byref(st) if st is not None else None)
    return r, [(arr[k].status, arr[k].out_len) for k in range(len(jobs))], (st.as_dict() if st is not None else None)


def pgz_wave_chunk_bytes(ctx: int, jobs, warps_per_block: int, waves: float):
    """(status, chunk_bytes, resident_warps): the part size giving about `waves` whole waves of the pass-1
    warps over the jobs' members (jobs: list of (gz_ptr, gz_len, out_ptr, out_cap))."""
    arr = _jobs(jobs)
    cb, rw = U64(0), ctypes.c_int(0)
    r = lib().pgz_wave_chunk_bytes(ctx, arr, len(jobs), warps_per_block, float(waves), ctypes.byref(cb),
                                   ctypes.byref(rw))
    return r, cb.value, rw.value


class Batch:
    """pgz_batch_prepare / pgz_batch_run / pgz_batch_free."""

    def __init__(self, ctx: int, jobs):
        self.arr = _jobs(jobs)
        h = VP()
        r = lib().pgz_batch_prepare(ctx, len(jobs), self.arr, ctypes.byref(h))
        if r:
            raise PgzError(r, "pgz_batch_prepare")
        self.h = h.value

    def run(self, stats: bool = False):
        st = pgz_stats() if stats else None
        r = lib().pgz_batch_run(self.h, self.arr, ctypes.byref(st) if st is not None else None)
        return r, [(self.arr[k].status, self.arr[k].out_len) for k in range(len(self.arr))], \
            (st.as_dict() if st is not None else None)

    def free(self):
        if self.h:
            lib().pgz_batch_free(self.h)
            self.h = None


def pgz_autotune(ctx: int, jobs, chunk_bytes, warps_per_block, reps: int = 3, sweep_exec: bool = False):
    """(status, [entry dicts], best dict); jobs: list of (gz_ptr, gz_len, out_ptr, out_cap) device addresses;
    sets the context's part size, CTA shape (and, with sweep_exec, the pass-1 execution form)."""
    arr = _jobs(jobs)
    cb = (U64 * len(chunk_bytes))(*chunk_bytes)
    wp = (ctypes.c_int * len(warps_per_block))(*warps_per_block)
    ent = (pgz_tune_entry * (len(chunk_bytes) * len(warps_per_block) * (2 if sweep_exec else 1)))()
    best = pgz_tune_entry()
    r = lib().pgz_autotune(ctx, arr, len(jobs), cb, len(chunk_bytes), wp, len(warps_per_block), 1 if sweep_exec else 0,
                           reps, ent, ctypes.byref(best))
    return r, [e.as_dict() for e in ent], best.as_dict()


class Server:
    """pgz_server_*: submitted requests are kept alive here until they are done."""

    def __init__(self, cfg: pgz_config, slots: int = 4, mem_budget: int = 0):
        h = VP()
        r = lib().pgz_server_create(ctypes.byref(h), ctypes.byref(cfg), slots, mem_budget)
        if r:
            raise PgzError(r, "pgz_server_create")
        self.h = h.value
        self.live = []

    def add_file(self, gz_ptr: int, gz_len: int) -> int:
        f = ctypes.c_int(-1)
        r = lib().pgz_server_add_file(self.h, gz_ptr, gz_len, ctypes.byref(f))
        if r:
            raise PgzError(r, "pgz_server_add_file")
        return f.value

    def submit(self, file: int, out_ptr: int, out_cap: int, offset: int = 0, length: int | None = None):
        """A whole member (length None) or the byte range [offset, offset + length); returns the request."""
        req = pgz_request(file=file, whole=1 if length is None else 0, offset=offset, length=length or 0,
                          out=out_ptr, out_cap=out_cap)
        r = lib().pgz_server_submit(self.h, ctypes.byref(req))
        if r:
            raise PgzError(r, "pgz_server_submit")
        self.live.append(req)
        return req

    def poll(self) -> int:
        n = ctypes.c_int(0)
        r = lib().pgz_server_poll(self.h, ctypes.byref(n))
        if r:
            raise PgzError(r, "pgz_server_poll")
        self.live = [q for q in self.live if q.status < 0]
        return n.value

    def drain(self):
        r = lib().pgz_server_drain(self.h)
        if r:
            raise PgzError(r, "pgz_server_drain")
        self.live = []

    def pending(self) -> int:
        return lib().pgz_server_pending(self.h)

    def close(self):
        if self.h:
            lib().pgz_server_destroy(self.h)
            self.h = None


def pgz_extract_sequences(ctx: int, sym_ptr: int, n: int, min_len: int, spans_ptr: int, max_spans: int):
    """(status, n_spans, n_undetermined); device addresses (spans: 2 * max_spans u64)."""
    a, b = U64(0), U64(0)
    r = lib().pgz_extract_sequences(ctx, sym_ptr, n, min_len, spans_ptr, max_spans, ctypes.byref(a), ctypes.byref(b))
    return r, a.value, b.value


def pgz_index_build(ctx: int, gz_ptr: int, gz_len: int) -> int:
    h = VP()
    r = lib().pgz_index_build(ctx, gz_ptr, gz_len, ctypes.byref(h))
    if r:
        raise PgzError(r, "pgz_index_build")
    return h.value


def pgz_index_info(idx: int):
    t, n = U64(0), U64(0)
    lib().pgz_index_info(idx, ctypes.byref(t), ctypes.byref(n))
    return t.value, n.value


def pgz_decompress_range(ctx: int, idx: int, d_off: int, length: int, out_ptr: int) -> int:
    return lib().pgz_decompress_range(ctx, idx, d_off, length, out_ptr)


def pgz_index_free(idx: int) -> None:
    lib().pgz_index_free(idx)


def pgz_inspect_parts(ctx: int):
    n = ctypes.c_int(0)
    lib().pgz_inspect_parts(ctx, 0, None, None, None, ctypes.byref(n))
    sb = np.zeros(n.value, dtype=np.uint64)
    ns = np.zeros(n.value, dtype=np.uint64)
    nph = np.zeros(n.value, dtype=np.uint64)
    r = lib().pgz_inspect_parts(ctx, n.value, sb.ctypes.data, ns.ctypes.data, nph.ctypes.data, ctypes.byref(n))
    if r:
        raise PgzError(r, "pgz_inspect_parts")
    return sb, ns, nph


def pgz_inspect_symbols(ctx: int, part: int) -> np.ndarray:
    n = U64(0)
    r = lib().pgz_inspect_symbols(ctx, part, None, 0, ctypes.byref(n))
    if r:
        raise PgzError(r, "pgz_inspect_symbols")
    out = np.zeros(n.value, dtype=np.uint16)
    if n.value:
        r = lib().pgz_inspect_symbols(ctx, part, out.ctypes.data, n.value, ctypes.byref(n))
        if r:
            raise PgzError(r, "pgz_inspect_symbols")
    return out


def pgz_inspect_window(ctx: int, part: int) -> np.ndarray:
    w = np.zeros(32768, dtype=np.uint8)
    r = lib().pgz_inspect_window(ctx, part, w.ctypes.data)
    if r:
        raise PgzError(r, "pgz_inspect_window")
    return w


def pgz_kernel_launches(ctx: int) -> int:
    return int(lib().pgz_kernel_launches(ctx))


_PART_FIELDS = [f for f, _ in pgz_part_state._fields_]


def pgz_recover_step(parts, s0_bit: int, mode: int = 0, last_seg: int = 1, confirm_blocks: int = 5):
    """parts: list of dicts with the pgz_part_state fields (missing ones 0; sync defaults to none).  Returns
    (action, parts after the step as dicts, false starts counted, part to grow or -1)."""
    arr = (pgz_part_state * len(parts))()
    for k, d in enumerate(parts):
        arr[k].sync = (1 << 64) - 1
        for f, v in d.items():
            if f not in _PART_FIELDS:
                raise KeyError(f)
            setattr(arr[k], f, v)
    fs = U64(0)
    g = ctypes.c_int(-1)
    a = lib().pgz_recover_step(len(parts), arr, s0_bit, mode, last_seg, confirm_blocks, ctypes.byref(fs),
                               ctypes.byref(g))
    return a, [{f: getattr(arr[k], f) for f in _PART_FIELDS} for k in range(len(parts))], fs.value, g.value


def pgz_decompress_noalloc(gz_ptr: int, gz_len: int, out_ptr: int, out_cap: int, stream: int | None = None):
    """(status, out_len): decompression with no device allocation (fixed scratch); device addresses."""
    n = U64(0)
    r = lib().pgz_decompress_noalloc(gz_ptr, gz_len, out_ptr, out_cap, ctypes.byref(n), stream)
    return r, n.value
