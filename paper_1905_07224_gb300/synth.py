"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no part of the decompression method: it only draws text with
numpy's PCG64 generator and compresses it with the host zlib library (called as
a compressor, RFC 1952 container, ``wbits=31``).  Both the CUDA path and the
CPU oracle consume what it returns; neither is imported here.

The text stands in for the FASTQ files the paper measures on (Section
"Experimental Results", ENA FASTQ files, and the FASTQ-like strings of Section
"Compression of FASTQ-like strings"), which are not available offline:

* ``fastq``  -- 4-line records ``@SIM.<i> length=<L>`` / L bases drawn
  uniformly from ACGT, replaced by 'N' with probability ``p_n`` / ``+`` /
  L Phred+33 quality characters ``clip(round(70 - 25*k/(L-1) + N(0,3)), 35, 73)``
  (values drift lower along the read).  Records are generated until the target
  size is reached and the text is cut to exactly ``n_bytes``.
* ``markov`` -- order-2 Markov ASCII text over bytes 32..126 and newline
  (96 symbols); each of the 96*96 contexts draws its next-symbol distribution
  from Dirichlet(0.1); initial context (0, 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import zlib

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
MARKOV_ALPHABET = np.array(list(range(32, 127)) + [10], dtype=np.uint8)  # 96 symbols


# ---------------------------------------------------------------------------
# FASTQ
# ---------------------------------------------------------------------------
def fastq(n_bytes: int, read_len: int = 100, p_n: float = 0.001, seed: int = 0) -> bytes:
    """Exactly ``n_bytes`` of synthetic FASTQ text (see module docstring)."""
    if n_bytes <= 0:
        return b""
    return _fastq_records(n_bytes, int(read_len), p_n, np.random.default_rng(seed), 0, 0)


def _fastq_records(n_bytes: int, L: int, p_n: float, rng, first: int, skip: int) -> bytes:
    """Records ``first``, ``first + 1``, ... drawn from ``rng``; the first ``skip`` bytes are dropped and
    exactly ``n_bytes`` are returned."""
    fixed = 2 * L + 4                      # seq + "\n+\n" + qual + "\n"
    min_rec = len(f"@SIM.{first} length={L}\n") + fixed
    n_rec = (n_bytes + skip) // min_rec + 2
    bases = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, size=(n_rec, L))]
    if p_n > 0:
        bases[rng.random((n_rec, L)) < p_n] = ord("N")
    drift = 70.0 - 25.0 * np.arange(L) / max(L - 1, 1)
    qual = np.clip(np.rint(drift[None, :] + rng.normal(0.0, 3.0, size=(n_rec, L))), 35, 73).astype(np.uint8)
    body = np.empty((n_rec, fixed), dtype=np.uint8)
    body[:, :L] = bases
    body[:, L:L + 3] = np.frombuffer(b"\n+\n", dtype=np.uint8)
    body[:, L + 3:2 * L + 3] = qual
    body[:, 2 * L + 3] = 10
    heads = [f"@SIM.{i} length={L}\n".encode() for i in range(first, first + n_rec)]
    hlen = np.fromiter((len(h) for h in heads), dtype=np.int64, count=n_rec)
    rec_len = hlen + fixed
    off = np.zeros(n_rec + 1, dtype=np.int64)
    np.cumsum(rec_len, out=off[1:])
    total = int(off[-1])
    out = np.empty(total, dtype=np.uint8)
    hbytes = np.frombuffer(b"".join(heads), dtype=np.uint8)
    hstart = np.zeros(n_rec, dtype=np.int64)
    np.cumsum(hlen[:-1], out=hstart[1:])
    out[np.repeat(off[:-1] - hstart, hlen) + np.arange(hbytes.size)] = hbytes
    out[(off[:-1] + hlen)[:, None] + np.arange(fixed)[None, :]] = body
    assert total >= n_bytes + skip
    return out[skip:skip + n_bytes].tobytes()


def _fastq_record_at(byte: int, L: int):
    """(record index, offset inside it) of byte ``byte`` of the record stream: a record's length depends only
    on the number of digits of its index."""
    fixed = 2 * L + 4
    tail = len(f" length={L}\n") + len("@SIM.") + fixed
    i, pos, d = 0, 0, 1
    while True:
        n = 9 * 10 ** (d - 1) if d > 1 else 10           # indices with d digits (0..9 for d = 1)
        size = n * (tail + d)
        if byte < pos + size:
            k = (byte - pos) // (tail + d)
            return i + k, (byte - pos) - k * (tail + d)
        i, pos, d = i + n, pos + size, d + 1


def _fastq_piece(args):
    n_bytes, L, p_n, seed, k, piece = args
    first, skip = _fastq_record_at(k * piece, L)
    return _fastq_records(n_bytes, L, p_n, np.random.default_rng([seed, k]), first, skip)


def fastq_large(n_bytes: int, read_len: int = 150, p_n: float = 0.01, seed: int = 2, piece: int = 256 << 20,
                processes: int | None = None) -> bytes:
    """Exactly ``n_bytes`` of FASTQ text for inputs too large for one draw: piece k covers bytes
    [k * piece, (k + 1) * piece) of the record stream (records numbered from 0, so the concatenation is one
    stream), with its own generator ``default_rng([seed, k])``; pieces are drawn in parallel."""
    import multiprocessing as mp
    L = int(read_len)
    jobs = [(min(piece, n_bytes - k * piece), L, p_n, seed, k, piece) for k in range((n_bytes + piece - 1) // piece)]
    if processes is None:
        processes = min(len(jobs), max(1, len(os.sched_getaffinity(0))))
    if processes <= 1 or len(jobs) <= 1:
        return b"".join(_fastq_piece(j) for j in jobs)
    with mp.get_context("spawn").Pool(processes) as pool:
        return b"".join(pool.map(_fastq_piece, jobs, chunksize=1))


# ---------------------------------------------------------------------------
# order-2 Markov text (sampled by a tiny C loop; the chain is sequential)
# ---------------------------------------------------------------------------
_MARKOV_SRC = os.path.join(_HERE, "synth_markov.c")
_MARKOV_SO = os.path.join(_HERE, "_synth_markov.so")
_markov_lib = None


def build_markov_sampler(force: bool = False) -> str:
    """Compile the Markov sampler (plain C, host only)."""
    if force or not os.path.exists(_MARKOV_SO) or os.path.getmtime(_MARKOV_SO) < os.path.getmtime(_MARKOV_SRC):
        tmp = _MARKOV_SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _MARKOV_SRC])
        os.replace(tmp, _MARKOV_SO)
    return _MARKOV_SO


def _markov():
    global _markov_lib
    if _markov_lib is None:
        lib = ctypes.CDLL(build_markov_sampler())
        lib.markov_sample.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p]
        lib.markov_sample.restype = None
        _markov_lib = lib
    return _markov_lib


def markov(n_bytes: int, seed: int = 0) -> bytes:
    """Exactly ``n_bytes`` of order-2 Markov ASCII text (see module docstring)."""
    if n_bytes <= 0:
        return b""
    rng = np.random.default_rng(seed)
    k = MARKOV_ALPHABET.size
    probs = rng.dirichlet(np.full(k, 0.1), size=k * k)            # (k*k, k)
    cdf = np.cumsum(probs, axis=1)
    cdf[:, -1] = 1.0
    cdf = np.ascontiguousarray(cdf, dtype=np.float64)
    u = rng.random(n_bytes)
    out = np.empty(n_bytes, dtype=np.uint8)
    _markov().markov_sample(cdf.ctypes.data, MARKOV_ALPHABET.ctypes.data, u.ctypes.data,
                            ctypes.c_int64(n_bytes), out.ctypes.data)
    return out.tobytes()


# ---------------------------------------------------------------------------
# compression (host zlib, called as a library) and the paper's workloads
# ---------------------------------------------------------------------------
def binary_records(n_bytes: int, seed: int = 0) -> bytes:
    """Structured binary data (bytes of every value): little-endian 14-byte records of a counter (u32, step
    3), six small integers (u8, 0..11) and a normal float32 rounded to 0.01; exactly n_bytes."""
    rng = np.random.default_rng(seed)
    n = n_bytes // 14 + 1
    rec = np.zeros(n, dtype=[("id", "<u4"), ("q", "u1", 6), ("x", "<f4")])
    rec["id"] = np.arange(n, dtype=np.uint32) * 3 + 1000
    rec["q"] = rng.integers(0, 12, size=(n, 6))
    rec["x"] = np.round(rng.normal(0, 1, n), 2).astype(np.float32)
    return rec.tobytes()[:n_bytes]


def gzip_compress(data: bytes, level: int = 6) -> bytes:
    """Single-member gzip (10-byte header) via host zlib at ``level``."""
    c = zlib.compressobj(level, zlib.DEFLATED, 31)
    return c.compress(data) + c.flush()


def _deflate_piece(args):
    data, dict_bytes, level, last = args
    c = zlib.compressobj(level, zlib.DEFLATED, -15, 8, zlib.Z_DEFAULT_STRATEGY, *([dict_bytes] if dict_bytes else []))
    return c.compress(data) + c.flush(zlib.Z_FINISH if last else zlib.Z_SYNC_FLUSH)


def bgzf_compress(data: bytes, level: int = 6, block: int = 65280, eof: bool = True) -> bytes:
    """BGZF (blocked gzip, SAM/BAM specification): ``data`` in members of at most ``block`` input bytes, each a
    gzip member whose header carries the extra subfield 'BC' (SLEN 2) holding the member's total size minus
    one; host zlib deflates each block (raw DEFLATE).  With ``eof`` the empty end-of-file member follows."""
    out = bytearray()
    members = [data[a:a + block] for a in range(0, len(data), block)] + ([b""] if eof else [])
    for chunk in members:
        c = zlib.compressobj(level, zlib.DEFLATED, -15)
        body = c.compress(chunk) + c.flush()
        size = 12 + 6 + len(body) + 8
        head = bytes([0x1F, 0x8B, 8, 4, 0, 0, 0, 0, 0, 255, 6, 0, ord("B"), ord("C"), 2, 0]) + \
            (size - 1).to_bytes(2, "little")
        out += head + body + (zlib.crc32(chunk) & 0xFFFFFFFF).to_bytes(4, "little") + \
            (len(chunk) & 0xFFFFFFFF).to_bytes(4, "little")
    return bytes(out)


def gzip_compress_parallel(data: bytes, level: int = 6, piece: int = 64 << 20, processes: int | None = None) -> bytes:
    """One gzip member (RFC 1952, 10-byte header) of ``data`` compressed by host zlib in parallel pieces, the
    way pigz does: piece k is deflated with the previous 32 KiB as its preset dictionary and ends with a sync
    flush (an empty stored block), so the pieces form one DEFLATE stream.  CRC-32 and ISIZE (length mod 2^32)
    come from ``zlib.crc32`` and ``len``."""
    import multiprocessing as mp
    n = len(data)
    mv = memoryview(data)
    jobs = []
    for a in range(0, max(n, 1), piece):
        b = min(n, a + piece)
        jobs.append((bytes(mv[a:b]), bytes(mv[max(0, a - 32768):a]) if a else b"", level, b >= n))
    if processes is None:
        processes = min(len(jobs), max(1, len(os.sched_getaffinity(0))))
    if processes <= 1 or len(jobs) <= 1:
        body = b"".join(_deflate_piece(j) for j in jobs)
    else:
        with mp.get_context("spawn").Pool(processes) as pool:
            body = b"".join(pool.map(_deflate_piece, jobs, chunksize=1))
    head = bytes([0x1F, 0x8B, 8, 0, 0, 0, 0, 0, 0, 255])
    tail = (zlib.crc32(data) & 0xFFFFFFFF).to_bytes(4, "little") + (n & 0xFFFFFFFF).to_bytes(4, "little")
    return head + body + tail


def log_uniform_sizes(n: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)).astype(np.int64)


def batch_manifest(n_files: int = 512, seed: int = 3, lo: int = 64 << 10, hi: int = 64 << 20):
    """(kind, n_bytes, level, seed) per file of the batched workload.

    Sizes are log-uniform in [lo, hi); even files are FASTQ (150 bp reads),
    odd files order-2 Markov text; levels drawn uniformly from {1, 6, 9}.
    """
    rng = np.random.default_rng(seed)
    sizes = log_uniform_sizes(n_files, lo, hi, rng)
    levels = rng.choice(np.array([1, 6, 9]), size=n_files)
    return [("fastq" if k % 2 == 0 else "markov", int(sizes[k]), int(levels[k]), seed * 100003 + k)
            for k in range(n_files)]


def make_file(kind: str, n_bytes: int, level: int, seed: int, read_len: int = 150, p_n: float = 0.001):
    """(raw, gz) for one manifest entry."""
    raw = fastq(n_bytes, read_len, p_n, seed) if kind == "fastq" else markov(n_bytes, seed)
    return raw, gzip_compress(raw, level)


def _make_file_star(args):
    return make_file(*args)


def make_files(entries, processes: int | None = None):
    """Generate and compress many files, in parallel (spawned processes)."""
    import multiprocessing as mp
    if processes is None:
        processes = min(len(entries), max(1, len(os.sched_getaffinity(0))))
    if processes <= 1 or len(entries) <= 1:
        return [make_file(*e) for e in entries]
    build_markov_sampler()
    ctx = mp.get_context("spawn")
    # largest first so the pool stays busy
    order = sorted(range(len(entries)), key=lambda k: -entries[k][1])
    with ctx.Pool(processes) as pool:
        res = pool.map(_make_file_star, [entries[k] for k in order], chunksize=1)
    out = [None] * len(entries)
    for k, r in zip(order, res):
        out[k] = r
    return out
