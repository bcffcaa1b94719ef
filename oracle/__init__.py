"""CPU oracle for the two-pass parallel gzip decompression (arXiv 1905.07224).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library under
``paper_1905_07224_gb300`` never does.  The C source ``oracle.c`` is a plain,
slow, bit-at-a-time decoder written from the RFC 1951/1952 format definitions
and the paper's algorithms; this module only marshals arguments.

Parity status: every exported function is pinned by ``tests/test_oracle*.py``
against host zlib, hand-built streams, closed forms or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

OK = 0
E_ARG, E_HEADER, E_DATA, E_TRUNC, E_CRC, E_ISIZE, E_CAPACITY, E_DIST = -1, -2, -3, -4, -5, -6, -7, -8
E_BYTE, E_SIZE, E_FINAL, E_TYPE, E_NOSYNC, E_NOMEM, E_UNSUPPORTED, E_CHAIN = -9, -10, -11, -12, -13, -14, -15, -16

NONE = (1 << 64) - 1
WSIZE = 32768
PH = 0x8000


def default_allowed() -> np.ndarray:
    """Reading of the paper's ASCII check: bytes 9, 10, 13 and 32..126."""
    m = np.zeros(32, dtype=np.uint8)
    for b in [9, 10, 13] + list(range(32, 127)):
        m[b >> 3] |= 1 << (b & 7)
    return m


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C compiler."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


_lib = None
P = ctypes.c_void_p
U64 = ctypes.c_uint64
U64P = ctypes.POINTER(ctypes.c_uint64)
I = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_crc32.argtypes = [ctypes.c_uint32, P, U64]
        L.orc_crc32.restype = ctypes.c_uint32
        L.orc_crc32_combine.argtypes = [ctypes.c_uint32, ctypes.c_uint32, U64]
        L.orc_crc32_combine.restype = ctypes.c_uint32
        L.orc_gzip_header.argtypes = [P, U64]
        L.orc_gzip_header.restype = ctypes.c_int64
        L.orc_gunzip.argtypes = [P, U64, P, U64, U64P, P, U64, U64P, ctypes.POINTER(I)]
        L.orc_gunzip.restype = I
        L.orc_inflate_from.argtypes = [P, U64, U64, U64, I, P, I, P, U64, U64P, U64P,
                                       ctypes.POINTER(I), U64P, U64P]
        L.orc_inflate_from.restype = I
        L.orc_block_ok.argtypes = [P, U64, U64, P, U64, U64, ctypes.POINTER(I)]
        L.orc_block_ok.restype = I
        L.orc_confirm.argtypes = [P, U64, U64, P, I]
        L.orc_confirm.restype = I
        L.orc_sync_scan.argtypes = [P, U64, U64, U64, P, U64, U64, I]
        L.orc_sync_scan.restype = ctypes.c_int64
        L.orc_translate.argtypes = [P, U64, P, P]
        L.orc_translate.restype = None
        L.orc_next_window.argtypes = [P, P, U64, P]
        L.orc_next_window.restype = None
        L.orc_two_pass.argtypes = [P, U64, I, P, U64, U64, I, P, U64, U64P, P, P, P, ctypes.POINTER(I)]
        L.orc_two_pass.restype = I
        L.orc_decompress_at.argtypes = [P, U64, U64, P, U64, U64, I, ctypes.c_uint8, P, P, U64,
                                        U64P, U64P, U64P]
        L.orc_decompress_at.restype = I
        _lib = L
    return _lib


def _buf(data) -> np.ndarray:
    if isinstance(data, np.ndarray):
        return np.ascontiguousarray(data, dtype=np.uint8)
    return np.frombuffer(bytes(data), dtype=np.uint8)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------
def crc32(data, crc: int = 0) -> int:
    a = _buf(data)
    return int(lib().orc_crc32(crc, _ptr(a), a.size))


def crc32_combine(crc_a: int, crc_b: int, len_b: int) -> int:
    return int(lib().orc_crc32_combine(crc_a, crc_b, len_b))


def gzip_header(gz) -> int:
    """Offset of the DEFLATE data, or a negative error."""
    a = _buf(gz)
    return int(lib().orc_gzip_header(_ptr(a), a.size))


def gunzip(gz, cap: int | None = None, max_blocks: int = 0):
    """(status, output bytes, block start bits, members)."""
    a = _buf(gz)
    if cap is None:
        cap = max(1 << 16, 1100 * a.size)
    out = np.empty(max(cap, 1), dtype=np.uint8)
    blocks = np.zeros(max(max_blocks, 1), dtype=np.uint64)
    n = U64(0)
    nb = U64(0)
    members = I(0)
    e = lib().orc_gunzip(_ptr(a), a.size, _ptr(out), cap, ctypes.byref(n), _ptr(blocks) if max_blocks else None,
                         max_blocks, ctypes.byref(nb), ctypes.byref(members))
    return e, out[:n.value].tobytes(), blocks[:min(nb.value, max_blocks)].copy(), members.value


def inflate_from(data, end_bit: int, start_bit: int, stop_bit: int = 0, known: bool = False,
                 allowed: np.ndarray | None = None, check_blocks: int = 0, cap: int | None = None,
                 count_only: bool = False):
    """Decode whole blocks from ``start_bit``; returns a dict of the results."""
    a = _buf(data)
    if cap is None:
        cap = max(1 << 16, 1100 * ((end_bit - start_bit) // 8 + 1))
    out = None if count_only else np.empty(max(cap, 1), dtype=np.uint16)
    n, pos, nb, nph = U64(0), U64(0), U64(0), U64(0)
    final = I(0)
    e = lib().orc_inflate_from(_ptr(a), end_bit, start_bit, stop_bit, int(known), _ptr(allowed), check_blocks,
                               _ptr(out), 0 if count_only else cap, ctypes.byref(n), ctypes.byref(pos),
                               ctypes.byref(final), ctypes.byref(nb), ctypes.byref(nph))
    return dict(status=e, sym=None if out is None else out[:n.value].copy(), n=n.value, pos=pos.value,
                final=bool(final.value), nblocks=nb.value, nph=nph.value)


def block_ok(data, end_bit: int, bit: int, allowed: np.ndarray | None = None,
             min_out: int = 1024, max_out: int = 4 << 20):
    """(holds, reason) of the block-start predicate at ``bit``."""
    a = _buf(data)
    why = I(0)
    ok = lib().orc_block_ok(_ptr(a), end_bit, bit, _ptr(allowed), min_out, max_out, ctypes.byref(why))
    return bool(ok), why.value


def confirm(data, end_bit: int, bit: int, allowed: np.ndarray | None = None, blocks: int = 5) -> bool:
    a = _buf(data)
    return bool(lib().orc_confirm(_ptr(a), end_bit, bit, _ptr(allowed), blocks))


def sync_scan(data, end_bit: int, lo: int, hi: int, allowed: np.ndarray | None = None,
              min_out: int = 1024, max_out: int = 4 << 20, confirm_blocks: int = 0) -> int:
    """Least bit of [lo, hi) passing the predicate (and confirmation); -1 if none."""
    a = _buf(data)
    return int(lib().orc_sync_scan(_ptr(a), end_bit, lo, hi, _ptr(allowed), min_out, max_out, confirm_blocks))


def translate(sym: np.ndarray, window: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(sym, dtype=np.uint16)
    w = np.ascontiguousarray(window, dtype=np.uint8)
    assert w.size == WSIZE
    out = np.empty(s.size, dtype=np.uint8)
    lib().orc_translate(_ptr(s), s.size, _ptr(w), _ptr(out))
    return out


def next_window(window: np.ndarray, sym: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(sym, dtype=np.uint16)
    w = np.ascontiguousarray(window, dtype=np.uint8)
    out = np.empty(WSIZE, dtype=np.uint8)
    lib().orc_next_window(_ptr(w), _ptr(s), s.size, _ptr(out))
    return out


def two_pass(gz, nparts: int, allowed: np.ndarray | None = None, min_out: int = 1024,
             max_out: int = 4 << 20, confirm_blocks: int = 5, cap: int | None = None):
    """The two-pass algorithm restated on one thread; returns a dict."""
    a = _buf(gz)
    if allowed is None:
        allowed = default_allowed()
    if cap is None:
        cap = max(1 << 16, 1100 * a.size)
    out = np.empty(cap, dtype=np.uint8)
    bits = np.zeros(nparts, dtype=np.uint64)
    plen = np.zeros(nparts, dtype=np.uint64)
    pnph = np.zeros(nparts, dtype=np.uint64)
    n = U64(0)
    nfalse = I(0)
    e = lib().orc_two_pass(_ptr(a), a.size, nparts, _ptr(allowed), min_out, max_out, confirm_blocks,
                           _ptr(out), cap, ctypes.byref(n), _ptr(bits), _ptr(plen), _ptr(pnph),
                           ctypes.byref(nfalse))
    return dict(status=e, out=out[:n.value].tobytes(), part_bits=bits, part_len=plen, part_nph=pnph,
                false_syncs=nfalse.value)


def decompress_at(gz, start_bit: int, fill: int = ord("?"), allowed: np.ndarray | None = None,
                  min_out: int = 1024, max_out: int = 4 << 20, confirm_blocks: int = 5,
                  cap: int | None = None):
    a = _buf(gz)
    if allowed is None:
        allowed = default_allowed()
    if cap is None:
        cap = max(1 << 16, 1100 * a.size)
    sym = np.empty(cap, dtype=np.uint16)
    byts = np.empty(cap, dtype=np.uint8)
    n, bb, fd = U64(0), U64(0), U64(0)
    e = lib().orc_decompress_at(_ptr(a), a.size, start_bit, _ptr(allowed), min_out, max_out, confirm_blocks,
                                fill, _ptr(sym), _ptr(byts), cap, ctypes.byref(n), ctypes.byref(bb),
                                ctypes.byref(fd))
    return dict(status=e, sym=sym[:n.value].copy(), bytes=byts[:n.value].tobytes(), block_bit=bb.value,
                first_determined=fd.value)


# Appendix "Heuristic extraction of DNA sequences in DEFLATE block": T D+ (U+ D+)* T with T a newline or an
# undetermined character, D a nucleotide, U an undetermined character; byte 0 stands for U in the mapped text
# (real byte 0 becomes byte 1, which is neither).
_SEQ_RE = None


def sequences(sym, min_len: int = 0):
    """The maximal non-overlapping substrings of decoded u16 symbols (bit 15 set: undetermined) that match
    T D+ (U+ D+)* T, without their delimiting T's, that are at least ``min_len`` long, leftmost first.
    A match needs its delimiters inside the array.  Returns [(start, length, contains_undetermined)]."""
    import re
    global _SEQ_RE
    if _SEQ_RE is None:
        _SEQ_RE = re.compile(rb"(?<=[\n\x00])[ACGTN]+(?:\x00+[ACGTN]+)*(?=[\n\x00])")
    s = np.asarray(sym, dtype=np.uint16)
    low = (s & 0xFF).astype(np.uint8)
    txt = np.where((s & 0x8000) != 0, 0, np.where(low == 0, 1, low)).astype(np.uint8).tobytes()
    out = []
    for m in _SEQ_RE.finditer(txt):
        if m.end() - m.start() >= min_len:
            out.append((m.start(), m.end() - m.start(), b"\x00" in m.group()))
    return out
