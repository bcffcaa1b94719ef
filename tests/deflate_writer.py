"""A tiny DEFLATE/gzip *encoder* used to hand-build test streams.

It writes RFC 1951 blocks from an explicit token list, so the expected output
of every stream it makes is known by construction.  It is independent of both
the oracle (a decoder) and the CUDA path.  Format facts used (RFC 1951):
data elements are packed LSB first (3.1.1); Huffman codes are packed MSB first
and are canonical (3.2.2); length codes 257..285 and distance codes 0..29 with
their extra bits (3.2.5); the fixed code (3.2.6); the dynamic header with the
code-length alphabet in the permuted order 16,17,18,0,8,7,9,6,10,5,11,4,12,3,
13,2,14,1,15 and the repeat codes 16/17/18 (3.2.7).
"""
from __future__ import annotations

import heapq
import struct
import zlib

CL_ORDER = [16, 17, 18, 0, 8, 7, 9, 6, 10, 5, 11, 4, 12, 3, 13, 2, 14, 1, 15]

# (code, base, extra bits) rows of RFC 1951 3.2.5, written out
LEN_ROWS = [(257, 3, 0), (258, 4, 0), (259, 5, 0), (260, 6, 0), (261, 7, 0), (262, 8, 0), (263, 9, 0),
            (264, 10, 0), (265, 11, 1), (266, 13, 1), (267, 15, 1), (268, 17, 1), (269, 19, 2), (270, 23, 2),
            (271, 27, 2), (272, 31, 2), (273, 35, 3), (274, 43, 3), (275, 51, 3), (276, 59, 3), (277, 67, 4),
            (278, 83, 4), (279, 99, 4), (280, 115, 4), (281, 131, 5), (282, 163, 5), (283, 195, 5),
            (284, 227, 5), (285, 258, 0)]
DIST_ROWS = [(0, 1, 0), (1, 2, 0), (2, 3, 0), (3, 4, 0), (4, 5, 1), (5, 7, 1), (6, 9, 2), (7, 13, 2),
             (8, 17, 3), (9, 25, 3), (10, 33, 4), (11, 49, 4), (12, 65, 5), (13, 97, 5), (14, 129, 6),
             (15, 193, 6), (16, 257, 7), (17, 385, 7), (18, 513, 8), (19, 769, 8), (20, 1025, 9),
             (21, 1537, 9), (22, 2049, 10), (23, 3073, 10), (24, 4097, 11), (25, 6145, 11), (26, 8193, 12),
             (27, 12289, 12), (28, 16385, 13), (29, 24577, 13)]


def len_code(n: int):
    assert 3 <= n <= 258
    if n == 258:
        return 285, 0, 0
    for code, base, extra in reversed(LEN_ROWS[:-1]):
        if n >= base:
            return code, n - base, extra
    raise AssertionError


def dist_code(d: int):
    assert 1 <= d <= 32768
    for code, base, extra in reversed(DIST_ROWS):
        if d >= base:
            return code, d - base, extra
    raise AssertionError


class BitWriter:
    def __init__(self):
        self.bits: list[int] = []

    def put(self, value: int, n: int):          # LSB first
        for i in range(n):
            self.bits.append((value >> i) & 1)

    def put_code(self, code: int, length: int):  # MSB first
        for i in range(length - 1, -1, -1):
            self.bits.append((code >> i) & 1)

    def align(self):
        while len(self.bits) % 8:
            self.bits.append(0)

    @property
    def nbits(self) -> int:
        return len(self.bits)

    def tobytes(self) -> bytes:
        b = self.bits + [0] * (-len(self.bits) % 8)
        return bytes(sum(b[i + k] << k for k in range(8)) for i in range(0, len(b), 8))


def canonical(lengths):
    """code per symbol for the given lengths (RFC 1951 3.2.2)."""
    maxl = max(lengths) if lengths else 0
    count = [0] * (max(maxl, 1) + 1)
    for l in lengths:
        if l:
            count[l] += 1
    nxt = [0] * (len(count) + 1)
    code = 0
    for bits in range(1, len(count)):
        code = (code + count[bits - 1]) << 1
        nxt[bits] = code
    codes = [None] * len(lengths)
    for s, l in enumerate(lengths):
        if l:
            codes[s] = nxt[l]
            nxt[l] += 1
    return codes


def huffman_lengths(freqs, n: int, maxlen: int = 15):
    """Complete Huffman code lengths for symbols with nonzero frequency."""
    used = [s for s in range(n) if freqs.get(s, 0) > 0]
    lengths = [0] * n
    if not used:
        return lengths
    if len(used) == 1:                      # make it complete with a dummy second symbol
        other = 0 if used[0] != 0 else 1
        lengths[used[0]] = 1
        lengths[other] = 1
        return lengths
    f = {s: freqs[s] for s in used}
    while True:                             # flatten frequencies until the limit holds
        lengths = [0] * n
        heap = [(f[s], i, [s]) for i, s in enumerate(used)]
        heapq.heapify(heap)
        k = len(heap)
        while len(heap) > 1:
            f1, _, a = heapq.heappop(heap)
            f2, _, b = heapq.heappop(heap)
            for s in a + b:
                lengths[s] += 1
            heapq.heappush(heap, (f1 + f2, k, a + b))
            k += 1
        if max(lengths) <= maxlen:
            return lengths
        f = {s: max(1, v >> 1) for s, v in f.items()}


def _rle_lengths(lengths):
    """(symbol, extra value, extra bits) list for the code-length sequence."""
    out = []
    i = 0
    while i < len(lengths):
        v = lengths[i]
        run = 1
        while i + run < len(lengths) and lengths[i + run] == v:
            run += 1
        if v == 0 and run >= 11:
            r = min(run, 138)
            out.append((18, r - 11, 7))
            i += r
        elif v == 0 and run >= 3:
            r = min(run, 10)
            out.append((17, r - 3, 3))
            i += r
        elif v != 0 and run >= 4:
            out.append((v, 0, 0))
            r = min(run - 1, 6)
            out.append((16, r - 3, 2))
            i += 1 + r
        else:
            out.append((v, 0, 0))
            i += 1
    return out


def write_stored(w: BitWriter, data: bytes, final: bool):
    w.put(1 if final else 0, 1)
    w.put(0, 2)
    w.align()
    w.put(len(data), 16)
    w.put(len(data) ^ 0xFFFF, 16)
    for b in data:
        w.put(b, 8)


def fixed_lit_lengths():
    return [8] * 144 + [9] * 112 + [7] * 24 + [8] * 8


def _emit_tokens(w: BitWriter, tokens, lcodes, llen, dcodes, dlen, eob: bool = True):
    for t in tokens:
        if t[0] == "lit":
            w.put_code(lcodes[t[1]], llen[t[1]])
        else:
            _, n, d = t
            c, ev, eb = len_code(n)
            w.put_code(lcodes[c], llen[c])
            w.put(ev, eb)
            c, ev, eb = dist_code(d)
            w.put_code(dcodes[c], dlen[c])
            w.put(ev, eb)
    if eob:
        w.put_code(lcodes[256], llen[256])


def write_fixed(w: BitWriter, tokens, final: bool):
    w.put(1 if final else 0, 1)
    w.put(1, 2)
    llen = fixed_lit_lengths()
    dlen = [5] * 32
    _emit_tokens(w, tokens, canonical(llen), llen, canonical(dlen), dlen)


def write_dynamic(w: BitWriter, tokens, final: bool, llen=None, dlen=None, use_rle: bool = True,
                  eob: bool = True):
    """A dynamic-Huffman block; code lengths default to Huffman codes of the tokens.  eob=False leaves out
    the end-of-block code, so a decoder reads on into whatever bits follow."""
    lf: dict[int, int] = {256: 1}
    df: dict[int, int] = {}
    for t in tokens:
        if t[0] == "lit":
            lf[t[1]] = lf.get(t[1], 0) + 1
        else:
            lf[len_code(t[1])[0]] = lf.get(len_code(t[1])[0], 0) + 1
            df[dist_code(t[2])[0]] = df.get(dist_code(t[2])[0], 0) + 1
    if llen is None:
        llen = huffman_lengths(lf, 286)
    if dlen is None:
        dlen = huffman_lengths(df, 30) if df else [1] + [0] * 29
    hlit = max(257, max(i for i, l in enumerate(llen) if l) + 1)
    hdist = max(1, max((i for i, l in enumerate(dlen) if l), default=0) + 1)
    seq = list(llen[:hlit]) + list(dlen[:hdist])
    cl_syms = _rle_lengths(seq) if use_rle else [(v, 0, 0) for v in seq]
    cf: dict[int, int] = {}
    for s, _, _ in cl_syms:
        cf[s] = cf.get(s, 0) + 1
    cl_len = huffman_lengths(cf, 19, maxlen=7)
    hclen = max(4, max(k for k, s in enumerate(CL_ORDER) if cl_len[s]) + 1)
    w.put(1 if final else 0, 1)
    w.put(2, 2)
    w.put(hlit - 257, 5)
    w.put(hdist - 1, 5)
    w.put(hclen - 4, 4)
    for k in range(hclen):
        w.put(cl_len[CL_ORDER[k]], 3)
    clc = canonical(cl_len)
    for s, ev, eb in cl_syms:
        w.put_code(clc[s], cl_len[s])
        w.put(ev, eb)
    _emit_tokens(w, tokens, canonical(llen), llen, canonical(dlen), dlen, eob)


def expand(tokens, prefix: bytes = b"") -> bytes:
    """The text a token list stands for (plain LZ77 copy semantics)."""
    out = bytearray(prefix)
    for t in tokens:
        if t[0] == "lit":
            out.append(t[1])
        else:
            _, n, d = t
            for _ in range(n):
                out.append(out[-d])
    return bytes(out[len(prefix):])


def gzip_wrap(deflate: bytes, data: bytes, flags: int = 0, name: bytes = b"", extra: bytes = b"",
              comment: bytes = b"", crc=None, isize=None) -> bytes:
    """RFC 1952 member around raw DEFLATE bytes."""
    hdr = bytearray(b"\x1f\x8b\x08" + bytes([flags]) + b"\x00\x00\x00\x00\x00\xff")
    if flags & 4:
        hdr += struct.pack("<H", len(extra)) + extra
    if flags & 8:
        hdr += name + b"\x00"
    if flags & 16:
        hdr += comment + b"\x00"
    if flags & 2:
        hdr += struct.pack("<H", zlib.crc32(bytes(hdr)) & 0xFFFF)
    c = zlib.crc32(data) if crc is None else crc
    n = len(data) & 0xFFFFFFFF if isize is None else isize
    return bytes(hdr) + deflate + struct.pack("<II", c, n)


def tokens_from_text(data: bytes, min_len: int = 3, window: int = 32768, max_chain: int = 16):
    """A simple greedy LZ77 tokenizer (hash of 3 bytes), for varied test blocks."""
    toks = []
    head: dict[bytes, list[int]] = {}
    i = 0
    while i < len(data):
        best_len, best_d = 0, 0
        key = data[i:i + 3]
        if len(key) == 3:
            for p in reversed(head.get(key, [])[-max_chain:]):
                d = i - p
                if d > window:
                    continue
                n = 0
                while n < 258 and i + n < len(data) and data[p + n] == data[i + n]:
                    n += 1
                if n > best_len:
                    best_len, best_d = n, d
        if best_len >= min_len:
            toks.append(("match", best_len, best_d))
            for k in range(best_len):
                if i + k + 3 <= len(data):
                    head.setdefault(data[i + k:i + k + 3], []).append(i + k)
            i += best_len
        else:
            toks.append(("lit", data[i]))
            if len(key) == 3:
                head.setdefault(key, []).append(i)
            i += 1
    return toks
