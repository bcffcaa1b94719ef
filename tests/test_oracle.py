"""Pins of the CPU oracle against things other than itself.

* CRC-32: the published check value, the empty string, host zlib.crc32, and
  the concatenation property against zlib.crc32 of the joined buffers.
* gunzip: host zlib (a library call) on seeded FASTQ/Markov text at levels
  1/6/9 plus edge inputs (empty, 1 byte, runs, 64 KiB + 1, binary data in
  stored blocks, fixed-Huffman and RLE strategies).
* hand-built streams (tests/deflate_writer.py, an independent encoder): the
  expected bytes are known by construction; also fed to zlib's raw inflater.
* corrupted streams: each defect yields its error code.
* block starts recorded by the oracle: re-decoded by zlib from that bit with
  the true preceding 32 KiB as dictionary must give the true suffix.
* symbolic decoding: substituting the true window into the symbols gives the
  true text (Section "Full file decompression in two passes"), and U_j stands
  for the byte 32768 - j positions before the part.
"""
import os
import struct
import zlib

import numpy as np
import pytest

import oracle
import deflate_writer as dw
from paper_1905_07224_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALLOWED = oracle.default_allowed()


# ---------------------------------------------------------------- CRC-32
def test_crc32_golden_check_values():
    for line in open(os.path.join(GOLDEN, "crc32_check.txt")):
        if line.startswith("#") or not line.strip():
            continue
        text, val = line.split()
        data = b"" if text == "@empty" else text.encode()
        assert oracle.crc32(data) == int(val, 16)


def test_crc32_matches_zlib_and_combine():
    rng = np.random.default_rng(5)
    for n in [0, 1, 2, 3, 7, 8, 100, 4097, 65536 + 3]:
        a = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert oracle.crc32(a) == zlib.crc32(a)
        assert oracle.crc32(a[n // 2:], oracle.crc32(a[:n // 2])) == zlib.crc32(a)
    for na, nb in [(0, 0), (0, 5), (5, 0), (1, 1), (13, 1000), (4096, 12345), (70000, 3)]:
        a = rng.integers(0, 256, na, dtype=np.uint8).tobytes()
        b = rng.integers(0, 256, nb, dtype=np.uint8).tobytes()
        assert oracle.crc32_combine(zlib.crc32(a), zlib.crc32(b), nb) == zlib.crc32(a + b)


# ---------------------------------------------------------------- gunzip vs zlib
def _inputs():
    yield "empty", b""
    yield "one", b"A"
    yield "run", b"a" * 100000
    yield "64k+1", synth.fastq(65537, 100, 0.001, 11)
    yield "fastq", synth.fastq(300000, 150, 0.01, 12)
    yield "markov", synth.markov(300000, 13)
    yield "binary", np.random.default_rng(14).integers(0, 256, 100000, dtype=np.uint8).tobytes()


@pytest.mark.parametrize("level", [0, 1, 6, 9])
def test_gunzip_roundtrip_levels(level):
    for name, data in _inputs():
        gz = synth.gzip_compress(data, level)
        e, out, _, members = oracle.gunzip(gz)
        assert e == 0, name
        assert out == data, name
        assert members == 1


@pytest.mark.parametrize("strategy", [zlib.Z_FIXED, zlib.Z_HUFFMAN_ONLY, zlib.Z_RLE, zlib.Z_FILTERED])
def test_gunzip_strategies(strategy):
    data = synth.fastq(200000, 100, 0.001, 21) + b"xxxxxxxxxxxxxxxxxxxxxxxxxxxxxxxxxxxx" * 50
    c = zlib.compressobj(6, zlib.DEFLATED, 31, 8, strategy)
    gz = c.compress(data) + c.flush()
    e, out, _, _ = oracle.gunzip(gz)
    assert e == 0 and out == data


def test_gunzip_multi_member_and_header_flags():
    a, b = b"first member\n" * 100, synth.fastq(5000, 100, 0.0, 3)
    gz = synth.gzip_compress(a, 6) + synth.gzip_compress(b, 1)
    e, out, _, members = oracle.gunzip(gz)
    assert (e, out, members) == (0, a + b, 2)
    raw = zlib.compressobj(6, zlib.DEFLATED, -15)
    deflate = raw.compress(a) + raw.flush()
    for flags in [2, 4, 8, 16, 2 | 4 | 8 | 16]:
        g = dw.gzip_wrap(deflate, a, flags=flags, name=b"f.txt", extra=b"\x01\x02\x03", comment=b"hello")
        assert zlib.decompress(g, 31) == a
        e, out, _, _ = oracle.gunzip(g)
        assert e == 0 and out == a
        assert oracle.gzip_header(g) == len(g) - len(deflate) - 8


# ---------------------------------------------------------------- hand-built streams
def _build(blocks):
    """blocks: list of (kind, payload); returns (raw deflate bytes, expected text)."""
    w = dw.BitWriter()
    text = b""
    for k, (kind, payload) in enumerate(blocks):
        final = k == len(blocks) - 1
        if kind == "stored":
            dw.write_stored(w, payload, final)
            text += payload
        else:
            seg = dw.expand(payload, text)
            (dw.write_fixed if kind == "fixed" else dw.write_dynamic)(w, payload, final)
            text += seg
    return w.tobytes(), text


def _hand_cases():
    lits = [("lit", c) for c in b"abcabcabc"]
    over = [("lit", ord("x")), ("match", 258, 1), ("match", 3, 1)]                    # distance-1 overlap
    big = synth.fastq(40000, 100, 0.0, 7)
    far = [("lit", b) for b in big[:32768]] + [("match", 258, 32768), ("match", 10, 32768)]   # max distance
    mixed = dw.tokens_from_text(synth.markov(20000, 9))
    return {
        "stored": [("stored", b"hello, stored block\n")],
        "stored_empty": [("stored", b"")],
        "fixed": [("fixed", lits + [("match", 6, 3)])],
        "fixed_overlap_258": [("fixed", over)],
        "dynamic": [("dynamic", dw.tokens_from_text(big))],
        "dynamic_maxdist": [("dynamic", far)],
        "multi": [("stored", b"head\n"), ("fixed", lits), ("dynamic", mixed), ("stored", b"tail\n")],
        "dynamic_single_dist_code": [("dynamic", [("lit", 65)] * 10 + [("match", 5, 1)])],
        "dynamic_no_matches": [("dynamic", [("lit", c) for c in b"only literals here"])],
    }


@pytest.mark.parametrize("name", sorted(_hand_cases()))
def test_hand_built_streams(name):
    deflate, text = _build(_hand_cases()[name])
    assert zlib.decompressobj(-15).decompress(deflate) == text        # the writer itself, pinned by zlib
    gz = dw.gzip_wrap(deflate, text)
    e, out, _, _ = oracle.gunzip(gz)
    assert e == 0 and out == text


def test_dynamic_header_without_rle_codes():
    toks = dw.tokens_from_text(b"the quick brown fox jumps over the lazy dog\n" * 40)
    w = dw.BitWriter()
    dw.write_dynamic(w, toks, True, use_rle=False)
    text = dw.expand(toks)
    gz = dw.gzip_wrap(w.tobytes(), text)
    assert zlib.decompress(gz, 31) == text
    e, out, _, _ = oracle.gunzip(gz)
    assert e == 0 and out == text


# ---------------------------------------------------------------- corrupted streams
def _good():
    deflate, text = _build([("stored", b"abc"), ("fixed", [("lit", 100), ("match", 4, 1)])])
    return deflate, text


def test_errors():
    deflate, text = _good()
    gz = dw.gzip_wrap(deflate, text)
    assert oracle.gunzip(gz)[0] == 0
    assert oracle.gunzip(dw.gzip_wrap(deflate, text, crc=zlib.crc32(text) ^ 1))[0] == oracle.E_CRC
    assert oracle.gunzip(dw.gzip_wrap(deflate, text, isize=len(text) + 1))[0] == oracle.E_ISIZE
    assert oracle.gunzip(b"\x1f\x8c" + gz[2:])[0] == oracle.E_HEADER
    assert oracle.gunzip(gz[:12])[0] == oracle.E_HEADER
    # bad NLEN
    w = dw.BitWriter()
    w.put(1, 1); w.put(0, 2); w.align(); w.put(3, 16); w.put(3, 16)
    for b in b"abc":
        w.put(b, 8)
    assert oracle.gunzip(dw.gzip_wrap(w.tobytes(), b"abc"))[0] == oracle.E_DATA
    # BTYPE 11
    w = dw.BitWriter(); w.put(1, 1); w.put(3, 2); w.put(0, 16)
    assert oracle.gunzip(dw.gzip_wrap(w.tobytes(), b""))[0] == oracle.E_DATA
    # distance beyond the output (empty context)
    w = dw.BitWriter(); dw.write_fixed(w, [("lit", 65), ("match", 3, 2)], True)
    assert oracle.gunzip(dw.gzip_wrap(w.tobytes(), b"AAAA"))[0] == oracle.E_DIST
    # literal/length code 286 in a fixed block (code 11000110 + ...)
    w = dw.BitWriter(); w.put(1, 1); w.put(1, 2)
    codes = dw.canonical(dw.fixed_lit_lengths())
    w.put_code(codes[286], 8); w.put(0, 16)
    assert oracle.gunzip(dw.gzip_wrap(w.tobytes(), b""))[0] == oracle.E_DATA
    # distance code 30 in a fixed block
    w = dw.BitWriter(); w.put(1, 1); w.put(1, 2)
    w.put_code(codes[65], 8); w.put_code(codes[257], 7); w.put_code(30, 5); w.put(0, 16)
    assert oracle.gunzip(dw.gzip_wrap(w.tobytes(), b""))[0] == oracle.E_DATA
    # over-subscribed literal/length code: three codes of length 1
    w = dw.BitWriter(); w.put(1, 1); w.put(2, 2); w.put(0, 5); w.put(0, 5); w.put(15, 4)
    cl = [0] * 19
    cl[1] = 1; cl[0] = 1                      # code-length code: symbols 0 and 1, length 1 each
    for k in range(19):
        w.put(cl[dw.CL_ORDER[k]], 3)
    clc = dw.canonical(cl)
    for s in [1, 1, 1] + [0] * 255:           # lengths 1,1,1 then zeros: over-subscribed
        w.put_code(clc[s], 1)
    w.put(0, 64)
    assert oracle.gunzip(dw.gzip_wrap(w.tobytes(), b""))[0] == oracle.E_DATA
    # truncated input
    big = synth.gzip_compress(synth.fastq(50000, 100, 0.0, 1), 6)
    assert oracle.gunzip(big[:len(big) // 2] + big[-8:])[0] in (oracle.E_TRUNC, oracle.E_DATA)
    # more data after the final block of a member is a second member: garbage there is a header error
    assert oracle.gunzip(gz + b"\x00\x01\x02")[0] == oracle.E_UNSUPPORTED


# ---------------------------------------------------------------- block starts and symbolic decode
def _shift_bits(buf: bytes, bit: int) -> bytes:
    a = np.frombuffer(buf, dtype=np.uint8)
    bits = np.unpackbits(a, bitorder="little")[bit:]
    return np.packbits(bits, bitorder="little").tobytes()


@pytest.fixture(scope="module")
def fastq_stream():
    data = synth.fastq(600000, 150, 0.001, 31)
    gz = synth.gzip_compress(data, 6)
    e, out, blocks, _ = oracle.gunzip(gz, max_blocks=10000)
    assert e == 0 and out == data
    return data, gz, [int(b) for b in blocks]


def _block_offsets(gz, blocks, total):
    end = (len(gz) - 8) * 8
    offs = []
    for b in blocks:
        r = oracle.inflate_from(gz, end, b, known=False, count_only=True)
        assert r["status"] == 0
        offs.append(total - r["n"])
    return offs


def test_recorded_block_starts_pinned_by_zlib(fastq_stream):
    data, gz, blocks = fastq_stream
    offs = _block_offsets(gz, blocks, len(data))
    assert offs[0] == 0 and offs == sorted(offs)
    for b, o in list(zip(blocks, offs))[1:]:
        d = zlib.decompressobj(-15, zdict=data[max(0, o - 32768):o])
        tail = d.decompress(_shift_bits(gz[:len(gz) - 8], b))
        assert tail == data[o:]


def test_symbolic_decode_identity(fastq_stream):
    data, gz, blocks = fastq_stream
    end = (len(gz) - 8) * 8
    offs = _block_offsets(gz, blocks, len(data))
    for b, o in list(zip(blocks, offs))[1:4]:
        r = oracle.inflate_from(gz, end, b, known=False)
        assert r["status"] == 0 and r["final"]
        sym = r["sym"]
        assert sym.size == len(data) - o
        ph = (sym & 0x8000) != 0
        assert r["nph"] == int(ph.sum())
        truth = np.frombuffer(data[o:], dtype=np.uint8)
        assert np.array_equal(sym[~ph].astype(np.uint8), truth[~ph])
        j = (sym[ph] & 0x7FFF).astype(np.int64)
        src = o - 32768 + j                       # U_j is the byte 32768 - j before the part
        assert np.all(src >= 0)
        assert np.array_equal(np.frombuffer(data, dtype=np.uint8)[src], truth[ph])
        # and through the oracle's own translation
        w = np.frombuffer(data[o - 32768:o], dtype=np.uint8)
        assert oracle.translate(sym, w).tobytes() == data[o:]


def test_predicate_on_true_block_starts_and_brute_force(fastq_stream):
    data, gz, blocks = fastq_stream
    end = (len(gz) - 8) * 8
    offs = _block_offsets(gz, blocks, len(data)) + [len(data)]
    a = np.unpackbits(np.frombuffer(gz, dtype=np.uint8), bitorder="little")
    expect = {}
    for k, b in enumerate(blocks):
        size = offs[k + 1] - offs[k]
        btype = int(a[b + 1]) | (int(a[b + 2]) << 1)
        expect[b] = (a[b] == 0) and btype == 2 and 1024 <= size < (4 << 20)
        assert oracle.block_ok(gz, end, b, ALLOWED)[0] == expect[b], (k, b)
    # brute force over every bit of the first 64 KiB of compressed data
    lo, hi = 80, min(end, 80 + 8 * 65536)
    passing = [b for b in range(lo, hi) if oracle.block_ok(gz, end, b, ALLOWED)[0]]
    true_pass = [b for b in blocks if lo <= b < hi and expect[b]]
    assert passing == true_pass
    # the scan returns the least passing bit of a range
    for s in [lo, true_pass[0], true_pass[0] + 1]:
        got = oracle.sync_scan(gz, end, s, end, ALLOWED)
        assert got == min(b for b in blocks if b >= s and expect[b])


def test_predicate_rejections():
    data = synth.fastq(100000, 100, 0.001, 2)
    raw = zlib.compressobj(6, zlib.DEFLATED, -15)
    deflate = raw.compress(data) + raw.flush()
    gz = dw.gzip_wrap(deflate, data)
    end = (len(gz) - 8) * 8
    e, _, blocks, _ = oracle.gunzip(gz, max_blocks=100)
    b = int(blocks[1])
    assert oracle.block_ok(gz, end, b, ALLOWED)[0]
    # a size bound above the block's size rejects it
    assert oracle.block_ok(gz, end, b, ALLOWED, min_out=10 ** 7)[1] == oracle.E_SIZE
    assert oracle.block_ok(gz, end, b, ALLOWED, max_out=100)[1] == oracle.E_SIZE
    # an allowed set without 'A' rejects it
    m = ALLOWED.copy()
    m[ord("A") >> 3] &= np.uint8(0xFF ^ (1 << (ord("A") & 7)))
    assert oracle.block_ok(gz, end, b, m)[1] == oracle.E_BYTE
    # final and stored/fixed blocks are never sync points
    w = dw.BitWriter(); dw.write_fixed(w, [("lit", 65)] * 2000, False); dw.write_stored(w, b"x", True)
    g2 = dw.gzip_wrap(w.tobytes(), b"A" * 2000 + b"x")
    assert oracle.block_ok(g2, (len(g2) - 8) * 8, 80, ALLOWED)[1] == oracle.E_TYPE
    w = dw.BitWriter(); dw.write_dynamic(w, [("lit", 65)] * 2000, True)
    g3 = dw.gzip_wrap(w.tobytes(), b"A" * 2000)
    assert oracle.block_ok(g3, (len(g3) - 8) * 8, 80, ALLOWED)[1] == oracle.E_FINAL


def test_confirm_and_decompress_at(fastq_stream):
    data, gz, blocks = fastq_stream
    end = (len(gz) - 8) * 8
    offs = _block_offsets(gz, blocks, len(data))
    for b in blocks[1:-1]:
        assert oracle.confirm(gz, end, b, ALLOWED, 5)
    start = blocks[3] - 1000
    r = oracle.decompress_at(gz, start, fill=ord("?"))
    assert r["status"] == 0 and r["block_bit"] == blocks[3]
    o = offs[3]
    truth = data[o:]
    got = r["bytes"]
    assert len(got) == len(truth)
    sym = r["sym"]
    ph = (sym & 0x8000) != 0
    tb = np.frombuffer(truth, dtype=np.uint8)
    gb = np.frombuffer(got, dtype=np.uint8)
    assert np.array_equal(gb[~ph], tb[~ph]) and np.all(gb[ph] == ord("?"))
    fd = r["first_determined"]
    assert fd == (int(np.nonzero(ph)[0][-1]) + 1 if ph.any() else 0)
    r0 = oracle.decompress_at(gz, 0)
    assert r0["status"] == 0 and r0["bytes"] == data and r0["first_determined"] == 0


# ---------------------------------------------------------------- two-pass restatement
@pytest.mark.parametrize("nparts", [1, 2, 3, 8, 40])
@pytest.mark.parametrize("level", [1, 6, 9])
def test_two_pass_equals_gunzip(nparts, level):
    data = synth.fastq(400000, 150, 0.001, 40 + level)
    gz = synth.gzip_compress(data, level)
    r = oracle.two_pass(gz, nparts)
    assert r["status"] == 0
    assert r["out"] == data
    e, _, blocks, _ = oracle.gunzip(gz, max_blocks=10000)
    starts = [int(b) for b in r["part_bits"] if b != oracle.NONE]
    assert set(starts) <= set(int(b) for b in blocks)
    assert int(r["part_len"].sum()) == len(data)
    assert r["part_nph"][0] == 0


def test_two_pass_markov_and_short_parts():
    data = synth.markov(200000, 77)
    gz = synth.gzip_compress(data, 9)
    for n in [2, 16, 64]:                    # at 64 most parts hold no block start (empty parts)
        r = oracle.two_pass(gz, n)
        assert r["status"] == 0 and r["out"] == data


def test_window_chain_pieces():
    rng = np.random.default_rng(3)
    w = rng.integers(32, 127, 32768, dtype=np.uint8)
    sym = rng.integers(32, 127, 1000).astype(np.uint16)
    sym[::7] = 0x8000 | rng.integers(0, 32768, sym[::7].size).astype(np.uint16)
    out = oracle.translate(sym, w)
    ph = (sym & 0x8000) != 0
    assert np.array_equal(out[~ph], sym[~ph].astype(np.uint8))
    assert np.array_equal(out[ph], w[sym[ph] & 0x7FFF])
    nw = oracle.next_window(w, sym)
    assert np.array_equal(nw[:32768 - 1000], w[1000:]) and np.array_equal(nw[32768 - 1000:], out)
    long = rng.integers(32, 127, 40000).astype(np.uint16)
    assert np.array_equal(oracle.next_window(w, long), long[-32768:].astype(np.uint8))


def _seq_syms(text: str):
    """'?' stands for an undetermined symbol."""
    return np.array([0x8000 | 7 if ch == "?" else ord(ch) for ch in text], dtype=np.uint16)


def test_sequence_heuristic_on_hand_cases():
    # Appendix "Heuristic extraction of DNA sequences in DEFLATE block": T D+ (U+ D+)* T, T = newline or U
    cases = {
        "\nACGT\n": [(1, 4, False)],
        "x\nACGT\nIIII": [(2, 4, False)],
        "\nAC??GT\n": [(1, 6, True)],
        "?ACG?TTx?GG\n": [(1, 3, False), (9, 2, False)],     # TT is followed by 'x': the match stops at G
        "+ACGT\n": [],                                       # a quality-like prefix is not a delimiter
        "\nACGTF\n": [],
        "\n??ACG\n": [(3, 3, False)],
        "ACGT\n": [],                                        # no delimiter before the array start
        "\nACGT": [],                                        # nor after its end
        "\nA\n\nC?N\n": [(1, 1, False), (4, 3, True)],
        "\n?\n": [],
    }
    for text, want in cases.items():
        assert oracle.sequences(_seq_syms(text)) == want, text
    assert oracle.sequences(_seq_syms("\nAC??GT\n\nACGTACGT\n"), min_len=8) == [(9, 8, False)]


def test_sequence_heuristic_brute_force():
    """Against the definition: every substring whose both neighbours are T's and whose text is D+(U+D+)*,
    keeping the maximal ones left to right without overlap."""
    rng = np.random.default_rng(5)
    alphabet = "ACGT?\nx"
    for _ in range(300):
        text = "".join(alphabet[k] for k in rng.integers(0, len(alphabet), size=int(rng.integers(1, 40))))
        n = len(text)

        def body_ok(a, b):
            seg = text[a:b + 1]
            if not seg or seg[0] == "?" or seg[-1] == "?":
                return False
            return all(c in "ACGTN?" for c in seg)

        def delim(i):
            return 0 <= i < n and text[i] in "\n?"

        want, i = [], 0
        while i < n:
            ends = [b for b in range(i, n) if delim(i - 1) and delim(b + 1) and body_ok(i, b)]
            if ends:
                b = max(ends)
                want.append((i, b - i + 1, "?" in text[i:b + 1]))
                i = b + 1
            else:
                i += 1
        assert oracle.sequences(_seq_syms(text)) == want, text


@pytest.mark.parametrize("level", [1, 6, 9])
def test_binary_safe_block_start_predicate(level):
    """Data with bytes of every value: with every byte allowed, the predicate rests on the block structure
    alone (complete codes, block size, distances) and the two passes split the member into parts and stay
    exact; with the ASCII mask no start passes and everything is decoded from the first block, still
    exactly.  Pinned by zlib's output."""
    raw = synth.binary_records(1 << 20, 7)
    assert len(set(raw)) == 256 or max(raw) > 126
    gz = synth.gzip_compress(raw, level)
    every = np.full(32, 0xFF, dtype=np.uint8)
    r = oracle.two_pass(gz, 32, allowed=every)
    assert r["status"] == 0 and r["out"] == raw == zlib.decompress(gz, 31)
    assert int((r["part_len"] > 0).sum()) >= 16
    r = oracle.two_pass(gz, 32)
    assert r["status"] == 0 and r["out"] == raw
    assert int((r["part_len"] > 0).sum()) == 1


def test_fuzz_against_zlib_every_window_size_and_strategy():
    """Seeded fuzz: inputs mixing text, binary records, long runs and random bytes, compressed by zlib with
    every window size (wbits 9..15), memLevel, strategy and level; the oracle's gunzip and its two passes
    must give zlib's output exactly (a smaller window is a special case of the 32 KiB one)."""
    rng = np.random.default_rng(11)
    strategies = [zlib.Z_DEFAULT_STRATEGY, zlib.Z_FILTERED, zlib.Z_HUFFMAN_ONLY, zlib.Z_RLE, zlib.Z_FIXED]
    every = np.full(32, 0xFF, dtype=np.uint8)
    for case in range(40):
        pieces = []
        for _ in range(int(rng.integers(1, 5))):
            kind = int(rng.integers(0, 4))
            n = int(rng.integers(1, 60000))
            if kind == 0:
                pieces.append(synth.fastq(n, 100, 0.01, int(rng.integers(1 << 30))))
            elif kind == 1:
                pieces.append(synth.binary_records(n, int(rng.integers(1 << 30))))
            elif kind == 2:
                pieces.append(bytes([int(rng.integers(256))]) * n)
            else:
                pieces.append(rng.integers(0, 256, n, dtype=np.uint8).tobytes())
        raw = b"".join(pieces)
        c = zlib.compressobj(int(rng.integers(0, 10)), zlib.DEFLATED, 16 + int(rng.integers(9, 16)),
                             int(rng.integers(1, 10)), strategies[int(rng.integers(len(strategies)))])
        gz = c.compress(raw) + c.flush()
        e, out, _, _ = oracle.gunzip(gz)
        assert e == 0 and out == raw, case
        for nparts in (3, 8):
            r = oracle.two_pass(gz, nparts, allowed=every)
            assert r["status"] == 0 and r["out"] == raw, (case, nparts)
