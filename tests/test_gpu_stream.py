"""Memory-bounded streaming (pgz_decompress_stream).

A member held in host memory is decoded in segments of its compressed data.
Each segment is one run of the pass kernels that starts at a known block start
with the window the previous segment left, and ends on the block start its
probe part found.  The output must equal the oracle's gunzip (and the
generator's bytes) for every segment size.  The trailer checks (CRC-32
carried across segments, ISIZE of the total) must hold, and a false block start
at a segment's end must be rejected by the chain check and searched past.
"""
import zlib

import numpy as np
import pytest

import oracle
import deflate_writer as dw
from gpu_util import Ctx
from paper_1905_07224_gb300 import synth

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.mark.parametrize("kind,level", [("fastq", 1), ("fastq", 6), ("markov", 9)])
def test_stream_matches_the_oracle(kind, level):
    raw = synth.fastq(12 * MIB, 150, 0.01, 11) if kind == "fastq" else synth.markov(8 * MIB, 12)
    gz = synth.gzip_compress(raw, level)
    e, ref, _, _ = oracle.gunzip(gz)
    assert e == 0 and ref == raw
    ctx = Ctx()
    try:
        for seg in [MIB, 3 * MIB, 0]:
            pieces = []
            st, n, s, _ = ctx.pgz.pgz_decompress_stream(ctx.h, gz, seg, sink=lambda v: pieces.append(bytes(v)),
                                                        stats=True)
            assert st == 0, (seg, ctx.pgz.pgz_strerror(st))
            assert n == len(ref) and b"".join(pieces) == ref
            segments = len(pieces)
            if seg == MIB:
                assert segments >= (len(gz) - 2 * MIB) // MIB    # the member really was cut into segments
            if seg == 0:
                assert segments == 1                              # 256 MiB segments: one run
            assert s["out_bytes"] == len(ref) and s["symbols"] == len(ref)
    finally:
        ctx.close()


def test_stream_of_a_small_member_and_the_empty_member():
    ctx = Ctx()
    try:
        for raw in [b"", b"A", synth.fastq(70000, 100, 0.0, 3)]:
            gz = synth.gzip_compress(raw, 6)
            st, n, _, out = ctx.pgz.pgz_decompress_stream(ctx.h, gz, MIB)
            assert st == 0 and n == len(raw) and out == raw
    finally:
        ctx.close()


def _probe_false_start_member(seg_bytes: int):
    """A member whose first segment (of seg_bytes compressed bytes from the first block) ends inside a stored
    block; the stored payload holds, just past the segment's end, a complete DEFLATE stream of seven dynamic
    blocks.  Each of those blocks passes the block-start checks, so the segment's probe finds them one after
    another before the true block start that follows the stored block."""
    text = synth.fastq(6 * MIB, 150, 0.001, 41)
    seg_end = 10 + seg_bytes                                  # gzip header of 10 bytes, then the first block
    c1 = zlib.compressobj(6, zlib.DEFLATED, -15)
    head = bytearray()
    used = 0
    while 10 + len(head) < seg_end - 50000:
        head += c1.compress(text[used:used + 32768]) + c1.flush(zlib.Z_SYNC_FLUSH)   # byte-aligned, not final
        used += 32768
    assert 10 + len(head) < seg_end - 1000
    wf = dw.BitWriter()
    fake_text = synth.fastq(14000, 100, 0.001, 42)
    for k in range(7):
        dw.write_dynamic(wf, dw.tokens_from_text(fake_text[2000 * k:2000 * (k + 1)]), k == 6)
    fake = wf.tobytes()
    pay0 = 10 + len(head) + 5                                 # stored block: 3 header bits + alignment, LEN, NLEN
    pad = b"\x00" * (seg_end + 100 - pay0)
    payload = pad + fake + b"\x00" * 64
    assert len(payload) <= 65535
    stored = bytes([0]) + len(payload).to_bytes(2, "little") + (len(payload) ^ 0xFFFF).to_bytes(2, "little")
    c2 = zlib.compressobj(6, zlib.DEFLATED, -15)
    tail = c2.compress(text[used:]) + c2.flush()
    data = text[:used] + payload + text[used:]
    gz = dw.gzip_wrap(bytes(head) + stored + payload + tail, data)
    return gz, data, pay0 + len(pad)


def test_false_block_start_at_a_segment_end_is_searched_past():
    gz, data, fake0 = _probe_false_start_member(MIB)
    assert oracle.block_ok(gz, (len(gz) - 8) * 8, fake0 * 8, oracle.default_allowed())[0]
    e, ref, _, _ = oracle.gunzip(gz)
    assert e == 0 and ref == data
    ctx = Ctx()
    try:
        pieces = []
        st, n, s, _ = ctx.pgz.pgz_decompress_stream(ctx.h, gz, MIB, sink=lambda v: pieces.append(bytes(v)),
                                                    stats=True)
        assert st == 0, ctx.pgz.pgz_strerror(st)
        assert b"".join(pieces) == data and n == len(data)
        assert len(pieces) >= 2 and s["false_syncs"] >= 1 and s["retries"] >= 1
    finally:
        ctx.close()


def test_stream_errors():
    raw = synth.fastq(6 * MIB, 150, 0.01, 12)
    gz = synth.gzip_compress(raw, 6)
    ctx = Ctx()
    pgz = ctx.pgz
    try:
        assert pgz.pgz_decompress_stream(ctx.h, gz, 4096)[0] == pgz.PGZ_E_ARG
        assert pgz.pgz_decompress_stream(ctx.h, b"\x00" * 100, MIB)[0] == pgz.PGZ_E_HEADER
        bad = bytearray(gz)
        bad[-8] ^= 1                                          # CRC-32
        st, n, _, _ = pgz.pgz_decompress_stream(ctx.h, bytes(bad), MIB)
        assert st == pgz.PGZ_E_CRC and 0 < n < len(raw)       # earlier segments were delivered
        bad = bytearray(gz)
        bad[-1] ^= 1                                          # ISIZE
        assert pgz.pgz_decompress_stream(ctx.h, bytes(bad), MIB)[0] == pgz.PGZ_E_ISIZE
        assert pgz.pgz_decompress_stream(ctx.h, gz + b"trailing data" * 9000, MIB)[0] == pgz.PGZ_E_UNSUPPORTED
        seen = []

        def stop_after_one(v):
            seen.append(len(v))
            return len(seen) >= 2
        st, n, _, _ = pgz.pgz_decompress_stream(ctx.h, gz, MIB, sink=stop_after_one)
        assert st == pgz.PGZ_E_ABORTED and n == seen[0] and len(seen) == 2
        # an exception in the sink stops the decode and reaches the caller
        def boom(v):
            raise KeyError("sink failed")
        with pytest.raises(KeyError):
            pgz.pgz_decompress_stream(ctx.h, gz, MIB, sink=boom)
        # the context still decodes after every failure
        st, n, _, out = pgz.pgz_decompress_stream(ctx.h, gz, MIB)
        assert st == 0 and out == raw
    finally:
        ctx.close()
