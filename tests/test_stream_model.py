"""The segment decomposition behind memory-bounded streaming, restated with the oracle's steps (no GPU).

A member is cut at block starts found past nominal segment ends (the probe). Each segment is decoded
symbolically from its start up to the next segment's start, resolved with the window that the earlier
segments left, and the window is carried on (Section "Undetermined context propagation technique": the
symbols of a segment depend on what precedes it only through the 32 KiB window before its start).  A
probe start that the previous segment does not land on exactly is false, and the search goes on after it.
The concatenated segments must be zlib's output.
"""
import zlib

import numpy as np
import pytest

import oracle
from paper_1905_07224_gb300 import synth


def _segmented(gz: bytes, seg_bytes: int):
    s0 = oracle.gzip_header(gz)
    assert s0 > 0
    end_bit = (len(gz) - 8) * 8
    allowed = oracle.default_allowed()
    b, first = s0 * 8, True
    window = np.zeros(oracle.WSIZE, dtype=np.uint8)
    out, cuts, false_probes = [], [], 0
    while True:
        nominal = (b // 8 + seg_bytes) * 8
        last = nominal >= end_bit
        stop = 0 if last else oracle.sync_scan(gz, end_bit, nominal, end_bit, allowed)
        while True:
            r = oracle.inflate_from(gz, end_bit, b, stop_bit=max(stop, 0), known=first)
            assert r["status"] == 0
            if last or stop < 0 or r["pos"] == stop:
                break
            false_probes += 1                                  # not a block start of this member: search on
            stop = oracle.sync_scan(gz, end_bit, stop + 1, end_bit, allowed)
        if stop < 0:                                           # no block start after the nominal end: to the end
            last = True
        out.append(oracle.translate(r["sym"], window).tobytes())
        window = oracle.next_window(window, r["sym"])
        if last or r["final"]:
            assert r["final"]
            break
        cuts.append(stop)
        b, first = stop, False
    return b"".join(out), cuts, false_probes, [len(x) for x in out]


@pytest.mark.parametrize("kind,level,seg", [("fastq", 6, 256 << 10), ("fastq", 1, 64 << 10),
                                            ("markov", 9, 64 << 10)])
def test_segments_with_carried_windows_give_the_exact_output(kind, level, seg):
    raw = synth.fastq(2 << 20, 150, 0.01, 21) if kind == "fastq" else synth.markov(1 << 20, 22)
    gz = synth.gzip_compress(raw, level)
    got, cuts, _, _ = _segmented(gz, seg)
    # really cut into segments (each ends at the first block start past its nominal end)
    assert len(cuts) >= max(2, (len(gz) - 18) // (2 * seg) - 1)
    assert got == zlib.decompress(gz, 31) == raw


def test_a_segment_that_ends_short_of_its_window_gets_the_zero_prefix():
    """A first segment of less than 32 KiB of output (its block ends at a sync flush after 10000 bytes): the
    window carried out of it is partly before the member, a part no valid stream references."""
    raw = synth.fastq(400000, 100, 0.0, 23)
    c = zlib.compressobj(9, zlib.DEFLATED, 31)
    gz = c.compress(raw[:10000]) + c.flush(zlib.Z_SYNC_FLUSH) + c.compress(raw[10000:]) + c.flush()
    got, cuts, _, lens = _segmented(gz, 1024)
    assert cuts and lens[0] == 10000 and got == raw


def test_a_false_block_start_past_the_segment_end_is_searched_past():
    """The member of the GPU streaming test whose stored block hides a seven-block DEFLATE stream just past
    the first segment's nominal end: the first probes land on those fake blocks and are rejected."""
    from test_gpu_stream import _probe_false_start_member
    gz, data, fake0 = _probe_false_start_member(1 << 20)
    got, cuts, false_probes, _ = _segmented(gz, 1 << 20)
    assert got == data
    assert false_probes >= 1 and cuts[0] > fake0 * 8
