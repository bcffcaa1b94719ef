"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is exact (bytes, u16 symbols, bit offsets, counts): the
method's arithmetic is integer-only.  Stage by stage:
  part start bits       == oracle.two_pass part_bits (block-start search)
  pass-1 symbols (u16)  == oracle.inflate_from(start, stop) of each part
  placeholder counts    == the oracle's counts
  windows w_i           == the 32 KiB of true output before part i
  output bytes          == oracle.gunzip == the generator's text
"""
import zlib

import numpy as np
import pytest

import oracle
import deflate_writer as dw
from gpu_util import Ctx, to_device, empty
from paper_1905_07224_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    """1 MiB FASTQ, 100 bp, seed 0, level 6, 8 parts (the small workload)."""
    data = synth.fastq(1 << 20, 100, 0.001, 0)
    gz = synth.gzip_compress(data, 6)
    return data, gz


def _check_parts(ctx, data, gz, nparts):
    ref = oracle.two_pass(gz, nparts)
    assert ref["status"] == 0 and ref["out"] == data
    pgz = ctx.pgz
    sb, ns, nph = pgz.pgz_inspect_parts(ctx.h)
    assert len(sb) == nparts
    ob = ref["part_bits"].astype(np.uint64)
    used = ob != np.uint64(oracle.NONE)
    assert np.array_equal(sb[used], ob[used])
    assert np.all(sb[~used] == np.uint64(pgz.NONE))
    assert np.array_equal(ns, ref["part_len"])
    assert np.array_equal(nph, ref["part_nph"])
    end = (len(gz) - 8) * 8
    starts = [int(b) for b in ob[used]]
    idx = np.nonzero(used)[0]
    off = 0
    for k, i in enumerate(idx):
        stop = starts[k + 1] if k + 1 < len(starts) else 0
        r = oracle.inflate_from(gz, end, starts[k], stop, known=(i == 0))
        assert r["status"] == 0
        got = pgz.pgz_inspect_symbols(ctx.h, int(i))
        assert np.array_equal(got, r["sym"]), f"part {i}"
        w = pgz.pgz_inspect_window(ctx.h, int(i))
        if i > 0:
            lo = max(0, off - 32768)
            truth_w = np.frombuffer(data[lo:off], dtype=np.uint8)
            assert np.array_equal(w[32768 - truth_w.size:], truth_w), f"window {i}"
        off += int(ns[i])


def test_small_workload_parts_and_output(cfg1):
    data, gz = cfg1
    ctx = Ctx(n_chunks=8)
    try:
        st, out, n, s = ctx.decompress(gz, stats=True)
        assert st == 0, ctx.pgz.pgz_strerror(st)
        assert n == len(data) and out == data
        _check_parts(ctx, data, gz, 8)
        assert s["placeholders"] > 0 and s["chunks"] == 8
    finally:
        ctx.close()


@pytest.mark.parametrize("nparts", [1, 2, 3, 64, 300])
def test_part_counts(cfg1, nparts):
    data, gz = cfg1
    ctx = Ctx(n_chunks=nparts)
    try:
        st, out, n, _ = ctx.decompress(gz)
        assert st == 0 and out == data
        _check_parts(ctx, data, gz, nparts)
    finally:
        ctx.close()


@pytest.mark.parametrize("tail", [0, 1])
@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("level", [1, 6, 9])
@pytest.mark.parametrize("kind", ["fastq", "markov"])
def test_levels_and_kinds(level, kind, pipe, tail):
    data = synth.fastq(3 << 20, 150, 0.01, 5) if kind == "fastq" else synth.markov(3 << 20, 6)
    gz = synth.gzip_compress(data, level)
    ctx = Ctx(n_chunks=24, exec_pipelined=pipe, determined_tail=tail)
    try:
        st, out, n, _ = ctx.decompress(gz)
        assert st == 0, ctx.pgz.pgz_strerror(st)
        assert out == data
        _check_parts(ctx, data, gz, 24)
    finally:
        ctx.close()


@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("kind,level", [("markov", 6), ("markov", 1), ("fastq", 9)])
def test_determined_tail(kind, level, pipe):
    """Once a part's last 32 KiB of output hold no placeholder, none can follow (Section "Undetermined context
    propagation technique"), and pass 1 (with the determined_tail option) stores the rest of the part as bytes.  The pass-1 symbols read back
    through the inspection call equal the oracle's symbolic decode, the windows and the output are exact, and
    the count of symbols stored as bytes is at most each part's symbols past its last placeholder plus
    32 KiB (positive for Markov text, whose matches rarely reach back to a part's start).  Byte ranges through
    the index read the tails too."""
    data = synth.markov(6 << 20, 41) if kind == "markov" else synth.fastq(6 << 20, 150, 0.001, 41)
    gz = synth.gzip_compress(data, level)
    n = 12
    ctx = Ctx(n_chunks=n, exec_pipelined=pipe, determined_tail=1)
    try:
        st, out, _, s = ctx.decompress(gz, stats=True)
        assert st == 0, ctx.pgz.pgz_strerror(st)
        assert out == data
        _check_parts(ctx, data, gz, n)
        ref = oracle.two_pass(gz, n)
        bits = [int(b) for b in ref["part_bits"]]
        used = [i for i, b in enumerate(bits) if b != oracle.NONE]
        end = (len(gz) - 8) * 8
        bound = 0
        for k, i in enumerate(used):
            stop = bits[used[k + 1]] if k + 1 < len(used) else 0
            sym = oracle.inflate_from(gz, end, bits[i], stop, known=(i == 0))["sym"]
            ph = np.nonzero(sym & 0x8000)[0]
            last = int(ph[-1]) + 1 if ph.size else 0
            bound += max(0, sym.size - (last + 32768))
        assert s["determined"] <= bound
        if kind == "markov":
            assert s["determined"] > 0
        P = ctx.pgz
        d = to_device(gz)
        idx = P.pgz_index_build(ctx.h, d.data_ptr(), len(gz))
        try:
            rng = np.random.default_rng(level + 10 * pipe)
            for off, ln in [(0, len(data)), (len(data) - 5000, 5000)] + \
                    [(int(o), 200000) for o in rng.integers(0, len(data) - 200000, 6)]:
                o = empty(ln)
                assert P.pgz_decompress_range(ctx.h, idx, off, ln, o.data_ptr()) == 0
                assert o[:ln].cpu().numpy().tobytes() == data[off:off + ln], (off, ln)
        finally:
            P.pgz_index_free(idx)
    finally:
        ctx.close()


@pytest.mark.parametrize("level", [1, 9])
def test_binary_data_with_every_byte_allowed(level):
    """Bytes of every value: with the allowed-byte mask opened to all 256 values, the block-start predicate
    rests on the block structure alone.  The output must be exact.  Every part start the run kept must be a
    true block start of the member (false ones are rejected by the chain check), and the member must really
    be split.  With the default ASCII mask no part start passes, and the first part decodes everything,
    exactly."""
    raw = synth.binary_records(1 << 20, 7)
    gz = synth.gzip_compress(raw, level)
    e, ref, blocks, _ = oracle.gunzip(gz, max_blocks=4096)
    assert e == 0 and ref == raw
    true_starts = {int(b) for b in blocks}
    every = np.full(32, 0xFF, dtype=np.uint8)
    ctx = Ctx(n_chunks=32, allowed=every)
    try:
        st, out, n, s = ctx.decompress(gz, stats=True)
        assert st == 0, ctx.pgz.pgz_strerror(st)
        assert out == raw
        sb, ns, _ = ctx.pgz.pgz_inspect_parts(ctx.h)
        kept = [int(b) for b, k in zip(sb, ns) if k > 0]
        assert set(kept) <= true_starts
        assert len(kept) >= 8
    finally:
        ctx.close()
    ctx = Ctx(n_chunks=32)
    try:
        st, out, n, s = ctx.decompress(gz, stats=True)
        assert st == 0 and out == raw
        assert s["empty_chunks"] == 31
    finally:
        ctx.close()


def _hand(blocks):
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
    return dw.gzip_wrap(w.tobytes(), text), text


@pytest.mark.parametrize("pipe", [0, 1])
def test_edge_inputs(pipe):
    big = synth.fastq(40000, 100, 0.0, 7)
    cases = {
        "empty": (synth.gzip_compress(b"", 6), b""),
        "one": (synth.gzip_compress(b"A", 6), b"A"),
        "run258": (synth.gzip_compress(b"z" * 300000, 9), b"z" * 300000),
        "64k+1": (synth.gzip_compress(synth.fastq(65537, 100, 0.0, 1), 6), synth.fastq(65537, 100, 0.0, 1)),
        "binary_stored": None,
        "hand": _hand([("stored", b"head\n"), ("fixed", [("lit", c) for c in b"abcabc"] + [("match", 258, 3)]),
                       ("dynamic", dw.tokens_from_text(big)), ("stored", b"tail\n")]),
        "maxdist": _hand([("dynamic", [("lit", b) for b in big[:32768]] + [("match", 258, 32768)])]),
        "header_flags": None,
    }
    binary = np.random.default_rng(1).integers(0, 256, 200000, dtype=np.uint8).tobytes()
    cases["binary_stored"] = (synth.gzip_compress(binary, 0), binary)
    raw = zlib.compressobj(6, zlib.DEFLATED, -15)
    txt = synth.markov(100000, 2)
    cases["header_flags"] = (dw.gzip_wrap(raw.compress(txt) + raw.flush(), txt, flags=2 | 4 | 8 | 16,
                                          name=b"x" * 5000, extra=b"e" * 300, comment=b"c"), txt)
    for nparts in [1, 4, 32]:
        ctx = Ctx(n_chunks=nparts, exec_pipelined=pipe)
        try:
            for name, (gz, text) in cases.items():
                st, out, n, _ = ctx.decompress(gz)
                assert st == 0, (name, nparts, ctx.pgz.pgz_strerror(st))
                assert out == text, (name, nparts)
        finally:
            ctx.close()


def test_errors():
    pgz_ok = synth.gzip_compress(synth.fastq(500000, 100, 0.0, 3), 6)
    data = synth.fastq(500000, 100, 0.0, 3)
    ctx = Ctx(n_chunks=8)
    try:
        P = ctx.pgz
        bad_crc = pgz_ok[:-8] + bytes([pgz_ok[-8] ^ 1]) + pgz_ok[-7:]
        assert ctx.decompress(bad_crc)[0] == P.PGZ_E_CRC
        bad_isize = pgz_ok[:-4] + bytes([pgz_ok[-4] ^ 1]) + pgz_ok[-3:]
        assert ctx.decompress(bad_isize)[0] == P.PGZ_E_ISIZE
        assert ctx.decompress(b"\x1f\x8c" + pgz_ok[2:])[0] == P.PGZ_E_HEADER
        assert ctx.decompress(pgz_ok[:len(pgz_ok) // 2] + pgz_ok[-8:])[0] in (P.PGZ_E_DATA, P.PGZ_E_CRC)
        assert ctx.decompress(pgz_ok + b"not a gzip member")[0] == P.PGZ_E_UNSUPPORTED
        st, _, n, _ = ctx.decompress(pgz_ok, out_cap=1000)
        assert st == P.PGZ_E_CAPACITY and n == len(data)
        # a distance before the member start
        w = dw.BitWriter()
        dw.write_fixed(w, [("lit", 65), ("match", 3, 2)], True)
        assert ctx.decompress(dw.gzip_wrap(w.tobytes(), b"AAAA"))[0] == P.PGZ_E_DATA
        # the context still works afterwards
        st, out, _, _ = ctx.decompress(pgz_ok)
        assert st == 0 and out == data
    finally:
        ctx.close()


def test_decompress_at_matches_oracle(cfg1):
    data, gz = cfg1
    ctx = Ctx(n_chunks=8)
    try:
        P = ctx.pgz
        d = to_device(gz)
        for start in [0, 80, 1000, (len(gz) // 3) * 8 + 5, (len(gz) * 2 // 3) * 8]:
            ref = oracle.decompress_at(gz, start, fill=ord("?"))
            cap = len(data) + 65536
            sym = empty(cap * 2)
            byt = empty(cap)
            st, n, bb, fd = P.pgz_decompress_at(ctx.h, d.data_ptr(), len(gz), start, sym.data_ptr(),
                                                byt.data_ptr(), ord("?"), cap)
            assert st == ref["status"] == 0
            assert bb == ref["block_bit"] and n == ref["sym"].size and fd == ref["first_determined"]
            s = sym.view(dtype=__import__("torch").int16)[:n].cpu().numpy().view(np.uint16)
            assert np.array_equal(s, ref["sym"])
            assert byt[:n].cpu().numpy().tobytes() == ref["bytes"]
        st, n, bb, fd = P.pgz_decompress_at(ctx.h, d.data_ptr(), len(gz), (len(gz) - 9) * 8, None, None, 63, 1 << 20)
        assert st == P.PGZ_E_NOSYNC
    finally:
        ctx.close()


def test_batch_and_graph():
    import torch
    man = synth.batch_manifest(12, seed=9, lo=1 << 10, hi=4 << 20)
    files = [synth.make_file(*e) for e in man]
    ctx = Ctx(n_chunks=0, chunk_bytes=128 << 10)
    try:
        P = ctx.pgz
        dev = [to_device(g) for _, g in files]
        outs = [empty(len(r) + 4096) for r, _ in files]
        jobs = [(dev[k].data_ptr(), len(files[k][1]), outs[k].data_ptr(), len(files[k][0]) + 4096)
                for k in range(len(files))]
        st, res, s = P.pgz_decompress_batch(ctx.h, jobs, stats=True)
        assert st == 0, [P.pgz_strerror(r[0]) for r in res]
        for k, (raw, _) in enumerate(files):
            assert res[k] == (0, len(raw))
            assert outs[k][:len(raw)].cpu().numpy().tobytes() == raw
        b = P.Batch(ctx.h, jobs)
        try:
            for _ in range(2):
                for o in outs:
                    o.zero_()
                torch.cuda.synchronize()
                st, res, s = b.run(stats=True)
                assert st == 0
                for k, (raw, _) in enumerate(files):
                    assert res[k] == (0, len(raw))
                    assert outs[k][:len(raw)].cpu().numpy().tobytes() == raw
        finally:
            b.free()
    finally:
        ctx.close()


def test_index_and_ranges(cfg1):
    data, gz = cfg1
    ctx = Ctx(n_chunks=16)
    try:
        P = ctx.pgz
        d = to_device(gz)
        idx = P.pgz_index_build(ctx.h, d.data_ptr(), len(gz))
        try:
            total, nparts = P.pgz_index_info(idx)
            assert total == len(data) and nparts >= 2
            rng = np.random.default_rng(4)
            ranges = [(0, 10), (len(data) - 10, 10), (123456, 70000), (0, len(data))]
            ranges += [(int(o), int(min(len(data) - o, l))) for o, l in
                       zip(rng.integers(0, len(data), 8), rng.integers(1, 300000, 8))]
            for off, ln in ranges:
                out = empty(ln)
                st = P.pgz_decompress_range(ctx.h, idx, off, ln, out.data_ptr())
                assert st == 0, P.pgz_strerror(st)
                assert out[:ln].cpu().numpy().tobytes() == data[off:off + ln], (off, ln)
        finally:
            P.pgz_index_free(idx)
    finally:
        ctx.close()


def test_host_entry_point(cfg1):
    data, gz = cfg1
    ctx = Ctx(n_chunks=8)
    try:
        out = np.zeros(len(data) + 100, dtype=np.uint8)
        st, n, s = ctx.pgz.pgz_decompress_host(ctx.h, gz, out, stats=True)
        assert st == 0 and n == len(data) and out[:n].tobytes() == data
        assert ctx.pgz.pgz_kernel_launches(ctx.h) > 0
    finally:
        ctx.close()


def test_host_batch_entry_point():
    """pgz_decompress_batch_host: members in host memory (page-locked and pageable), cut into groups whose
    copies overlap the decoding.  Six 64 MiB members of Markov text (about 300 MiB compressed) make the batch
    span three groups (a short first and last one); a member with a hidden false block start needs recovery
    inside the last group; a member with a wrong trailer CRC fails alone.  Every other output is exact."""
    import torch
    import confirm_streams as cs
    m = cs.find("invalid", 2)
    raws = [synth.markov(64 << 20, 30 + k) for k in range(6)] + [synth.fastq(3 << 20, 150, 0.001, 34), m.data]
    gzs = [synth.gzip_compress(r, 1) for r in raws[:7]] + [m.gz]
    bad = bytearray(synth.gzip_compress(raws[6], 6))
    bad[-8] ^= 1
    raws.insert(2, raws[6])
    gzs.insert(2, bytes(bad))
    ctx = Ctx(n_chunks=0, chunk_bytes=64 << 10)
    try:
        P = ctx.pgz
        for pinned in (True, False):
            ins = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()) for g in gzs]
            outs = [torch.zeros(len(r) + 4096, dtype=torch.uint8) for r in raws]
            if pinned:
                ins = [t.pin_memory() for t in ins]
                outs = [t.pin_memory() for t in outs]
            jobs = [(ins[k].data_ptr(), len(gzs[k]), outs[k].data_ptr(), outs[k].numel()) for k in range(len(gzs))]
            for _ in range(2):
                for o in outs:
                    o.zero_()
                st, res, s = P.pgz_decompress_batch_host(ctx.h, jobs, stats=True)
                assert st == P.PGZ_E_CRC
                for k, raw in enumerate(raws):
                    if k == 2:
                        assert res[k][0] == P.PGZ_E_CRC
                        continue
                    assert res[k] == (0, len(raw)), (k, P.pgz_strerror(res[k][0]))
                    assert outs[k][:len(raw)].numpy().tobytes() == raw, k
                assert s["out_bytes"] >= sum(len(r) for k, r in enumerate(raws) if k != 2)
    finally:
        ctx.close()


def test_multi_member_files():
    """RFC 1952 2.2: a gzip file is a series of members; the output is their concatenation (the oracle decodes
    every member)."""
    a = synth.fastq(700000, 150, 0.001, 21)
    b = synth.markov(300000, 22)
    c = synth.fastq(90000, 100, 0.001, 23)
    cases = [
        [(a, 1), (b, 9)],
        [(a, 6), (b"", 6), (c, 1), (b, 6)],
        [(c, 9)] * 5,
    ]
    for nparts in (1, 8):
        ctx = Ctx(n_chunks=nparts)
        try:
            for members in cases:
                gz = b"".join(synth.gzip_compress(d, lv) for d, lv in members)
                want = b"".join(d for d, _ in members)
                e, ref, _, _ = oracle.gunzip(gz, cap=len(want) + 1024)
                assert e == 0 and ref == want
                st, out, n, s = ctx.decompress(gz, stats=True)
                assert st == 0, ctx.pgz.pgz_strerror(st)
                assert out == want
                # the host-buffer entry point takes the same path
                host_out = np.zeros(len(want) + 64, dtype=np.uint8)
                st, n, _ = ctx.pgz.pgz_decompress_host(ctx.h, gz, host_out)
                assert st == 0 and host_out[:n].tobytes() == want
                # a damaged second member is caught by its own trailer
                second = len(synth.gzip_compress(members[0][0], members[0][1]))
                bad = bytearray(gz)
                bad[second + len(synth.gzip_compress(members[1][0], members[1][1])) - 5] ^= 1
                assert ctx.decompress(bytes(bad))[0] in (ctx.pgz.PGZ_E_CRC, ctx.pgz.PGZ_E_ISIZE)
        finally:
            ctx.close()


@pytest.mark.parametrize("level", [1, 6, 9])
def test_bgzf_members_in_one_run(level):
    """BGZF: every member's size is in its header, so all members are found from the headers and decoded in
    one run."""
    data = synth.fastq(3 << 20, 150, 0.001, 24 + level)
    bz = synth.bgzf_compress(data, level)
    ctx = Ctx()
    try:
        st, out, n, s = ctx.decompress(bz, stats=True)
        assert st == 0, ctx.pgz.pgz_strerror(st)
        assert out == data
        assert s["chunks"] >= (len(data) + 65279) // 65280 + 1      # at least one part per member
        st, _, n, _ = ctx.decompress(bz, out_cap=len(data) - 1)
        assert st == ctx.pgz.PGZ_E_CAPACITY and n == len(data)
        bad = bytearray(bz)
        bad[len(bz) // 2] ^= 0x10                                 # inside some member's data
        assert ctx.decompress(bytes(bad))[0] in (ctx.pgz.PGZ_E_DATA, ctx.pgz.PGZ_E_CRC, ctx.pgz.PGZ_E_ISIZE,
                                                 ctx.pgz.PGZ_E_HEADER, ctx.pgz.PGZ_E_UNSUPPORTED)
    finally:
        ctx.close()


def _false_start_stream():
    """A member whose stored block carries, as payload, a complete valid DEFLATE stream (six non-final dynamic
    blocks of text and a final one): inside the payload that stream's first block passes every block-start
    check, but it is not a block start of the member."""
    text = synth.fastq(120000, 100, 0.001, 31)
    fake_text = synth.fastq(14000, 100, 0.001, 32)
    wf = dw.BitWriter()
    for k in range(7):
        part = fake_text[2000 * k:2000 * (k + 1)]
        dw.write_dynamic(wf, dw.tokens_from_text(part), k == 6)
    fake = wf.tobytes()
    pad = b"\x00" * 4000
    payload = pad + fake + b"\x00" * 64
    w = dw.BitWriter()
    dw.write_dynamic(w, dw.tokens_from_text(text[:60000]), False)
    head_bits = w.nbits
    dw.write_stored(w, payload, False)
    dw.write_dynamic(w, dw.tokens_from_text(text[60000:]), True)
    data = text[:60000] + payload + text[60000:]
    gz = dw.gzip_wrap(w.tobytes(), data)
    pay0 = 10 + ((head_bits + 3 + 7) // 8) + 4            # header, first block, stored header; byte of the payload
    return gz, data, pay0, pay0 + len(pad)


def test_false_block_start_is_caught_by_the_chain_check():
    gz, data, pad0, fake0 = _false_start_stream()
    assert gz[fake0:fake0 + 1] and oracle.block_ok(gz, (len(gz) - 8) * 8, fake0 * 8, oracle.default_allowed())[0]
    csize = len(gz) - 18
    # part counts whose nominal start of some part falls in the padding before the hidden stream
    picks = [n for n in range(8, 200) if any(pad0 <= 10 + i * ((csize + n - 1) // n) < fake0 for i in range(1, n))]
    assert picks
    for n in picks[:3]:
        ref = oracle.two_pass(gz, n)
        assert ref["status"] == 0 and ref["out"] == data
        ctx = Ctx(n_chunks=n)
        try:
            st, out, _, s = ctx.decompress(gz, stats=True)
            assert st == 0, ctx.pgz.pgz_strerror(st)
            assert out == data
            assert s["false_syncs"] >= 1 and s["retries"] >= 1
            assert s["false_syncs"] == ref["false_syncs"]
            sb, _, _ = ctx.pgz.pgz_inspect_parts(ctx.h)
            assert np.array_equal(sb, ref["part_bits"].astype(np.uint64))
        finally:
            ctx.close()


def _spans(ctx, sym_np, min_len, max_spans=1 << 16):
    import torch
    d = torch.from_numpy(sym_np.astype(np.int16).view(np.int16).copy()).cuda() if sym_np.size else \
        torch.zeros(1, dtype=torch.int16, device="cuda")
    sp = torch.zeros(2 * max_spans, dtype=torch.int64, device="cuda")
    st, n, nu = ctx.pgz.pgz_extract_sequences(ctx.h, d.data_ptr(), sym_np.size, min_len, sp.data_ptr(), max_spans)
    assert st == 0
    a = sp[:2 * min(n, max_spans)].cpu().numpy().view(np.uint64).reshape(-1, 2)
    got = sorted((int(s), int(l & ((1 << 63) - 1)), bool(l >> 63)) for s, l in a)
    return got, n, nu


def test_sequence_heuristic_matches_the_oracle():
    """Appendix "Heuristic extraction of DNA sequences in DEFLATE block" on the GPU against the oracle: random
    symbol strings (runs across the kernel's segments included) and the symbols of a random access into FASTQ
    (with undetermined characters)."""
    ctx = Ctx()
    try:
        rng = np.random.default_rng(11)
        alphabet = np.array([ord(c) for c in "ACGTN\nx"] + [0x8000 | 5, 0], dtype=np.uint16)
        for size, weights in [(5000, None), (70000, [8, 8, 8, 8, 1, 2, 3, 4, 1])]:
            p = None if weights is None else np.array(weights, float) / sum(weights)
            s = alphabet[rng.choice(alphabet.size, size=size, p=p)]
            for min_len in (0, 3, 20):
                want = oracle.sequences(s, min_len)
                got, n, nu = _spans(ctx, s, min_len)
                assert got == want and n == len(want) and nu == sum(u for _, _, u in want), (size, min_len)
        # random access into FASTQ: the paper's use of the heuristic
        data = synth.fastq(1 << 20, 100, 0.001, 12)
        gz = synth.gzip_compress(data, 6)
        for start in (300_000 * 8, 41_234 * 8 + 3):
            r = oracle.decompress_at(gz, start, cap=len(data) + 4096)
            assert r["status"] == 0
            want = oracle.sequences(r["sym"], 50)
            got, n, nu = _spans(ctx, r["sym"], 50)
            assert got == want and n == len(want)
            # reads are found (an undetermined newline can also join a read to quality characters that look
            # like bases: the heuristic's false positives, as the paper notes)
            assert n > 100 and any(l == 100 for _, l, _ in want)
        # fewer slots than spans: the count is still complete
        s = np.array([ord(c) for c in "\nACGT" * 50 + "\n"], dtype=np.uint16)
        got, n, nu = _spans(ctx, s, 1, max_spans=7)
        assert n == 50 and len(got) == 7
    finally:
        ctx.close()
