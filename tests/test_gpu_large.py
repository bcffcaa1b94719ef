"""Full-size cases: the 4 GiB member whose ISIZE wraps to 0, the autotuner, and
the batch of 512 members decoded in one graph-captured run.

Outputs are compared byte for byte with the generator's text (which host zlib
compressed, so it is the exact decompression); a sample of the members is also
compared with the CPU oracle.
"""
import numpy as np
import pytest

import oracle
from gpu_util import Ctx, to_device, empty
from paper_1905_07224_gb300 import synth

pytestmark = pytest.mark.gpu


def _same_on_device(out, raw: bytes) -> bool:
    import torch
    ref = torch.from_numpy(np.frombuffer(raw, dtype=np.uint8).copy()).cuda()
    return bool(torch.equal(out[:len(raw)], ref))


@pytest.mark.slow
def test_4gib_member_isize_wraps_to_zero():
    """4 GiB of FASTQ (150 bp, 1 % N, seed 2) at gzip -6: ISIZE = 2^32 mod 2^32 = 0 (RFC 1952)."""
    raw = synth.fastq_large(4 << 30, 150, 0.01, 2)
    gz = synth.gzip_compress_parallel(raw, 6)
    assert int.from_bytes(gz[-4:], "little") == 0
    ctx = Ctx()
    d = to_device(gz)
    out = empty(len(raw) + 4096)
    st, n, s = ctx.pgz.pgz_decompress(ctx.h, d.data_ptr(), len(gz), out.data_ptr(), out.numel(), True)
    assert st == 0, ctx.pgz.pgz_strerror(st)
    assert n == len(raw) == 4 << 30
    assert _same_on_device(out, raw)
    # the trailer is checked: a wrong ISIZE or CRC is reported, not ignored
    bad = bytearray(gz[-8:])
    bad[4] ^= 1
    d[len(gz) - 4:len(gz)].copy_(d.new_tensor(list(bad[4:])))
    st, _, _ = ctx.pgz.pgz_decompress(ctx.h, d.data_ptr(), len(gz), out.data_ptr(), out.numel(), False)
    assert st == ctx.pgz.PGZ_E_ISIZE
    bad = bytearray(gz[-8:])
    bad[0] ^= 1
    d[len(gz) - 8:len(gz)].copy_(d.new_tensor(list(bad)))
    st, _, _ = ctx.pgz.pgz_decompress(ctx.h, d.data_ptr(), len(gz), out.data_ptr(), out.numel(), False)
    assert st == ctx.pgz.PGZ_E_CRC
    ctx.close()


def test_autotune_picks_the_fastest_working_pair():
    raw = synth.fastq(32 << 20, 150, 0.01, 2)
    gz = synth.gzip_compress(raw, 6)
    ctx = Ctx()
    d = to_device(gz)
    out = empty(len(raw) + 4096)
    chunks, wpbs = [32 << 10, 64 << 10, 256 << 10], [2, 4, 8]
    job = [(d.data_ptr(), len(gz), out.data_ptr(), out.numel())]
    st, entries, best = ctx.pgz.pgz_autotune(ctx.h, job, chunks, wpbs, 2)
    assert st == 0
    assert len(entries) == 9 and all(e["status"] == 0 and e["ms"] > 0 for e in entries)
    assert [(e["chunk_bytes"], e["warps_per_block"]) for e in entries] == [(c, w) for c in chunks for w in wpbs]
    assert best["ms"] == min(e["ms"] for e in entries)
    assert _same_on_device(out, raw)
    # the context now decodes with the chosen pair
    out.zero_()
    st, n, s = ctx.pgz.pgz_decompress(ctx.h, d.data_ptr(), len(gz), out.data_ptr(), out.numel(), True)
    assert st == 0 and n == len(raw) and _same_on_device(out, raw)
    parts = (len(gz) - 18 + best["chunk_bytes"] - 1) // best["chunk_bytes"]
    assert s["chunks"] == parts
    # the pass-1 execution form as a third dimension: both forms decode, the context keeps the fastest
    st, entries, best = ctx.pgz.pgz_autotune(ctx.h, job, [64 << 10], [4], 1, sweep_exec=True)
    assert st == 0 and [e["exec_pipelined"] for e in entries] == [0, 1]
    assert all(e["status"] == 0 for e in entries) and best["ms"] == min(e["ms"] for e in entries)
    assert _same_on_device(out, raw)
    # invalid lists are rejected without running anything
    assert ctx.pgz.pgz_autotune(ctx.h, job, [1024], [4], 1)[0] == ctx.pgz.PGZ_E_ARG
    assert ctx.pgz.pgz_autotune(ctx.h, job, [65536], [3], 1)[0] == ctx.pgz.PGZ_E_ARG
    ctx.close()


def test_a_cached_tuning_is_applied_without_timing(tmp_path):
    from paper_1905_07224_gb300 import tune_cache as tc
    raw = synth.fastq(8 << 20, 150, 0.01, 3)
    gz = synth.gzip_compress(raw, 1)
    d = to_device(gz)
    out = empty(len(raw) + 4096)
    job = [(d.data_ptr(), len(gz), out.data_ptr(), out.numel())]
    key = tc.cache_key("test-gpu", gz[8], len(gz))
    path = str(tmp_path / "tune.json")
    ctx = Ctx()
    st, e, hit = tc.autotune_cached(ctx.pgz, ctx.h, job, key, tc.TuneCache(path), [32 << 10, 128 << 10], [4, 8], 1)
    assert st == 0 and not hit
    ctx.close()
    ctx = Ctx()                                           # a new context: the stored choice, no timing
    st, e, hit = tc.autotune_cached(ctx.pgz, ctx.h, job, key, tc.TuneCache(path), [32 << 10], [4], 1)
    assert st == 0 and hit
    out.zero_()
    st, n, s = ctx.pgz.pgz_decompress(ctx.h, d.data_ptr(), len(gz), out.data_ptr(), out.numel(), True)
    assert st == 0 and n == len(raw) and _same_on_device(out, raw)
    assert s["chunks"] == (len(gz) - 18 + e["chunk_bytes"] - 1) // e["chunk_bytes"]
    # invalid values leave the context as it was
    assert ctx.pgz.pgz_set_tuning(ctx.h, 1024, 4, 0) == ctx.pgz.PGZ_E_ARG
    assert ctx.pgz.pgz_set_tuning(ctx.h, 65536, 5, 0) == ctx.pgz.PGZ_E_ARG
    assert ctx.pgz.pgz_set_tuning(ctx.h, 65536, 4, 7) == ctx.pgz.PGZ_E_ARG
    st, n, s = ctx.pgz.pgz_decompress(ctx.h, d.data_ptr(), len(gz), out.data_ptr(), out.numel(), True)
    assert st == 0 and s["chunks"] == (len(gz) - 18 + e["chunk_bytes"] - 1) // e["chunk_bytes"]
    ctx.close()


@pytest.mark.parametrize("wpb", [2, 8])
def test_cta_shapes_match_the_oracle(wpb):
    data = synth.fastq(1 << 20, 100, 0.001, 0)
    gz = synth.gzip_compress(data, 6)
    ctx = Ctx(n_chunks=8, warps_per_block=wpb)
    st, out, n, s = ctx.decompress(gz, stats=True)
    assert st == 0 and out == data
    ref = oracle.two_pass(gz, 8)
    sb, ns, nph = ctx.pgz.pgz_inspect_parts(ctx.h)
    assert np.array_equal(ns, ref["part_len"]) and np.array_equal(nph, ref["part_nph"])
    ctx.close()


@pytest.mark.slow
def test_batch_of_512_members_in_one_graph():
    """512 members, log-uniform 64 KiB .. 64 MiB (seed 3), FASTQ and Markov text, levels 1/6/9."""
    import torch
    entries = synth.batch_manifest(512, 3)
    files = synth.make_files(entries)
    ctx = Ctx()
    pgz = ctx.pgz
    d_in = [to_device(gz) for _, gz in files]
    d_out = [empty(len(raw) + 4096) for raw, _ in files]
    jobs = [(d_in[k].data_ptr(), len(gz), d_out[k].data_ptr(), d_out[k].numel()) for k, (_, gz) in enumerate(files)]
    b = pgz.Batch(ctx.h, jobs)
    for run in range(2):                                  # the captured graph is re-launched
        for o in d_out:
            o.zero_()
        r, res, _ = b.run()
        assert r == 0
        torch.cuda.synchronize()
        for k, (raw, _) in enumerate(files):
            assert res[k] == (0, len(raw)), k
            assert _same_on_device(d_out[k], raw), k
    b.free()
    # a sample of members against the oracle, byte for byte
    small = sorted(range(len(files)), key=lambda k: len(files[k][0]))[:4]
    for k in small:
        e, out, _, _ = oracle.gunzip(files[k][1], cap=len(files[k][0]) + 1024)
        assert e == 0 and out == files[k][0]
        assert d_out[k][:len(out)].cpu().numpy().tobytes() == out
    ctx.close()


def _scan_ranges(gz: bytes, nparts: int = 0, chunk_bytes: int = 0):
    """Scan ranges [lo_i, hi_i) of a member's parts of equal compressed size, as the library plans them:
    nparts parts, or one per chunk_bytes of compressed data (at most one per 64 bytes)."""
    s0 = oracle.gzip_header(gz)
    csize = len(gz) - 8 - s0
    end = (len(gz) - 8) * 8
    n = nparts or max(1, -(-csize // chunk_bytes))
    n = max(1, min(n, max(1, csize // 64)))
    per = -(-csize // n)
    return [((s0 + i * per) * 8, min((s0 + (i + 1) * per) * 8, end)) for i in range(n)]


def _oracle_start(gz: bytes, lo: int, hi: int) -> int:
    """The oracle's block start of a part: the lowest bit of [lo, hi) passing the block checks and the
    five-block confirmation (none: the library's NONE)."""
    b = oracle.sync_scan(gz, (len(gz) - 8) * 8, lo, hi, oracle.default_allowed(), confirm_blocks=5)
    return b if b >= 0 else pgz_none()


def pgz_none() -> int:
    return (1 << 64) - 1


@pytest.mark.slow
def test_two_256mib_files_full_size():
    """The benchmark's workload: 2 x 256 MiB FASTQ (150 bp, seed 1) at gzip -1 and -9, batched (graph, 64 KiB
    parts, 4 warps per block) and plain (1024 parts per file); sampled parts' u16 symbols against the oracle."""
    import torch
    files = synth.make_files([("fastq", 256 << 20, 1, 1), ("fastq", 256 << 20, 9, 1)])
    ctx = Ctx(chunk_bytes=65536, warps_per_block=4)
    pgz = ctx.pgz
    d_in = [to_device(gz) for _, gz in files]
    d_out = [empty(len(raw) + 4096) for raw, _ in files]
    jobs = [(d_in[k].data_ptr(), len(gz), d_out[k].data_ptr(), d_out[k].numel()) for k, (_, gz) in enumerate(files)]
    b = pgz.Batch(ctx.h, jobs)
    r, res, _ = b.run()
    assert r == 0
    torch.cuda.synchronize()
    for k, (raw, _) in enumerate(files):
        assert res[k] == (0, len(raw)) and _same_on_device(d_out[k], raw)
    b.free()
    # the same batch without the graph, for its part starts: sampled parts of each file against the
    # oracle's own search over the part's scan range (the lowest bit passing the block checks and the
    # confirmation)
    r, _, _ = pgz.pgz_decompress_batch(ctx.h, jobs)
    assert r == 0
    sb, _, _ = pgz.pgz_inspect_parts(ctx.h)
    base = 0
    for raw, gz in files:
        ranges = _scan_ranges(gz, chunk_bytes=65536)
        for i in (1, len(ranges) // 2, len(ranges) - 1):
            assert int(sb[base + i]) == _oracle_start(gz, *ranges[i]), i
        base += len(ranges)
    assert base == len(sb)
    ctx.close()
    plain = Ctx(n_chunks=1024)
    try:
        for (raw, gz), d, o in zip(files, d_in, d_out):
            o.zero_()
            st, n, s = pgz.pgz_decompress(plain.h, d.data_ptr(), len(gz), o.data_ptr(), o.numel(), True)
            assert st == 0 and n == len(raw) and _same_on_device(o, raw)
            assert s["chunks"] == 1024 and s["empty_chunks"] == 0
            sb, ns, nph = pgz.pgz_inspect_parts(plain.h)
            end = (len(gz) - 8) * 8
            ranges = _scan_ranges(gz, nparts=1024)
            for i in (1, 511, 1023):
                assert int(sb[i]) == _oracle_start(gz, *ranges[i]), i
                stop = int(sb[i + 1]) if i + 1 < len(sb) else 0
                ref = oracle.inflate_from(gz, end, int(sb[i]), stop, known=False, cap=int(ns[i]) + 4096)
                assert ref["status"] == 0
                assert np.array_equal(pgz.pgz_inspect_symbols(plain.h, i), ref["sym"]), i
                assert int(nph[i]) == int(np.count_nonzero(ref["sym"] & 0x8000)), i
    finally:
        plain.close()
