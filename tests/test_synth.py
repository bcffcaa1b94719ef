"""The seeded input generators used by the large cases (CPU only)."""
import re
import zlib

from paper_1905_07224_gb300 import synth


def test_fastq_large_is_one_record_stream():
    a = synth.fastq_large(3 << 20, 150, 0.01, 7, piece=1 << 20, processes=1)
    assert len(a) == 3 << 20
    assert a.startswith(b"@SIM.0 length=150\n")
    heads = [int(x) for x in re.findall(rb"\n@SIM\.(\d+) length=150\n", a)]
    assert heads == list(range(1, len(heads) + 1))          # numbering runs on across piece boundaries
    assert synth.fastq_large(3 << 20, 150, 0.01, 7, piece=1 << 20, processes=1) == a
    lines = a.split(b"\n")
    for k in range(0, len(lines) - 4, 4):
        if lines[k].startswith(b"@SIM."):
            seq, plus, qual = lines[k + 1], lines[k + 2], lines[k + 3]
            if len(seq) == 150 and len(qual) == 150:
                assert plus == b"+" and set(seq) <= set(b"ACGTN") and min(qual) >= 35 and max(qual) <= 73


def test_parallel_gzip_is_one_member():
    data = synth.fastq_large(3 << 20, 150, 0.01, 7, piece=1 << 20, processes=1)
    gz = synth.gzip_compress_parallel(data, 6, piece=1 << 20, processes=1)
    assert gz[:3] == b"\x1f\x8b\x08"
    assert zlib.decompress(gz, 31) == data
    d = zlib.decompressobj(31)
    assert d.decompress(gz) == data and d.eof and d.unused_data == b""
    assert int.from_bytes(gz[-4:], "little") == len(data) & 0xFFFFFFFF
    assert int.from_bytes(gz[-8:-4], "little") == zlib.crc32(data)
    # about the size of a single-stream compression (preset dictionaries across pieces)
    assert len(gz) < 1.01 * len(synth.gzip_compress(data, 6))


def test_bgzf_members_carry_their_sizes():
    import gzip
    data = synth.fastq(300000, 150, 0.001, 9)
    bz = synth.bgzf_compress(data, 6)
    assert gzip.decompress(bz) == data
    off, n = 0, 0
    while off < len(bz):
        assert bz[off:off + 4] == b"\x1f\x8b\x08\x04" and bz[off + 12:off + 16] == b"BC\x02\x00"
        off += int.from_bytes(bz[off + 16:off + 18], "little") + 1
        n += 1
    assert off == len(bz) and n == (len(data) + 65279) // 65280 + 1
