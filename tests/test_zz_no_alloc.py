"""pgz_decompress_noalloc: the entry point for callers that cannot allocate.

Some callers cannot let a library allocate device memory (their own allocator
owns the GPU, a fixed memory budget, or no cudaFree synchronisation allowed in
their loop).  This entry point keeps all scratch in a fixed device array; this
test calls it through the C ABI twice in a row, on different inputs and on the
same input again, and requires byte-identical output to pgz_decompress (the
path is integer-exact, so the tolerance is zero), plus the size limit error,
its recovery paths, that it leaves the device's free memory unchanged, and
that it works as the first library call of a fresh process.
"""
import numpy as np
import pytest

from gpu_util import Ctx, to_device, empty
from paper_1905_07224_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_decompress_on_consecutive_calls():
    import torch
    inputs = [synth.fastq(3 << 20, 150, 0.001, 21), synth.markov(1 << 20, 22), synth.fastq(3 << 20, 150, 0.001, 21)]
    gzs = [synth.gzip_compress(inputs[0], 6), synth.gzip_compress(inputs[1], 1), synth.gzip_compress(inputs[2], 6)]
    ctx = Ctx(n_chunks=0, chunk_bytes=32768)
    try:
        P = ctx.pgz
        for raw, gz in zip(inputs, gzs):
            st, ref, n, _ = ctx.decompress(gz, out_cap=len(raw) + 4096)
            assert st == 0 and ref == raw
            d = to_device(gz)
            out = empty(len(raw) + 4096)
            out.fill_(0xAB)
            torch.cuda.synchronize()
            st, n = P.pgz_decompress_noalloc(d.data_ptr(), len(gz), out.data_ptr(), len(raw) + 4096, None)
            torch.cuda.synchronize()
            assert st == 0, P.pgz_strerror(st)
            assert n == len(raw)
            assert out[:n].cpu().numpy().tobytes() == ref
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    from paper_1905_07224_gb300 import pgz as P
    raw = synth.fastq(5 << 20, 150, 0.001, 23)
    gz = synth.gzip_compress(raw, 1)
    d = to_device(gz)
    out = empty(len(raw) + 4096)
    st, n = P.pgz_decompress_noalloc(d.data_ptr(), len(gz), out.data_ptr(), len(raw) + 4096, None)
    torch.cuda.synchronize()
    assert st == P.PGZ_E_ARG and n == 0


def _noalloc(P, gz: bytes, cap: int):
    import torch
    d = to_device(gz)
    out = empty(cap)
    out.fill_(0xAB)
    torch.cuda.synchronize()
    st, n = P.pgz_decompress_noalloc(d.data_ptr(), len(gz), out.data_ptr(), cap, None)
    torch.cuda.synchronize()
    return st, out[:n].cpu().numpy().tobytes() if st == 0 else b""


def test_noalloc_recovers_like_decompress():
    """The recovery paths inside the fixed scratch: a member whose stored block hides a chain of blocks that
    passes the block checks but fails its confirmation (a part's search must go on past it), and a member
    whose last quarter is one repeated byte (its part overflows its share of the symbol array, so the plan
    is redone with fewer parts).  Output equal to pgz_decompress and to the generator's bytes."""
    import confirm_streams as cs
    m = cs.find("invalid", 2)
    mixed = synth.markov(3 << 20, 24) + b"A" * (1 << 20)
    cases = [(m.gz, m.data), (synth.gzip_compress(mixed, 6), mixed)]
    ctx = Ctx(n_chunks=0, chunk_bytes=32768)
    try:
        P = ctx.pgz
        for gz, raw in cases:
            st, ref, _, _ = ctx.decompress(gz, out_cap=len(raw) + 4096)
            assert st == 0 and ref == raw
            for _ in range(2):
                st, got = _noalloc(P, gz, len(raw) + 4096)
                assert st == 0, P.pgz_strerror(st)
                assert got == ref
    finally:
        ctx.close()


def test_noalloc_allocates_no_device_memory():
    """After one warm call, further calls leave the device's free memory unchanged."""
    import torch
    from paper_1905_07224_gb300 import pgz as P
    raw = synth.fastq(2 << 20, 150, 0.001, 25)
    gz = synth.gzip_compress(raw, 6)
    d = to_device(gz)
    out = empty(len(raw) + 4096)
    torch.cuda.synchronize()
    st, n = P.pgz_decompress_noalloc(d.data_ptr(), len(gz), out.data_ptr(), len(raw) + 4096, None)
    torch.cuda.synchronize()
    assert st == 0 and n == len(raw)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        st, n = P.pgz_decompress_noalloc(d.data_ptr(), len(gz), out.data_ptr(), len(raw) + 4096, None)
        torch.cuda.synchronize()
        assert st == 0 and n == len(raw)
    assert torch.cuda.mem_get_info()[0] == free0
    assert out[:n].cpu().numpy().tobytes() == raw


_FIRST_CALL = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_1905_07224_gb300 import pgz, synth
raw = synth.fastq(1 << 20, 100, 0.001, 26)
gz = synth.gzip_compress(raw, 9)
d = torch.from_numpy(np.frombuffer(gz, dtype=np.uint8).copy()).cuda()
out = torch.zeros(len(raw) + 4096, dtype=torch.uint8, device="cuda")
torch.cuda.synchronize()
st, n = pgz.pgz_decompress_noalloc(d.data_ptr(), len(gz), out.data_ptr(), out.numel(), None)
torch.cuda.synchronize()
assert st == 0, pgz.pgz_strerror(st)
assert n == len(raw) and out[:n].cpu().numpy().tobytes() == raw
print("first call ok")
"""


def test_noalloc_as_the_first_call_of_a_process():
    """In a fresh process whose first library call is this entry point (no context created before), so that
    its own set-up runs: the output is exact."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "first call ok" in r.stdout
