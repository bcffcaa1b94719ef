"""pgz_decompress_noalloc: the entry point for callers that cannot allocate.

Some callers cannot let a library allocate device memory (their own allocator
owns the GPU, a fixed memory budget, or no cudaFree synchronisation allowed in
their loop).  This entry point keeps all scratch in a fixed device array; this
test calls it through the C ABI twice in a row, on different inputs and on the
same input again, and requires byte-identical output to pgz_decompress (the
path is integer-exact, so the tolerance is zero), plus the size limit error.
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
