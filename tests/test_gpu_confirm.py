"""The confirmation of block starts on the GPU (Section "Detection of DEFLATE block start positions").

The members of confirm_streams.py hide chains of blocks inside a stored block: their starts pass every
block check, but each chain breaks within the five-block confirmation window.  The GPU's part starts must
be those the construction gives (the least accepted true block start in each part's scan range), as the
oracle's are.  Part counts are swept so that a failed confirmation is seen both inside one part and
across part ends (a part that ends on the next part's start before its window is complete takes the rest
of the window from that part's blocks, or decodes past its end to finish it).
"""
import numpy as np
import pytest

import oracle
import confirm_streams as cs
from gpu_util import Ctx, to_device, empty

pytestmark = pytest.mark.gpu

CASES = [("invalid", 2), ("invalid", 4), ("runaway", 1), ("runaway", 3)]


@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("tail,hidden", CASES)
def test_part_starts_follow_the_construction(tail, hidden, pipe):
    m = cs.find(tail, hidden)
    retried = 0
    for n in range(2, 301, 3):
        ref = oracle.two_pass(m.gz, n)
        want = np.array(m.expected_part_starts(n), dtype=np.uint64)
        assert np.array_equal(ref["part_bits"].astype(np.uint64), want)
        ctx = Ctx(n_chunks=n, exec_pipelined=pipe)
        try:
            st, out, _, s = ctx.decompress(m.gz, stats=True)
            assert st == 0, (n, ctx.pgz.pgz_strerror(st))
            assert out == m.data, n
            sb, ns, nph = ctx.pgz.pgz_inspect_parts(ctx.h)
            assert np.array_equal(sb, want), (n, [(i, int(a), int(b)) for i, (a, b) in enumerate(zip(sb, want)) if a != b])
            assert np.array_equal(ns, ref["part_len"]) and np.array_equal(nph, ref["part_nph"]), n
            assert s["false_syncs"] == ref["false_syncs"] == 0, n
            retried += s["retries"] > 0
        finally:
            ctx.close()
    assert retried > 20


def test_decompress_at_skips_a_failed_start():
    """Problem 1 from a bit before a hidden chain: the decode starts at the first accepted true start."""
    m = cs.find("runaway", 1)
    t = min(a for a in m.accepted_starts() if a > m.hidden[-1])
    ctx = Ctx()
    try:
        import torch
        d = to_device(m.gz)
        cap = 4 * len(m.data)
        sym = torch.zeros(cap, dtype=torch.int16, device="cuda")
        byt = empty(cap)
        for start in (m.hidden[0] - 40, m.hidden[0]):
            st, n, bb, fd = ctx.pgz.pgz_decompress_at(ctx.h, d.data_ptr(), len(m.gz), start, sym.data_ptr(),
                                                       byt.data_ptr(), ord("?"), cap)
            assert st == 0, ctx.pgz.pgz_strerror(st)
            assert bb == t
            r = oracle.decompress_at(m.gz, start, cap=cap)
            assert r["status"] == 0 and r["block_bit"] == t and n == len(r["sym"])
            assert np.array_equal(sym[:n].cpu().numpy().view(np.uint16), r["sym"])
    finally:
        ctx.close()
