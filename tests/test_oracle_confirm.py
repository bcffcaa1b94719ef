"""Pins of the oracle's block-start confirmation (Section "Detection of DEFLATE block start positions").

A block start is taken only if its block and the five blocks after it decode; if not, the search goes on
from the bit after that start.  The members come from confirm_streams.py: a stored block hides chains of
blocks whose starts pass every block check but break within the confirmation window.  Every expected value
is computed from the construction (the members' true blocks and which of them pass), not from the oracle.
An oracle whose confirmation never rejected, or that resumed the search at the end of the failed start's
first block, fails these tests.
"""
import numpy as np
import pytest

import oracle
import confirm_streams as cs

CASES = [("invalid", 2), ("invalid", 4), ("runaway", 1), ("runaway", 3)]


@pytest.fixture(scope="module", params=CASES, ids=[f"{t}-{h}" for t, h in CASES])
def member(request):
    oracle.build()
    tail, hidden = request.param
    return cs.find(tail, hidden)


def test_member_decodes(member):
    e, out, _, _ = oracle.gunzip(member.gz)
    assert e == 0 and out == member.data


def test_hidden_starts_pass_the_block_checks_but_not_the_confirmation(member):
    al = oracle.default_allowed()
    for h in member.hidden:
        ok, why = oracle.block_ok(member.gz, member.end_bit, h, al)
        assert ok and why == 0
        assert not oracle.confirm(member.gz, member.end_bit, h, al, blocks=5)


def test_the_failing_block_position_decides():
    """The "invalid" chain H_1 .. H_k is followed by a block of type 11, the (k - j + 2)-th block from H_j.
    A window that ends before it accepts H_j; one that reaches it rejects H_j."""
    m = cs.find("invalid", 4)
    al = oracle.default_allowed()
    k = len(m.hidden)
    for j, h in enumerate(m.hidden, start=1):
        fail_at = k - j + 2                       # 1-based position of the type-11 block from H_j
        assert oracle.confirm(m.gz, m.end_bit, h, al, blocks=fail_at - 2)
        assert not oracle.confirm(m.gz, m.end_bit, h, al, blocks=fail_at - 1)


def test_true_starts_follow_the_construction(member):
    """Each true block start is accepted exactly when the construction says so: the first block (its window
    reaches the stored block of zero bytes) and the final block are not."""
    al = oracle.default_allowed()
    acc = set(member.accepted_starts())
    for b in member.blocks:
        ok = oracle.block_ok(member.gz, member.end_bit, b.bit, al)[0] and \
            oracle.confirm(member.gz, member.end_bit, b.bit, al, blocks=5)
        assert ok == (b.bit in acc), b
    assert len(acc) == 3


def test_search_resumes_after_the_failed_start(member):
    """From anywhere before the hidden chain, the least accepted bit is the first accepted true start after
    it.  For the "runaway" chain that start lies inside the first block of the failed start, so resuming at
    the end of that block (the other reading of the passage) would give the next one instead."""
    al = oracle.default_allowed()
    acc = member.accepted_starts()
    t = min(a for a in acc if a > member.hidden[-1])
    for lo in (member.hidden[0] - 8 * 100, member.hidden[0] - 3, member.hidden[0]):
        assert oracle.sync_scan(member.gz, member.end_bit, lo, member.end_bit, al, confirm_blocks=5) == t
    # without the confirmation the hidden start is taken
    assert oracle.sync_scan(member.gz, member.end_bit, member.hidden[0] - 3, member.end_bit, al) == member.hidden[0]
    if member.runaway_end is not None:
        assert member.hidden[-1] < t < member.runaway_end
        after = min(a for a in acc if a >= member.runaway_end)
        assert after != t


@pytest.mark.parametrize("tail,hidden", CASES)
def test_two_passes_take_the_constructed_part_starts(tail, hidden):
    """Part counts from 2 to 300 (every third): the oracle's part starts are the construction's, the output is exact,
    and no start is merged (every hidden start fails its confirmation before the chain check sees it)."""
    m = cs.find(tail, hidden)
    covered = 0
    for n in range(2, 301, 3):
        r = oracle.two_pass(m.gz, n)
        assert r["status"] == 0 and r["out"] == m.data, n
        want = np.array(m.expected_part_starts(n), dtype=np.uint64)
        assert np.array_equal(r["part_bits"].astype(np.uint64), want), n
        assert r["false_syncs"] == 0, n
        covered += any(lo <= m.hidden[0] < hi for lo, hi in m.nominal(n)[1:])
    assert covered > 40
