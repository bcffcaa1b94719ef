"""The recovery step the library runs after a pass-1 run of one member (host logic; no GPU needed).

pgz_recover_step runs the library's own recovery on a hand-made description of a member's parts, so each
rule of Section "Detection of DEFLATE block start positions" and Section "Full file decompression in two
passes" is checked on its own, with the expected plan written from the rule:

- a searched start whose block or one of the five blocks after it fails the checks is dropped, and the
  search goes on from the bit after it; the window of a part that ends exactly on the next part's start
  continues with that part's checked blocks;
- a part that does not end exactly on the next part's start shows that start to be false: the next part is
  merged into it when its own confirmation passed, decoded past its stop first when the run left it open,
  searched on from the bit after it when it ends a streamed segment;
- a part whose symbols overflowed is given more capacity;
- an error at the member start, at a known start or in data after the final block is final.

Starts dropped through their confirmation are not counted as false starts (the oracle's two_pass counts
only starts that the previous part does not land on); merged and re-searched segment ends are.
"""
import pytest

S0 = 80                      # the member's first DEFLATE bit
NONE = (1 << 64) - 1


@pytest.fixture(scope="module")
def P():
    from paper_1905_07224_gb300 import build
    build.build()
    from paper_1905_07224_gb300 import pgz
    return pgz


def done(lo, sync, end, blocks, confirmed=1, **kw):
    return dict(lo=lo, sync=sync, end=end, blocks=blocks, confirmed=confirmed, state=3, **kw)


def failed(lo, sync, end, blocks, err, confirmed=0, **kw):
    return dict(lo=lo, sync=sync, end=end, blocks=blocks, confirmed=confirmed, state=4, err=err, **kw)


def plan_of(parts):
    return [(p["lo"], p.get("disabled", 0), p.get("confirm_ext", 0)) for p in parts]


def step(P, parts, **kw):
    a, out, fs, g = P.pgz_recover_step(parts, S0, **kw)
    return a, [(p["lo"], p["disabled"], p["confirm_ext"]) for p in out], fs, g


def test_a_clean_run_stops_with_the_plan_unchanged(P):
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 2000, 7), done(1900, 2000, 3000, 8)]
    assert step(P, parts) == (P.PGZ_RECOVER_STOP, plan_of(parts), 0, -1)


def test_a_start_whose_own_window_fails_is_searched_on_from_the_next_bit(P):
    # part 2 decoded two blocks, the third failed: position 3 of its window of 6
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 2000, 7), failed(1900, 2000, 2600, 2, P.PGZ_PART_CONFIRM)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 0 and g == -1
    assert plan == [(S0, 0, 0), (900, 0, 0), (2001, 0, 0)]


def test_the_window_continues_into_the_next_part_and_fails_there(P):
    # part 1 ended exactly on part 2's start after two blocks (window not complete); part 2 passed one block
    # and failed its second: part 1's window fails at its 4th block, part 2's at its 2nd
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 2000, 2, confirmed=0),
             failed(1900, 2000, 2500, 1, P.PGZ_PART_CONFIRM)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 0
    assert plan == [(S0, 0, 0), (1001, 0, 0), (2001, 0, 0)]


def test_a_failure_past_the_window_does_not_reject_the_previous_start(P):
    # part 2 failed at its 5th block: for part 1 (two blocks of its own) that is block 7, past the window
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 2000, 2, confirmed=0),
             failed(1900, 2000, 2900, 4, P.PGZ_PART_CONFIRM)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 0
    assert plan == [(S0, 0, 0), (900, 0, 0), (2001, 0, 0)]


def test_the_window_skips_parts_with_no_start(P):
    # part 2 found no start; part 1 ended on part 3's start, whose first block passed and second failed
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 3000, 3, confirmed=0), dict(lo=1900, state=2),
             failed(2900, 3000, 3300, 1, P.PGZ_PART_CONFIRM)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 0
    assert plan == [(S0, 0, 0), (1001, 0, 0), (1900, 0, 0), (3001, 0, 0)]


def test_a_false_start_whose_confirmation_passed_is_merged(P):
    # part 1 did not land on part 2's start; part 2's own window passed: part 2 has no start in its range
    parts = [done(S0, S0, 1000, 9), failed(900, 1000, 2050, 8, P.PGZ_PART_CHAIN, confirmed=1),
             done(1900, 2000, 3000, 8)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 1 and g == -1
    assert plan == [(S0, 0, 0), (900, 0, 0), (1900, 1, 0)]


def test_an_open_confirmation_is_settled_by_decoding_past_the_stop_first(P):
    # part 2 stopped at part 3's start after two blocks, but part 3 started elsewhere (2990): its window is open
    parts = [done(S0, S0, 1000, 9), failed(900, 1000, 2050, 8, P.PGZ_PART_CHAIN, confirmed=1),
             done(1900, 2000, 2980, 2, confirmed=0), done(2900, 2990, 4000, 8)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 0
    assert plan == [(S0, 0, 0), (900, 0, 0), (1900, 0, 1), (2900, 0, 0)]
    # the same once part 2 has already decoded past its stop: merged
    parts[2]["confirm_ext"] = 1
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 1
    assert plan == [(S0, 0, 0), (900, 0, 0), (1900, 1, 1), (2900, 0, 0)]


def test_a_false_start_at_a_segment_end_is_searched_on_from_the_next_bit(P):
    parts = [done(S0, S0, 1000, 9), failed(900, 1000, 2050, 8, P.PGZ_PART_CHAIN, confirmed=1),
             dict(lo=1900, sync=2000, end=2000, state=3, probe=1)]
    a, plan, fs, g = step(P, parts, mode=3, last_seg=0)
    assert a == P.PGZ_RECOVER_RERUN and fs == 1
    assert plan == [(S0, 0, 0), (900, 0, 0), (2001, 0, 0)]


def test_overflow_asks_for_capacity(P):
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 2000, 7), failed(1900, 2000, 2400, 3, P.PGZ_PART_OVERFLOW),
             done(2900, 3000, 4000, 7)]
    assert step(P, parts)[0::3] == (P.PGZ_RECOVER_GROW, 2)
    # also when the overflowed part is the one a chain failure points at
    parts = [done(S0, S0, 1000, 9), failed(900, 1000, 2050, 8, P.PGZ_PART_CHAIN, confirmed=1),
             failed(1900, 2000, 2100, 1, P.PGZ_PART_OVERFLOW)]
    assert step(P, parts)[0::3] == (P.PGZ_RECOVER_GROW, 2)


def test_errors_that_are_final(P):
    # data after the member's final block
    parts = [done(S0, S0, 1000, 9), failed(900, 1000, 2000, 3, P.PGZ_PART_TRAIL, confirmed=1)]
    assert step(P, parts) == (P.PGZ_RECOVER_STOP, plan_of(parts), 0, -1)
    # invalid data at the member start
    parts = [failed(S0, S0, 500, 1, P.PGZ_PART_DATA), done(900, 1000, 2000, 7)]
    assert step(P, parts) == (P.PGZ_RECOVER_STOP, plan_of(parts), 0, -1)
    # invalid data after a known block start
    parts = [done(S0, S0, 1000, 9), failed(1000, 1000, 1500, 1, P.PGZ_PART_DATA, given=1)]
    assert step(P, parts) == (P.PGZ_RECOVER_STOP, plan_of(parts), 0, -1)
    # a streamed segment whose last part found no start: only a longer look-ahead helps
    parts = [done(S0, S0, 1000, 9), dict(lo=900, state=2)]
    assert step(P, parts, mode=3, last_seg=0) == (P.PGZ_RECOVER_STOP, plan_of(parts), 0, -1)


def test_a_searched_start_failing_past_its_window_is_merged(P):
    # part 2's window passed, then its decoding hit invalid data: its start is false, part 1 decodes on
    parts = [done(S0, S0, 1000, 9), done(900, 1000, 2000, 7), failed(1900, 2000, 2800, 8, P.PGZ_PART_DATA,
                                                                     confirmed=1)]
    a, plan, fs, g = step(P, parts)
    assert a == P.PGZ_RECOVER_RERUN and fs == 1
    assert plan == [(S0, 0, 0), (900, 0, 0), (1900, 1, 0)]


def test_without_confirmation_blocks_a_failed_start_is_still_searched_on(P):
    parts = [done(S0, S0, 1000, 9), failed(900, 1000, 1200, 0, P.PGZ_PART_CONFIRM)]
    a, plan, fs, g = step(P, parts, confirm_blocks=0)
    assert a == P.PGZ_RECOVER_RERUN and fs == 0
    assert plan == [(S0, 0, 0), (1001, 0, 0)]


def test_bad_arguments(P):
    import ctypes
    fs, g = ctypes.c_uint64(0), ctypes.c_int(0)
    arr = (P.pgz_part_state * 1)()
    L = P.lib()
    assert L.pgz_recover_step(0, arr, S0, 0, 1, 5, ctypes.byref(fs), ctypes.byref(g)) == -1
    assert L.pgz_recover_step(1, None, S0, 0, 1, 5, ctypes.byref(fs), ctypes.byref(g)) == -1
    assert L.pgz_recover_step(1, arr, S0, 0, 1, -1, ctypes.byref(fs), ctypes.byref(g)) == -1
    assert L.pgz_recover_step(1, arr, S0, 7, 1, 5, ctypes.byref(fs), ctypes.byref(g)) == -1
