"""gzip members built to test the confirmation of block starts (Section "Detection of DEFLATE block start
positions": once a block at a candidate bit decodes, the next five blocks must decode too, else the search
goes on from the bit after the candidate).

Each member is written block by block with the independent encoder in deflate_writer.py.  A stored block
of the member carries, as its payload, a *hidden* chain of DEFLATE blocks: their starts pass every block
check, but the chain breaks within the confirmation window, so none of them may be taken as a part start.
Two ways to break it:

  "invalid":  after the hidden blocks come the three header bits of a block of type 11 (reserved);
  "runaway":  the last hidden block uses a complete code over the allowed bytes and end-of-block only and
              has no end-of-block code of its own, so a decoder reads on, past the stored block's end, over
              the member's next true block start, until the first end-of-block codeword in the member's
              own bits; the block header read there has type 11.  This is checked by parsing the bits with
              that (known) code here, not with the oracle; seeds whose header there is not type 11 are
              skipped.

Everything a test expects is computed from the construction: the members' true block starts, which of
them pass the block checks and the confirmation (every literal of the start's block and of the five blocks
after it in the allowed set, a block of 1 KiB .. 4 MiB symbols, a non-final dynamic block), and the part
start that follows for each planned part: the least such start in its scan range.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import deflate_writer as dw
from paper_1905_07224_gb300 import synth

ALLOWED = frozenset([9, 10, 13] + list(range(32, 127)))
NONE = (1 << 64) - 1
HEADER_BYTES = 10


def literal_only_lengths():
    """Code lengths of a complete literal/length code over the 98 allowed bytes and end-of-block: 29 codes
    of 6 bits and 70 of 7 bits (29/64 + 70/128 = 1).  End-of-block gets one of the 7-bit codes."""
    syms = sorted(ALLOWED) + [256]
    llen = [0] * 257
    for k, s in enumerate(syms):
        llen[s] = 6 if k < 29 else 7
    return llen


@dataclass
class Block:
    bit: int            # absolute bit offset in the member of the block's first header bit
    kind: str           # "dynamic" or "stored"
    final: bool
    nsym: int           # symbols the block decodes to
    allowed: bool       # every literal of the block is an allowed byte


@dataclass
class Member:
    gz: bytes
    data: bytes
    blocks: list = field(default_factory=list)   # the member's true blocks, in order
    hidden: list = field(default_factory=list)   # absolute bit offsets of the hidden chain's block starts
    runaway_end: int | None = None               # "runaway": bit where the last hidden block ends

    @property
    def s0(self) -> int:
        return HEADER_BYTES

    @property
    def end_bit(self) -> int:
        return (len(self.gz) - 8) * 8

    def accepted_starts(self, confirm_blocks: int = 5, min_block: int = 1024, max_block: int = 4 << 20):
        """True block starts that pass the block checks and the confirmation, from the construction."""
        out = []
        for m, b in enumerate(self.blocks):
            if b.kind != "dynamic" or b.final or not (min_block <= b.nsym < max_block):
                continue
            window = []
            for x in self.blocks[m:m + confirm_blocks + 1]:
                window.append(x)
                if x.final:
                    break
            if all(x.allowed for x in window):
                out.append(b.bit)
        return out

    def nominal(self, nparts: int):
        """Scan ranges [lo_i, hi_i) of n parts of equal compressed size."""
        csize = len(self.gz) - 8 - self.s0
        per = (csize + nparts - 1) // nparts
        return [((self.s0 + i * per) * 8, min((self.s0 + (i + 1) * per) * 8, self.end_bit)) for i in range(nparts)]

    def expected_part_starts(self, nparts: int, confirm_blocks: int = 5):
        """Part starts from the construction: part 0 at the member start; part i the least accepted true
        block start in its scan range, or none (every hidden start fails its confirmation)."""
        acc = self.accepted_starts(confirm_blocks)
        out = []
        for i, (lo, hi) in enumerate(self.nominal(nparts)):
            if i == 0:
                out.append(self.s0 * 8)
                continue
            c = [t for t in acc if lo <= t < hi] if lo < self.end_bit else []
            out.append(min(c) if c else NONE)
        return out


def _bits_of(gz: bytes, start: int):
    """The member's bits from `start` on, one at a time (RFC 1951 3.1.1: LSB first in each byte)."""
    for p in range(start, len(gz) * 8):
        yield (gz[p >> 3] >> (p & 7)) & 1


def _runaway_end(gz: bytes, start: int, llen) -> int:
    """Where a block coded with the literal-only code ends when decoding starts at `start` (the first bit
    after its header): the bit after the first end-of-block codeword (codes MSB first, RFC 1951 3.2.2)."""
    codes = dw.canonical(llen)
    table = {(llen[s], codes[s]): s for s in range(len(llen)) if llen[s]}
    code, n, p = 0, 0, start
    for bit in _bits_of(gz, start):
        code, n, p = (code << 1) | bit, n + 1, p + 1
        s = table.get((n, code))
        if s is not None:
            if s == 256:
                return p
            code, n = 0, 0
        assert n <= 7
    raise AssertionError("no end-of-block")


def build(tail: str, hidden_blocks: int = 2, seed: int = 0, pad: int = 4000, head_bytes: int = 60000,
          after=(15000, 15000, 15000, 20000)) -> Member:
    """A member: a dynamic block of FASTQ text, a stored block whose payload is `pad` zero bytes followed by
    the hidden chain (hidden_blocks dynamic blocks of 2000 bytes of text, then the tail), then dynamic
    blocks of text of the sizes in `after`, the last one final."""
    text = synth.fastq(head_bytes + sum(after), 100, 0.001, 300 + seed)
    fake = synth.fastq(2000 * hidden_blocks + 3000, 100, 0.001, 400 + seed)
    hw = dw.BitWriter()
    hidden_rel = []
    for k in range(hidden_blocks):
        hidden_rel.append(hw.nbits)
        dw.write_dynamic(hw, dw.tokens_from_text(fake[2000 * k:2000 * (k + 1)]), False)
    lit = literal_only_lengths()
    runaway_rel = None
    if tail == "invalid":
        hw.put(0, 1)
        hw.put(3, 2)                                  # BTYPE = 11
    elif tail == "runaway":
        hidden_rel.append(hw.nbits)
        chars = [c for c in fake[2000 * hidden_blocks:] if c in ALLOWED][:1100]
        dw.write_dynamic(hw, [("lit", c) for c in chars], False, llen=lit, dlen=[1] + [0] * 29, eob=False)
        runaway_rel = hw.nbits
    else:
        raise ValueError(tail)
    payload = b"\x00" * pad + hw.tobytes()
    w = dw.BitWriter()
    blocks = []

    def put(kind, content, final, writer):
        blocks.append(Block(HEADER_BYTES * 8 + w.nbits, kind, final, len(content),
                            all(c in ALLOWED for c in content)))
        writer()

    put("dynamic", text[:head_bytes], False, lambda: dw.write_dynamic(w, dw.tokens_from_text(text[:head_bytes]), False))
    stored_bit = w.nbits
    put("stored", payload, False, lambda: dw.write_stored(w, payload, False))
    pos = head_bytes
    for k, n in enumerate(after):
        chunk = text[pos:pos + n]
        last = k == len(after) - 1
        put("dynamic", chunk, last, lambda c=chunk, f=last: dw.write_dynamic(w, dw.tokens_from_text(c), f))
        pos += n
    data = text[:head_bytes] + payload + text[head_bytes:]
    gz = dw.gzip_wrap(w.tobytes(), data)
    pay0 = HEADER_BYTES * 8 + ((stored_bit + 3 + 7) // 8) * 8 + 32      # first payload bit
    m = Member(gz, data, blocks, [pay0 + pad * 8 + r for r in hidden_rel])
    if runaway_rel is not None:
        # the runaway block's literals end on a codeword boundary at runaway_rel; decoding goes on from there
        m.runaway_end = _runaway_end(gz, pay0 + pad * 8 + runaway_rel, lit)
    return m


def header_type_at(gz: bytes, bit: int) -> int:
    """BTYPE of a block header at `bit`."""
    b = list(_bits_of(gz, bit))[:3]
    return b[1] | (b[2] << 1)


def find(tail: str, hidden_blocks: int = 2, **kw) -> Member:
    """The first seed whose member breaks its hidden chain as intended (for "runaway": the header where the
    runaway block ends has type 11, and that end lies past the stored block, over the next true start)."""
    for seed in range(64):
        m = build(tail, hidden_blocks, seed, **kw)
        if tail == "invalid":
            return m
        t = m.blocks[2].bit                       # the first true block after the stored block
        if m.runaway_end > t and header_type_at(m.gz, m.runaway_end) == 3:
            return m
    raise AssertionError("no seed gives the construction")
