/*
 * oracle.c -- the CPU oracle for the two-pass parallel gzip decompression of
 * Kerbiriou & Chikhi, "Parallel decompression of gzip-compressed files and
 * random access to DNA sequences" (arXiv 1905.07224).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Plain, slow, single-threaded and deliberately literal:
 *  - bits are read one at a time (RFC 1951 section 3.1.1, LSB first);
 *  - Huffman codes are decoded one bit at a time against the canonical code
 *    definition (RFC 1951 section 3.2.2), no lookup tables;
 *  - the length and distance base tables are generated from their rule
 *    (RFC 1951 section 3.2.5);
 *  - CRC-32 is computed one bit at a time from the reflected polynomial
 *    0xEDB88320 (RFC 1952 section 8), and combined with polynomial
 *    arithmetic modulo P(x) in GF(2).
 *
 * What the paper fixes and where:
 *  - decompress(C, w): Algorithm "DEFLATE decompression" (Section "DEFLATE
 *    algorithm"): literals are appended to the context, matches copy from it.
 *  - undetermined / symbolic context: Section "Undetermined context
 *    propagation technique" and Section "Full file decompression in two
 *    passes (pugz)": the initial context of a part is [U_0 .. U_32767];
 *    back-references into it propagate the symbols U_j.
 *  - block start detection: Section "Detection of DEFLATE block start
 *    positions" and Appendix "DEFLATE block decompression checks".
 *  - two passes: Section "Full file decompression in two passes (pugz)":
 *    pass 1 decodes every part with a symbolic context; pass 2 resolves the
 *    windows w_i sequentially, then translates U_j -> w_i[j] in every part.
 *  - CRC-32 / ISIZE are not computed by the paper's implementation (Section
 *    "Discussion"); they follow RFC 1952.
 *
 * Readings of points the paper leaves open are listed next to the code that
 * takes them (look for "Reading").
 *
 * Symbol encoding of a symbolic stream: a value < 0x100 is a byte; 0x8000|j
 * is the placeholder U_j (0 <= j < 32768) of the part's initial context.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    ORC_OK = 0,
    ORC_E_ARG = -1,
    ORC_E_HEADER = -2,
    ORC_E_DATA = -3,       /* invalid DEFLATE content */
    ORC_E_TRUNC = -4,      /* a read went past the end of the compressed data */
    ORC_E_CRC = -5,
    ORC_E_ISIZE = -6,
    ORC_E_CAPACITY = -7,
    ORC_E_DIST = -8,       /* distance beyond the known (empty) context */
    ORC_E_BYTE = -9,       /* literal outside the allowed byte set */
    ORC_E_SIZE = -10,      /* block output outside [min_out, max_out) */
    ORC_E_FINAL = -11,     /* predicate: BFINAL set */
    ORC_E_TYPE = -12,      /* predicate: not a dynamic block; or BTYPE 11 */
    ORC_E_NOSYNC = -13,
    ORC_E_NOMEM = -14,
    ORC_E_UNSUPPORTED = -15,
    ORC_E_CHAIN = -16      /* a part did not end on the next part's start */
};

#define WSIZE 32768u
#define PH 0x8000u

/* ------------------------------------------------------------------ */
/* bit reader: RFC 1951 3.1.1, data elements packed LSB first          */
/* ------------------------------------------------------------------ */
typedef struct {
    const uint8_t* p;
    uint64_t end;      /* bit index one past the last readable bit */
    uint64_t pos;      /* next bit to read */
    int overrun;
} rd_t;

static uint32_t rd_bit(rd_t* r) {
    if (r->pos >= r->end) { r->overrun = 1; r->pos++; return 0; }
    uint32_t b = (r->p[r->pos >> 3] >> (r->pos & 7)) & 1u;
    r->pos++;
    return b;
}

/* an n-bit integer, least significant bit first */
static uint32_t rd_bits(rd_t* r, int n) {
    uint32_t v = 0;
    for (int i = 0; i < n; i++) v |= rd_bit(r) << i;
    return v;
}

/* ------------------------------------------------------------------ */
/* canonical Huffman codes: RFC 1951 3.2.2                             */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t count[16];    /* number of codes of each length */
    uint32_t first[16];    /* numerically smallest code of each length */
    uint32_t offset[16];   /* index in sym[] of the first symbol of each length */
    uint16_t sym[320];     /* symbols ordered by (code length, symbol value) */
    int ncodes;
    int maxlen;
} huff_t;

/* returns 0 for a complete code, 1 for an incomplete one, -1 if over-subscribed */
static int huff_build(huff_t* h, const uint8_t* len, int n) {
    memset(h, 0, sizeof *h);
    for (int i = 0; i < n; i++) h->count[len[i]]++;
    h->count[0] = 0;
    int64_t left = 1;                        /* Kraft: unused codes at each length */
    for (int L = 1; L <= 15; L++) {
        left = 2 * left - (int64_t)h->count[L];
        if (left < 0) return -1;
        if (h->count[L]) h->maxlen = L;
        h->ncodes += (int)h->count[L];
    }
    uint32_t code = 0;                       /* RFC 1951 3.2.2, step 2 */
    for (int L = 1; L <= 15; L++) {
        code = (code + h->count[L - 1]) << 1;
        h->first[L] = code;
    }
    uint32_t off = 0;
    for (int L = 1; L <= 15; L++) { h->offset[L] = off; off += h->count[L]; }
    uint32_t next[16];
    memcpy(next, h->offset, sizeof next);
    for (int i = 0; i < n; i++)              /* RFC 1951 3.2.2, step 3: codes in symbol order */
        if (len[i]) h->sym[next[len[i]]++] = (uint16_t)i;
    return left > 0 ? 1 : 0;
}

/* read a code MSB first, one bit at a time; -1 if no code matches */
static int huff_decode(rd_t* r, const huff_t* h) {
    uint32_t v = 0;
    for (int L = 1; L <= 15; L++) {
        v = (v << 1) | rd_bit(r);
        if (h->count[L] && v >= h->first[L] && v - h->first[L] < h->count[L])
            return h->sym[h->offset[L] + (v - h->first[L])];
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* length and distance codes: RFC 1951 3.2.5, generated from the rule  */
/* ------------------------------------------------------------------ */
static uint16_t len_base[29], dist_base[30];
static uint8_t len_extra[29], dist_extra[30];
static int tables_ready = 0;
static huff_t fixed_lit, fixed_dist;

static void init_tables(void) {
    if (tables_ready) return;
    /* length codes 257..284: four codes per extra-bit count from 1 upward,
       after eight codes with none; 285 is the single length 258 */
    uint32_t base = 3;
    for (int k = 0; k < 28; k++) {
        len_extra[k] = (uint8_t)(k < 8 ? 0 : k / 4 - 1);
        len_base[k] = (uint16_t)base;
        base += 1u << len_extra[k];
    }
    len_base[28] = 258;
    len_extra[28] = 0;
    /* distance codes 0..29: two codes per extra-bit count from 1 upward,
       after four codes with none */
    base = 1;
    for (int k = 0; k < 30; k++) {
        dist_extra[k] = (uint8_t)(k < 4 ? 0 : k / 2 - 1);
        dist_base[k] = (uint16_t)base;
        base += 1u << dist_extra[k];
    }
    /* the fixed code, RFC 1951 3.2.6 */
    uint8_t l[288];
    for (int i = 0; i < 288; i++) l[i] = (uint8_t)(i < 144 ? 8 : i < 256 ? 9 : i < 280 ? 7 : 8);
    huff_build(&fixed_lit, l, 288);
    for (int i = 0; i < 32; i++) l[i] = 5;
    huff_build(&fixed_dist, l, 32);
    tables_ready = 1;
}

/* ------------------------------------------------------------------ */
/* CRC-32: RFC 1952 section 8, one bit at a time                       */
/* ------------------------------------------------------------------ */
#define CRC_POLY 0xEDB88320u   /* x^32+x^26+...+1, bit-reversed, x^32 dropped */

/* `crc` is a finished CRC of the preceding bytes (0 for none), as zlib's crc32() */
uint32_t orc_crc32(uint32_t crc, const uint8_t* p, uint64_t n) {
    uint32_t c = ~crc;
    for (uint64_t i = 0; i < n; i++) {
        c ^= p[i];
        for (int k = 0; k < 8; k++) c = (c & 1u) ? (c >> 1) ^ CRC_POLY : (c >> 1);
    }
    return ~c;
}

/* a*b mod P(x).  Reflected representation: bit 31-k holds the coefficient of x^k. */
static uint32_t gf2_mulmod(uint32_t a, uint32_t b) {
    uint32_t prod = 0;
    for (int k = 0; k < 32; k++) {           /* b holds b(x) * x^k mod P */
        if (a & (0x80000000u >> k)) prod ^= b;
        b = (b & 1u) ? (b >> 1) ^ CRC_POLY : (b >> 1);   /* multiply by x */
    }
    return prod;
}

/* x^e mod P by square-and-multiply */
static uint32_t gf2_xpow(uint64_t e) {
    uint32_t result = 0x80000000u;           /* 1 */
    uint32_t sq = 0x40000000u;               /* x */
    while (e) {
        if (e & 1) result = gf2_mulmod(result, sq);
        sq = gf2_mulmod(sq, sq);
        e >>= 1;
    }
    return result;
}

/* CRC of A||B from crc(A), crc(B) and |B|.  The CRC register is linear in
   (initial register, message): advancing crc(A) over |B| zero bytes is a
   multiplication by x^(8|B|) mod P, and adding crc(B) supplies B's own
   contribution; the initial-register and final-inversion terms of B's CRC
   cancel those carried over from A. */
uint32_t orc_crc32_combine(uint32_t crc_a, uint32_t crc_b, uint64_t len_b) {
    uint32_t shift = gf2_xpow(8 * len_b);
    return gf2_mulmod(crc_a, shift) ^ crc_b;
}

/* ------------------------------------------------------------------ */
/* gzip container: RFC 1952 section 2.3                                */
/* ------------------------------------------------------------------ */
/* returns the offset of the DEFLATE data or a negative error */
int64_t orc_gzip_header(const uint8_t* gz, uint64_t len) {
    if (len < 18) return ORC_E_HEADER;
    if (gz[0] != 0x1f || gz[1] != 0x8b || gz[2] != 8) return ORC_E_HEADER;
    uint8_t flg = gz[3];
    if (flg & 0xe0) return ORC_E_HEADER;     /* reserved flag bits */
    uint64_t pos = 10;
    if (flg & 4) {                           /* FEXTRA */
        if (pos + 2 > len) return ORC_E_HEADER;
        uint64_t xlen = gz[pos] | ((uint64_t)gz[pos + 1] << 8);
        pos += 2 + xlen;
        if (pos > len) return ORC_E_HEADER;
    }
    for (int f = 8; f <= 16; f <<= 1) {      /* FNAME, FCOMMENT: zero-terminated */
        if (flg & f) {
            while (pos < len && gz[pos] != 0) pos++;
            if (pos >= len) return ORC_E_HEADER;
            pos++;
        }
    }
    if (flg & 2) {                           /* FHCRC: low 16 bits of the header's CRC-32 */
        if (pos + 2 > len) return ORC_E_HEADER;
        uint32_t c = orc_crc32(0, gz, pos) & 0xffffu;
        if (c != (gz[pos] | ((uint32_t)gz[pos + 1] << 8))) return ORC_E_HEADER;
        pos += 2;
    }
    if (pos + 8 > len) return ORC_E_HEADER;
    return (int64_t)pos;
}

/* ------------------------------------------------------------------ */
/* decompress(C, w): Algorithm "DEFLATE decompression"                 */
/* ------------------------------------------------------------------ */
typedef struct {
    rd_t r;
    uint16_t* out16;       /* symbolic output (or NULL) */
    uint8_t* out8;         /* byte output (known context only) (or NULL) */
    uint64_t cap;          /* output capacity in symbols (ignored when counting only) */
    uint64_t n;            /* symbols produced so far in this call */
    uint64_t block_n;      /* symbols produced by the current block */
    uint64_t max_block;    /* stop (ORC_E_SIZE) once a block reaches this many symbols; 0 = none */
    int known;             /* 1: the context before the start is empty (stream start) */
    int count_only;        /* 1: do not store symbols (predicate, confirmation) */
    const uint8_t* allowed;/* 32-byte set of literal bytes to accept, when check_lits */
    int check_lits;
    uint64_t nph;          /* placeholder symbols produced (not when counting only) */
} dec_t;

static int allowed_has(const uint8_t* a, unsigned b) { return (a[b >> 3] >> (b & 7)) & 1; }

static int emit(dec_t* d, uint32_t s) {
    if (!d->count_only) {
        if (d->n >= d->cap) return ORC_E_CAPACITY;
        if (d->out16) d->out16[d->n] = (uint16_t)s;
        else d->out8[d->n] = (uint8_t)s;
    }
    if (s & PH) d->nph++;
    d->n++;
    d->block_n++;
    if (d->max_block && d->block_n >= d->max_block) return ORC_E_SIZE;
    return ORC_OK;
}

static int emit_literal(dec_t* d, uint32_t byte) {
    if (d->check_lits && !allowed_has(d->allowed, byte)) return ORC_E_BYTE;
    return emit(d, byte);
}

/* the symbol `dist` positions back from the next output position */
static uint32_t back_symbol(const dec_t* d, uint64_t dist) {
    if (dist <= d->n) return d->out16 ? d->out16[d->n - dist] : d->out8[d->n - dist];
    /* before the start: source position p = n - dist < 0 is U_{32768 + p} */
    return PH | (uint32_t)(WSIZE - (dist - d->n));
}

static int copy_match(dec_t* d, uint32_t len, uint32_t dist) {
    if (dist > WSIZE) return ORC_E_DATA;
    if (d->known && dist > d->n) return ORC_E_DIST;
    for (uint32_t k = 0; k < len; k++) {
        uint32_t s = d->count_only ? 0 : back_symbol(d, dist);   /* counting needs no values */
        int e = emit(d, s);
        if (e) return e;
    }
    return ORC_OK;
}

static int codes(dec_t* d, const huff_t* lit, const huff_t* dst) {
    for (;;) {
        int sym = huff_decode(&d->r, lit);
        if (d->r.overrun) return ORC_E_TRUNC;
        if (sym < 0) return ORC_E_DATA;
        if (sym < 256) {
            int e = emit_literal(d, (uint32_t)sym);
            if (e) return e;
        } else if (sym == 256) {
            return ORC_OK;
        } else {
            sym -= 257;
            if (sym >= 29) return ORC_E_DATA;          /* 286, 287 */
            uint32_t len = len_base[sym] + rd_bits(&d->r, len_extra[sym]);
            int ds = huff_decode(&d->r, dst);
            if (d->r.overrun) return ORC_E_TRUNC;
            if (ds < 0 || ds >= 30) return ORC_E_DATA;  /* no code, or 30, 31 */
            uint32_t dist = dist_base[ds] + rd_bits(&d->r, dist_extra[ds]);
            if (d->r.overrun) return ORC_E_TRUNC;
            int e = copy_match(d, len, dist);
            if (e) return e;
        }
    }
}

static int stored(dec_t* d) {
    d->r.pos = (d->r.pos + 7) & ~(uint64_t)7;          /* to a byte boundary */
    uint32_t len = rd_bits(&d->r, 16);
    uint32_t nlen = rd_bits(&d->r, 16);
    if (d->r.overrun) return ORC_E_TRUNC;
    if ((len ^ 0xffffu) != nlen) return ORC_E_DATA;
    for (uint32_t i = 0; i < len; i++) {
        uint32_t b = rd_bits(&d->r, 8);
        if (d->r.overrun) return ORC_E_TRUNC;
        int e = emit_literal(d, b);
        if (e) return e;
    }
    return ORC_OK;
}

/* Reading of "valid" codes (RFC 1951 3.2.7 and the behaviour of zlib, the
   producer): over-subscribed codes are invalid; the code-length code must be
   complete; the literal/length code must contain end-of-block and be
   complete, or consist of one code of length 1; the distance code must be
   complete, or consist of one code of length 1, or be empty (then no match
   may occur). */
static int dynamic_header(rd_t* r, huff_t* lit, huff_t* dst) {
    static const uint8_t order[19] = {16, 17, 18, 0, 8, 7, 9, 6, 10, 5, 11, 4, 12, 3, 13, 2, 14, 1, 15};
    int nlen = (int)rd_bits(r, 5) + 257;
    int ndist = (int)rd_bits(r, 5) + 1;
    int ncode = (int)rd_bits(r, 4) + 4;
    if (r->overrun) return ORC_E_TRUNC;
    if (nlen > 286 || ndist > 30) return ORC_E_DATA;
    uint8_t lengths[320];
    memset(lengths, 0, sizeof lengths);
    for (int i = 0; i < ncode; i++) lengths[order[i]] = (uint8_t)rd_bits(r, 3);
    if (r->overrun) return ORC_E_TRUNC;
    huff_t cl;
    if (huff_build(&cl, lengths, 19) != 0) return ORC_E_DATA;
    int total = nlen + ndist;
    int i = 0;
    memset(lengths, 0, sizeof lengths);
    while (i < total) {
        int sym = huff_decode(r, &cl);
        if (r->overrun) return ORC_E_TRUNC;
        if (sym < 0) return ORC_E_DATA;
        if (sym < 16) { lengths[i++] = (uint8_t)sym; continue; }
        uint8_t val = 0;
        int rep;
        if (sym == 16) {
            if (i == 0) return ORC_E_DATA;
            val = lengths[i - 1];
            rep = 3 + (int)rd_bits(r, 2);
        } else if (sym == 17) {
            rep = 3 + (int)rd_bits(r, 3);
        } else {
            rep = 11 + (int)rd_bits(r, 7);
        }
        if (r->overrun) return ORC_E_TRUNC;
        if (i + rep > total) return ORC_E_DATA;
        while (rep--) lengths[i++] = val;
    }
    if (lengths[256] == 0) return ORC_E_DATA;          /* no end-of-block code */
    int e = huff_build(lit, lengths, nlen);
    if (e < 0 || (e > 0 && !(lit->ncodes == 1 && lit->maxlen == 1))) return ORC_E_DATA;
    e = huff_build(dst, lengths + nlen, ndist);
    if (e < 0 || (e > 0 && !(dst->ncodes == 0 || (dst->ncodes == 1 && dst->maxlen == 1)))) return ORC_E_DATA;
    return ORC_OK;
}

/* one block; *final receives BFINAL */
static int block(dec_t* d, int* final) {
    huff_t lit, dst;
    *final = (int)rd_bit(&d->r);
    uint32_t type = rd_bits(&d->r, 2);
    if (d->r.overrun) return ORC_E_TRUNC;
    d->block_n = 0;
    if (type == 0) return stored(d);
    if (type == 1) return codes(d, &fixed_lit, &fixed_dist);
    if (type == 2) {
        int e = dynamic_header(&d->r, &lit, &dst);
        if (e) return e;
        return codes(d, &lit, &dst);
    }
    return ORC_E_DATA;                                 /* BTYPE 11 */
}

/* ------------------------------------------------------------------ */
/* exported: decode blocks from a bit offset                           */
/* ------------------------------------------------------------------ */
/*
 * Decode whole blocks from `start_bit` of `data` (bits [0, end_bit) readable).
 * Stops before a block whose start is >= stop_bit (stop_bit = 0: no such stop),
 * or after the block with BFINAL set.  known = 1: the context is empty (a
 * distance beyond the output is an error), else the symbolic context
 * [U_0 .. U_32767] precedes the start.  If `allowed` is given, literals of the
 * first `check_blocks` blocks must lie in it.  out16 receives symbols (may be
 * NULL with cap = 0 to count only).  Results: *out_len symbols, *pos_out the
 * bit position where decoding stopped, *final_out whether a final block was
 * decoded, *nblocks, *nph placeholder symbols.
 */
int orc_inflate_from(const uint8_t* data, uint64_t end_bit, uint64_t start_bit, uint64_t stop_bit,
                     int known, const uint8_t* allowed, int check_blocks,
                     uint16_t* out16, uint64_t cap, uint64_t* out_len, uint64_t* pos_out,
                     int* final_out, uint64_t* nblocks, uint64_t* nph) {
    init_tables();
    dec_t d;
    memset(&d, 0, sizeof d);
    d.r.p = data; d.r.end = end_bit; d.r.pos = start_bit;
    d.out16 = out16; d.cap = cap; d.count_only = (out16 == NULL);
    d.known = known; d.allowed = allowed;
    uint64_t nb = 0;
    int final = 0, e = ORC_OK;
    for (;;) {
        if (stop_bit && d.r.pos >= stop_bit) break;
        d.check_lits = (allowed != NULL) && (nb < (uint64_t)check_blocks);
        e = block(&d, &final);
        if (e) break;
        nb++;
        if (final) break;
    }
    if (out_len) *out_len = d.n;
    if (pos_out) *pos_out = d.r.pos;
    if (final_out) *final_out = final;
    if (nblocks) *nblocks = nb;
    if (nph) *nph = d.nph;
    return e;
}

/* ------------------------------------------------------------------ */
/* block start detection: Section "Detection of DEFLATE block start     */
/* positions" and Appendix "DEFLATE block decompression checks"        */
/* ------------------------------------------------------------------ */
/*
 * The predicate at bit `b`:
 *  - BFINAL = 0 (the last block is never a sync target);
 *  - BTYPE = 10.  Reading: only dynamic blocks are accepted as sync points
 *    (stored and fixed blocks are still decoded inside a part);
 *  - the dynamic header describes valid codes (see dynamic_header);
 *  - trial decode of the block with a symbolic context: every literal in the
 *    allowed byte set, every code valid, no read past the data;
 *  - Reading of the size bounds: min_out <= symbols of the block < max_out
 *    (1 KiB and 4 MiB by default).
 * Returns 1 if it holds, else 0; *why receives the failing reason (or 0).
 */
int orc_block_ok(const uint8_t* data, uint64_t end_bit, uint64_t b, const uint8_t* allowed,
                 uint64_t min_out, uint64_t max_out, int* why) {
    init_tables();
    dec_t d;
    memset(&d, 0, sizeof d);
    d.r.p = data; d.r.end = end_bit; d.r.pos = b;
    d.count_only = 1; d.allowed = allowed; d.check_lits = (allowed != NULL);
    d.max_block = max_out;
    int e;
    uint32_t bfinal = rd_bit(&d.r);
    uint32_t type = rd_bits(&d.r, 2);
    if (d.r.overrun) e = ORC_E_TRUNC;
    else if (bfinal) e = ORC_E_FINAL;
    else if (type != 2) e = ORC_E_TYPE;
    else {
        huff_t lit, dst;
        e = dynamic_header(&d.r, &lit, &dst);
        if (!e) e = codes(&d, &lit, &dst);
        if (!e && d.block_n < min_out) e = ORC_E_SIZE;
    }
    if (why) *why = e;
    return e == ORC_OK;
}

/* The confirmation of Section "Detection of DEFLATE block start positions":
   from b, the first block and `confirm` more blocks (fewer if a final block
   comes first) decode without error with a symbolic context, literals in the
   allowed set. */
int orc_confirm(const uint8_t* data, uint64_t end_bit, uint64_t b, const uint8_t* allowed, int confirm) {
    init_tables();
    dec_t d;
    memset(&d, 0, sizeof d);
    d.r.p = data; d.r.end = end_bit; d.r.pos = b;
    d.count_only = 1; d.allowed = allowed; d.check_lits = (allowed != NULL);
    int final = 0, e = ORC_OK;
    for (int k = 0; k <= confirm; k++) {
        e = block(&d, &final);
        if (e || final) break;
    }
    return e == ORC_OK;
}

/* Brute force over every bit of [from, to): the least b where the predicate
   holds (and, if confirm > 0, the confirmation too).  -1 if none. */
int64_t orc_sync_scan(const uint8_t* data, uint64_t end_bit, uint64_t from, uint64_t to,
                      const uint8_t* allowed, uint64_t min_out, uint64_t max_out, int confirm) {
    if (to > end_bit) to = end_bit;
    for (uint64_t b = from; b < to; b++) {
        if (!orc_block_ok(data, end_bit, b, allowed, min_out, max_out, NULL)) continue;
        if (confirm > 0 && !orc_confirm(data, end_bit, b, allowed, confirm)) continue;
        return (int64_t)b;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* gunzip: RFC 1952 members decoded one after another                  */
/* ------------------------------------------------------------------ */
/*
 * The plain definition of the result: every member's DEFLATE stream decoded
 * with decompress(C, w = empty), its CRC-32 and ISIZE checked.  Block start
 * bit offsets (from the start of `gz`) are recorded into block_bits if given.
 */
int orc_gunzip(const uint8_t* gz, uint64_t len, uint8_t* out, uint64_t cap, uint64_t* out_len,
               uint64_t* block_bits, uint64_t max_blocks, uint64_t* nblocks_out, int* members_out) {
    init_tables();
    uint64_t pos = 0, produced = 0, nb = 0;
    int members = 0, e = ORC_OK;
    while (pos < len) {
        int64_t h = orc_gzip_header(gz + pos, len - pos);
        if (h < 0) { e = members ? ORC_E_UNSUPPORTED : (int)h; break; }
        dec_t d;
        memset(&d, 0, sizeof d);
        d.r.p = gz; d.r.end = (len - 8) * 8; d.r.pos = (pos + (uint64_t)h) * 8;
        d.out8 = out + produced; d.cap = cap - produced; d.known = 1;
        int final = 0;
        do {
            if (block_bits && nb < max_blocks) block_bits[nb] = d.r.pos;
            nb++;
            e = block(&d, &final);
        } while (!e && !final);
        if (e) break;
        uint64_t tp = (d.r.pos + 7) >> 3;                  /* trailer on the next byte boundary */
        if (tp + 8 > len) { e = ORC_E_TRUNC; break; }
        uint32_t crc = gz[tp] | ((uint32_t)gz[tp + 1] << 8) | ((uint32_t)gz[tp + 2] << 16) | ((uint32_t)gz[tp + 3] << 24);
        uint32_t isz = gz[tp + 4] | ((uint32_t)gz[tp + 5] << 8) | ((uint32_t)gz[tp + 6] << 16) | ((uint32_t)gz[tp + 7] << 24);
        if (orc_crc32(0, out + produced, d.n) != crc) { e = ORC_E_CRC; break; }
        if ((uint32_t)d.n != isz) { e = ORC_E_ISIZE; break; }
        produced += d.n;
        pos = tp + 8;
        members++;
    }
    if (out_len) *out_len = produced;
    if (nblocks_out) *nblocks_out = nb;
    if (members_out) *members_out = members;
    return e;
}

/* ------------------------------------------------------------------ */
/* pass 2 pieces: Section "Full file decompression in two passes"      */
/* ------------------------------------------------------------------ */
/* translation of one part: U_j -> w[j], bytes unchanged */
void orc_translate(const uint16_t* sym, uint64_t n, const uint8_t* w, uint8_t* out) {
    for (uint64_t t = 0; t < n; t++)
        out[t] = (sym[t] & PH) ? w[sym[t] & (WSIZE - 1)] : (uint8_t)sym[t];
}

/* w_next = last 32768 characters of (w followed by the translated part).
   Reading for a part shorter than 32 KiB: the window keeps the tail of w. */
void orc_next_window(const uint8_t* w, const uint16_t* sym, uint64_t n, uint8_t* w_next) {
    uint8_t* ext = (uint8_t*)malloc(WSIZE + n);
    memcpy(ext, w, WSIZE);
    orc_translate(sym, n, w, ext + WSIZE);
    memcpy(w_next, ext + n, WSIZE);
    free(ext);
}

/* ------------------------------------------------------------------ */
/* the two-pass algorithm, restated on one CPU thread                   */
/* ------------------------------------------------------------------ */
/*
 * Section "Full file decompression in two passes (pugz)":
 *  1. the DEFLATE data of one gzip member is cut into n parts of equal
 *     compressed size; part i >= 1 starts at the least bit of
 *     [nominal_i, nominal_{i+1}) where a block start is detected and
 *     confirmed (orc_sync_scan); a part with none is empty (Reading);
 *  2. pass 1: part 0 is decoded with the empty context, every other part with
 *     the symbolic context, each up to the start of the next part.  Reading:
 *     if a part does not end exactly on the next part's start, that start was
 *     false; the part then continues to the start after it (merge);
 *  3. pass 2: w_1 is the last 32 KiB of D_0, w_{i+1} is w_i followed by D_i
 *     translated with w_i, cut to its last 32 KiB; then every D_i is
 *     translated with w_i;
 *  4. CRC-32 and ISIZE of the output are checked against the trailer.
 * part_bits[i] receives the start bit of part i (UINT64_MAX when empty),
 * part_len[i] its symbol count, part_nph[i] its placeholder symbols.
 */
int orc_two_pass(const uint8_t* gz, uint64_t len, int nparts, const uint8_t* allowed,
                 uint64_t min_out, uint64_t max_out, int confirm,
                 uint8_t* out, uint64_t cap, uint64_t* out_len,
                 uint64_t* part_bits, uint64_t* part_len, uint64_t* part_nph, int* false_syncs) {
    init_tables();
    if (nparts < 1) return ORC_E_ARG;
    int64_t h = orc_gzip_header(gz, len);
    if (h < 0) return (int)h;
    uint64_t s0 = (uint64_t)h, end_bit = (len - 8) * 8;
    uint64_t csize = (len - 8) - s0;
    uint64_t per = (csize + (uint64_t)nparts - 1) / (uint64_t)nparts;
    uint64_t* start = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nparts + 1));
    uint16_t** D = (uint16_t**)calloc((size_t)nparts, sizeof(uint16_t*));
    uint64_t* n = (uint64_t*)calloc((size_t)nparts, sizeof(uint64_t));
    if (!start || !D || !n) { free(start); free(D); free(n); return ORC_E_NOMEM; }
    const uint64_t NONE = ~(uint64_t)0;
    int e = ORC_OK, nfalse = 0;
    start[0] = s0 * 8;
    for (int i = 1; i < nparts; i++) {
        uint64_t lo = (s0 + (uint64_t)i * per) * 8, hi = (s0 + (uint64_t)(i + 1) * per) * 8;
        if (lo >= end_bit) { start[i] = NONE; continue; }
        int64_t b = orc_sync_scan(gz, end_bit, lo, hi < end_bit ? hi : end_bit, allowed, min_out, max_out, confirm);
        start[i] = b < 0 ? NONE : (uint64_t)b;
    }
    start[nparts] = NONE;
    /* pass 1 */
    uint64_t cap_sym = 0;
    for (int i = 0; i < nparts && !e; i++) {
        if (start[i] == NONE) continue;
        for (;;) {
            int k = i + 1;
            while (k < nparts && start[k] == NONE) k++;
            uint64_t stop = k < nparts ? start[k] : 0;
            /* size the part's buffer from a first counting pass */
            uint64_t cnt = 0, pos = 0, nb = 0, nph = 0;
            int final = 0;
            e = orc_inflate_from(gz, end_bit, start[i], stop, i == 0, NULL, 0, NULL, 0, &cnt, &pos, &final, &nb, &nph);
            if (e) break;
            if (k < nparts && pos != stop) {       /* did not land on the next start: it was false */
                start[k] = NONE;
                nfalse++;
                continue;
            }
            cap_sym = cnt ? cnt : 1;
            D[i] = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)cap_sym);
            if (!D[i]) { e = ORC_E_NOMEM; break; }
            e = orc_inflate_from(gz, end_bit, start[i], stop, i == 0, NULL, 0, D[i], cap_sym, &n[i], &pos, &final, &nb, &nph);
            if (part_nph) part_nph[i] = nph;
            if (!e && k >= nparts) {              /* the last part ends the member */
                if (!final) e = ORC_E_DATA;
                else if (((pos + 7) >> 3) + 8 != len) e = ORC_E_UNSUPPORTED;   /* more data after the member */
            }
            break;
        }
    }
    uint64_t total = 0;
    for (int i = 0; i < nparts; i++) total += n[i];
    if (!e && total > cap) e = ORC_E_CAPACITY;
    if (!e) {
        /* pass 2: windows in order, then translation */
        uint8_t* w = (uint8_t*)calloc(WSIZE, 1);
        uint8_t* wn = (uint8_t*)calloc(WSIZE, 1);
        uint64_t off = 0;
        for (int i = 0; i < nparts; i++) {
            if (start[i] == NONE) continue;
            orc_translate(D[i], n[i], w, out + off);
            orc_next_window(w, D[i], n[i], wn);
            uint8_t* t = w; w = wn; wn = t;
            off += n[i];
        }
        free(w); free(wn);
        uint64_t tp = len - 8;
        uint32_t crc = gz[tp] | ((uint32_t)gz[tp + 1] << 8) | ((uint32_t)gz[tp + 2] << 16) | ((uint32_t)gz[tp + 3] << 24);
        uint32_t isz = gz[tp + 4] | ((uint32_t)gz[tp + 5] << 8) | ((uint32_t)gz[tp + 6] << 16) | ((uint32_t)gz[tp + 7] << 24);
        if (orc_crc32(0, out, total) != crc) e = ORC_E_CRC;
        else if ((uint32_t)total != isz) e = ORC_E_ISIZE;
    }
    if (out_len) *out_len = total;
    for (int i = 0; i < nparts; i++) {
        if (part_bits) part_bits[i] = start[i];
        if (part_len) part_len[i] = n[i];
        free(D[i]);
    }
    if (false_syncs) *false_syncs = nfalse;
    free(start); free(D); free(n);
    return e;
}

/* ------------------------------------------------------------------ */
/* Problem "Random access in DEFLATE stream": decode from a bit offset  */
/* ------------------------------------------------------------------ */
/*
 * From compressed bit `start_bit` of a gzip member: find the next confirmed
 * block start (or take the stream start when start_bit is at or before it,
 * with the empty context), then decode to the end of the member with the
 * symbolic context.  sym receives the symbols; bytes (optional) the same with
 * every placeholder replaced by `fill` (the undetermined '?' context of
 * Section "Undetermined context propagation technique").
 * *first_determined = one past the last placeholder (0 if none).
 */
int orc_decompress_at(const uint8_t* gz, uint64_t len, uint64_t start_bit, const uint8_t* allowed,
                      uint64_t min_out, uint64_t max_out, int confirm, uint8_t fill,
                      uint16_t* sym, uint8_t* bytes, uint64_t cap, uint64_t* out_len,
                      uint64_t* block_bit, uint64_t* first_determined) {
    init_tables();
    int64_t h = orc_gzip_header(gz, len);
    if (h < 0) return (int)h;
    uint64_t s0 = (uint64_t)h * 8, end_bit = (len - 8) * 8;
    uint64_t b;
    int known = 0;
    if (start_bit <= s0) { b = s0; known = 1; }
    else {
        int64_t f = orc_sync_scan(gz, end_bit, start_bit, end_bit, allowed, min_out, max_out, confirm);
        if (f < 0) return ORC_E_NOSYNC;
        b = (uint64_t)f;
    }
    uint64_t n = 0, pos = 0, nb = 0, nph = 0;
    int final = 0;
    int e = orc_inflate_from(gz, end_bit, b, 0, known, NULL, 0, sym, cap, &n, &pos, &final, &nb, &nph);
    if (!e && !final) e = ORC_E_DATA;
    uint64_t fd = 0;
    for (uint64_t t = 0; t < n; t++) {
        if (sym[t] & PH) fd = t + 1;
        if (bytes) bytes[t] = (sym[t] & PH) ? fill : (uint8_t)sym[t];
    }
    if (out_len) *out_len = n;
    if (block_bit) *block_bit = b;
    if (first_determined) *first_determined = fd;
    return e;
}
