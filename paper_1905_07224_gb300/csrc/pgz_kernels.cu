// pgz_kernels.cu -- sm_103a kernels of the two-pass parallel gzip decompression
// (Kerbiriou & Chikhi, arXiv 1905.07224, Section "Full file decompression in
// two passes (pugz)").
//
//   k_sync      pass 1a: per part, the first bit of [lo, hi) where a DEFLATE
//               block starts (Section "Detection of DEFLATE block start
//               positions", Appendix "DEFLATE block decompression checks"):
//               a warp tests 1024 bit offsets per step (one 32-bit window per
//               lane, bit-parallel header tests), __ballot_sync + __ffs elect
//               the lowest candidate, and the candidate's whole block is then
//               decoded as the final check -- into the part's own output, so
//               pass 1 resumes after it.
//   k_inflate   pass 1b: decode(C_i, w^_i) (Algorithm "DEFLATE decompression"
//               with the symbolic context [U_0..U_32767]) up to the next
//               part's block start.  One warp per part: the lanes decode
//               segments of a block in parallel and meet (see par_block), then
//               write the tokens' symbols cooperatively.  The 32 KiB window is
//               the part's own u16 output in global memory; a source before
//               the part start p < 0 is the placeholder U_{32768+p}, computed,
//               not stored.
//   k_plan      output offsets of the parts (prefix of their lengths), error
//               aggregation, ISIZE and capacity checks.
//   k_chain_*   pass 2a: w_{i+1} from w_i and the tail of D_i (Section "Full
//               file decompression in two passes").  Each part's tail is a map
//               from w_i to w_{i+1} whose entries are bytes or indices; maps
//               compose, so groups of parts are composed in parallel, walked
//               across groups, then expanded per part.
//   k_translate pass 2b: U_j -> w_i[j] for every symbol, written to the
//               final output with 8-byte aligned stores (HBM-bound).
//   k_crc       CRC-32 (RFC 1952) of the output: raw CRCs of 128-byte pieces,
//               combined by multiplication with x^(8n) mod P in GF(2) and
//               XOR-accumulated per member.
//   k_finalize  finished CRC-32 against the trailer.
//
// No kernel waits on another block or warp; every read of the compressed
// data, the symbol scratch and the output is bounds-checked.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "pgz_internal.h"
#include "../../include/pgz.h"

namespace pgz {
namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int LB = 10;          // literal/length lookup bits
constexpr int DB = 8;           // distance lookup bits
constexpr uint32_t kPoly = 0xEDB88320u;

// RFC 1951 3.2.5: length codes 257..285 and distance codes 0..29
__constant__ uint16_t c_lbase[29] = {3, 4, 5, 6, 7, 8, 9, 10, 11, 13, 15, 17, 19, 23, 27, 31,
                                     35, 43, 51, 59, 67, 83, 99, 115, 131, 163, 195, 227, 258};
__constant__ uint8_t c_lext[29] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2,
                                   3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 5, 0};
__constant__ uint16_t c_dbase[30] = {1, 2, 3, 4, 5, 7, 9, 13, 17, 25, 33, 49, 65, 97, 129,
                                     193, 257, 385, 513, 769, 1025, 1537, 2049, 3073, 4097,
                                     6145, 8193, 12289, 16385, 24577};
__constant__ uint8_t c_dext[30] = {0, 0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5, 6, 6,
                                   7, 7, 8, 8, 9, 9, 10, 10, 11, 11, 12, 12, 13, 13};
// RFC 1951 3.2.7: order of the code-length code lengths
__constant__ uint8_t c_clorder[19] = {16, 17, 18, 0, 8, 7, 9, 6, 10, 5, 11, 4, 12, 3, 13, 2, 14, 1, 15};
// CRC-32 tables (filled by upload_crc_tables)
__constant__ uint32_t c_crc_tab[4][256];   // [0][b]: register after byte b from a zero register; [k]: k more zero bytes
__constant__ uint32_t c_x2k[64];           // x^(2^k) mod P
__constant__ uint32_t c_lane_shift[32];    // x^(8*kPiece*k) mod P
__constant__ uint32_t c_seg_shift[4][256]; // [j][b]: (byte b at byte j of a register) x^(8*kCrcSeg) mod P

// literal/length lookup entry: bits 0-4 bits to drop, 8-16 value, 17-19
// extra-bit count (K_LENX), 28-31 kind.  K_LEN carries the exact length
// (code and extra bits both inside the lookup width), K_LENX the base.
// K_LIT2: two literals whose codes both fit the lookup width: bits 8-15 and
// 16-23 the bytes, 24-27 the first code's length, 0-4 both lengths.
enum : uint32_t { K_LIT = 0, K_LIT2 = 1, K_LEN = 2, K_LENX = 3, K_EOB = 4, K_LONG = 5, K_BAD = 6 };
// distance lookup entry: bits 0-3 code length, 4-7 extra bits, 8-9 kind, 16-31 base
enum : uint32_t { DK_OK = 0, DK_LONG = 1, DK_BAD = 2 };

struct WarpSmem {
    uint32_t lit[1 << LB];
    uint32_t dist[1 << DB];
    uint16_t lsym[288];
    uint16_t dsym[32];
    uint16_t lfirst[16], lcount[16], loff[16];
    uint16_t dfirst[16], dcount[16], doff[16];
    uint32_t cnt[16];
    uint32_t allowed[8];
    uint32_t lmax, dmax, table_kind, pad;
    uint8_t lens[320];
    uint8_t cllens[32];
    uint32_t masks[32 * 32];   // parallel decoding: token starts in the first 1024 bits of each lane's segment;
                               // reused by exec_range: words 0-511 the entries of two passes of 256
                               // positions, 512-767 the batch's tokens, 768-1023 their output offsets
};

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    uint32_t lo = __shfl_sync(FULL, (uint32_t)v, src), hi = __shfl_sync(FULL, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

// ---------------------------------------------------------------------------
// bit input: RFC 1951 3.1.1, LSB first; 32-bit words, bounds-checked; the
// next word is loaded one refill ahead
// ---------------------------------------------------------------------------
struct BitIn {
    const uint32_t* w;   // the member's bytes as 32-bit words (4-byte aligned)
    const uint8_t* b;
    uint64_t nbytes;
    uint32_t nfull;      // words wholly inside the member
    uint32_t lo, hi;     // buffered bits [0, 32) and [32, 64); zero above cnt
    uint32_t cnt;        // buffered bits
    uint32_t nxt;        // word(wi), loaded one refill ahead
    uint32_t wi;         // next word to merge into the buffer

    __device__ __forceinline__ void setup(const uint8_t* gz, uint64_t len) {
        w = reinterpret_cast<const uint32_t*>(gz);
        b = gz;
        nbytes = len;
        nfull = (uint32_t)((len >> 2) < 0xffffffffull ? (len >> 2) : 0xffffffffull);
    }
    __device__ __forceinline__ uint32_t word(uint64_t i) const {
        if (i < nfull) return __ldg(w + i);
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t p = i * 4 + k;
            if (p < nbytes) v |= (uint32_t)__ldg(b + p) << (8 * k);
        }
        return v;
    }
    // SAFE: the caller has checked that word wi lies inside the member
    template <bool SAFE = false>
    __device__ __forceinline__ void refill() {
        if (cnt <= 32) {
            lo |= __funnelshift_lc(0u, nxt, cnt);    // nxt << cnt, 0 when cnt = 32
            hi |= __funnelshift_lc(nxt, 0u, cnt);    // nxt >> (32 - cnt), nxt when cnt = 32
            cnt += 32;
            ++wi;
            nxt = SAFE ? __ldg(w + wi) : word(wi);
        }
    }
    __device__ __forceinline__ void seek(uint64_t bit) {
        wi = (uint32_t)(bit >> 5);
        const uint32_t s = (uint32_t)(bit & 31);
        lo = word(wi) >> s;
        hi = 0;
        cnt = 32 - s;
        ++wi;
        nxt = word(wi);
        refill();
    }
    __device__ __forceinline__ uint64_t pos() const { return (uint64_t)wi * 32 - cnt; }
    __device__ __forceinline__ uint32_t peek(uint32_t n) const { return lo & ((1u << n) - 1u); }   // n < 32
    __device__ __forceinline__ void drop(uint32_t n) {                                           // n < 32
        lo = __funnelshift_r(lo, hi, n);
        hi >>= n;
        cnt -= n;
    }
};

// ---------------------------------------------------------------------------
// canonical Huffman codes (RFC 1951 3.2.2), built by one warp
// ---------------------------------------------------------------------------
struct CodeInfo {
    int status;   // 0 complete, 1 incomplete, -1 over-subscribed
    int ncodes;
    int maxlen;
};

__device__ CodeInfo build_code(WarpSmem& S, const uint8_t* lens, int n, uint16_t* first, uint16_t* count,
                               uint16_t* off, uint16_t* sym, int lane) {
    if (lane < 16) S.cnt[lane] = 0;
    __syncwarp();
    for (int s = lane; s < n; s += 32) {
        const uint32_t l = lens[s];
        if (l) atomicAdd(&S.cnt[l], 1u);
    }
    __syncwarp();
    CodeInfo ci{0, 0, 0};
    int left = 1;
    uint32_t code = 0, o = 0, prev = 0;
    for (int L = 1; L <= 15; ++L) {
        const uint32_t c = S.cnt[L];
        left = 2 * left - (int)c;
        if (left < 0) ci.status = -1;
        if (c) ci.maxlen = L;
        ci.ncodes += (int)c;
        code = (code + prev) << 1;
        prev = c;
        if (lane == 0) {
            first[L] = (uint16_t)code;
            count[L] = (uint16_t)c;
            off[L] = (uint16_t)o;
        }
        o += c;
    }
    if (lane == 0) first[0] = count[0] = off[0] = 0;
    if (ci.status == 0 && left > 0) ci.status = 1;
    __syncwarp();
    if (ci.status < 0) return ci;
    if (lane < 16) S.cnt[lane] = off[lane];
    __syncwarp();
    for (int s0 = 0; s0 < n; s0 += 32) {          // symbols in (length, value) order
        const int s = s0 + lane;
        const uint32_t l = (s < n) ? lens[s] : 0u;
        const uint32_t peers = __match_any_sync(FULL, l);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        const uint32_t base = S.cnt[l];
        if (s < n && l) sym[base + rank] = (uint16_t)s;
        __syncwarp();
        if (rank == 0 && l) S.cnt[l] = base + __popc(peers);
        __syncwarp();
    }
    return ci;
}

// lut[x] for every NB-bit stream pattern x: the code of length <= NB that
// prefixes it (make(symbol, length, x)), else `miss` (a longer code, or none)
template <int NB, typename Make>
__device__ void fill_lut(uint32_t* lut, const uint16_t* first, const uint16_t* count, const uint16_t* off,
                         const uint16_t* sym, int maxlen, uint32_t miss, Make make, int lane) {
    const int top = maxlen < NB ? maxlen : NB;
    for (uint32_t v = lane; v < (1u << NB); v += 32) {      // v: NB code bits, first bit most significant
        const uint32_t x = __brev(v) >> (32 - NB);
        uint32_t e = miss;
        for (int L = 1; L <= top; ++L) {
            const uint32_t d = (v >> (NB - L)) - first[L];
            if (d < count[L]) {
                e = make(sym[off[L] + d], (uint32_t)L, x, v);
                break;
            }
        }
        lut[x] = e;
    }
}

// codes longer than the lookup width: compare the first L bits with each
// length's code range
__device__ __forceinline__ int decode_long(uint32_t bits15, int nb, const uint16_t* first, const uint16_t* count,
                                           const uint16_t* off, const uint16_t* sym, int maxlen, uint32_t& len) {
    const uint32_t v = __brev(bits15) >> 17;
    for (int L = nb + 1; L <= maxlen; ++L) {
        const uint32_t d = (v >> (15 - L)) - first[L];
        if (d < count[L]) {
            len = (uint32_t)L;
            return sym[off[L] + d];
        }
    }
    return -1;
}

// x: the lookup index (stream bits), whose bits after the code are the
// length's extra bits when they fit
__device__ __forceinline__ uint32_t lit_entry(uint32_t s, uint32_t L, uint32_t x) {
    if (s < 256) return (K_LIT << 28) | (s << 8) | L;
    if (s == 256) return (K_EOB << 28) | L;
    if (s < 286) {
        const uint32_t k = s - 257, base = c_lbase[k], E = c_lext[k];
        if (L + E <= (uint32_t)LB) return (K_LEN << 28) | ((base + ((x >> L) & ((1u << E) - 1u))) << 8) | (L + E);
        return (K_LENX << 28) | (E << 17) | (base << 8) | L;
    }
    return (K_BAD << 28) | L;
}

__device__ __forceinline__ uint32_t dist_entry(uint32_t s, uint32_t L) {
    if (s < 30) return ((uint32_t)c_dbase[s] << 16) | ((uint32_t)c_dext[s] << 4) | L;
    return (DK_BAD << 8) | L;
}

// a literal followed, inside the lookup width, by a second literal: one entry
struct LitMake {
    const uint16_t *first, *count, *off, *sym;
    __device__ uint32_t operator()(uint32_t s, uint32_t L, uint32_t x, uint32_t v) const {
        const uint32_t e = lit_entry(s, L, x);
        if (s >= 256 || L >= (uint32_t)LB - 1) return e;
        const uint32_t rest = LB - L, v2 = v & ((1u << rest) - 1u);   // the next code bits, first bit most significant
        for (uint32_t L2 = 1; L2 <= rest; ++L2) {
            const uint32_t d = (v2 >> (rest - L2)) - first[L2];
            if (d < count[L2]) {
                const uint32_t s2 = sym[off[L2] + d];
                if (s2 >= 256) return e;
                return (K_LIT2 << 28) | (L << 24) | (s2 << 16) | (s << 8) | (L + L2);
            }
        }
        return e;
    }
};
struct DistMake {
    __device__ uint32_t operator()(uint32_t s, uint32_t L, uint32_t, uint32_t) const { return dist_entry(s, L); }
};
struct ClMake {
    __device__ uint32_t operator()(uint32_t s, uint32_t L, uint32_t, uint32_t) const { return s | (L << 8); }
};

// Reading of valid codes, as RFC 1951 3.2.7 and its producer zlib use them:
// code-length code complete; literal/length code complete or one code of
// length 1, with an end-of-block code; distance code complete, one code of
// length 1, or empty.  HDR_ONLY: stop after the checks (block-start search);
// an over-subscribed length set ends the decoding early either way.
template <bool HDR_ONLY>
__device__ int read_dynamic(WarpSmem& S, BitIn& br, int lane) {
    if (lane == 0) S.table_kind = 0;
    br.refill();
    const uint32_t hlit = br.peek(5) + 257;
    br.drop(5);
    const uint32_t hdist = br.peek(5) + 1;
    br.drop(5);
    const uint32_t hclen = br.peek(4) + 4;
    br.drop(4);
    if (hlit > 286 || hdist > 30) return CE_DATA;
    S.cllens[lane] = 0;
    __syncwarp();
    br.refill();
    const uint32_t n1 = hclen < 10 ? hclen : 10;
    if ((uint32_t)lane < n1) S.cllens[c_clorder[lane]] = (uint8_t)((br.lo >> (3 * lane)) & 7);
    br.drop(3 * n1);
    br.refill();
    if (hclen > 10) {
        if ((uint32_t)lane >= 10 && (uint32_t)lane < hclen)
            S.cllens[c_clorder[lane]] = (uint8_t)((br.lo >> (3 * (lane - 10))) & 7);
        br.drop(3 * (hclen - 10));
    }
    __syncwarp();
    CodeInfo ci = build_code(S, S.cllens, 19, S.dfirst, S.dcount, S.doff, S.dsym, lane);
    if (ci.status != 0) return CE_DATA;
    __syncwarp();
    fill_lut<7>(S.dist, S.dfirst, S.dcount, S.doff, S.dsym, ci.maxlen, 0u, ClMake(), lane);
    __syncwarp();
    const uint32_t total = hlit + hdist;
    uint32_t i = 0, prev = 0;
    uint32_t kl = 0, kd = 0, nl = 0, nd = 0, ml = 0, md = 0;   // Kraft sums (units of 2^-15), counts, max lengths
    bool eob = false;
    while (i < total) {
        br.refill();
        const uint32_t e = S.dist[br.peek(7)];
        const uint32_t s = e & 0xffu;
        br.drop(e >> 8);
        uint32_t rep = 1, val;
        if (s < 16) {
            val = s;
            prev = s;
        } else if (s == 16) {
            if (i == 0) return CE_DATA;
            val = prev;
            rep = 3 + br.peek(2);
            br.drop(2);
        } else if (s == 17) {
            val = 0;
            rep = 3 + br.peek(3);
            br.drop(3);
            prev = 0;
        } else {
            val = 0;
            rep = 11 + br.peek(7);
            br.drop(7);
            prev = 0;
        }
        if (i + rep > total) return CE_DATA;
        if (val) {
            const uint32_t e2 = i + rep;
            const uint32_t nlit = i < hlit ? ((e2 < hlit ? e2 : hlit) - i) : 0u;
            const uint32_t ndst = rep - nlit;
            kl += nlit * (32768u >> val);
            kd += ndst * (32768u >> val);
            nl += nlit;
            nd += ndst;
            if (nlit && val > ml) ml = val;
            if (ndst && val > md) md = val;
            if (i <= 256 && 256 < e2) eob = true;
            if (kl > 32768u || kd > 32768u) return CE_DATA;       // over-subscribed
        }
        if (!HDR_ONLY) {
            if (rep == 1) {
                if (lane == 0) S.lens[i] = (uint8_t)val;
            } else {
                for (uint32_t j = lane; j < rep; j += 32) S.lens[i + j] = (uint8_t)val;
            }
        }
        i += rep;
    }
    if (!eob) return CE_DATA;
    if (!(kl == 32768u || (nl == 1 && ml == 1))) return CE_DATA;
    if (!(kd == 32768u || nd == 0 || (nd == 1 && md == 1))) return CE_DATA;
    if (HDR_ONLY) return CE_OK;
    __syncwarp();
    ci = build_code(S, S.lens, (int)hlit, S.lfirst, S.lcount, S.loff, S.lsym, lane);
    if (ci.status < 0) return CE_DATA;
    __syncwarp();
    fill_lut<LB>(S.lit, S.lfirst, S.lcount, S.loff, S.lsym, ci.maxlen, K_LONG << 28,
                 LitMake{S.lfirst, S.lcount, S.loff, S.lsym}, lane);
    if (lane == 0) S.lmax = (uint32_t)ci.maxlen;
    ci = build_code(S, S.lens + hlit, (int)hdist, S.dfirst, S.dcount, S.doff, S.dsym, lane);
    if (ci.status < 0) return CE_DATA;
    __syncwarp();
    fill_lut<DB>(S.dist, S.dfirst, S.dcount, S.doff, S.dsym, ci.maxlen, DK_LONG << 8, DistMake(), lane);
    if (lane == 0) {
        S.dmax = (uint32_t)ci.maxlen;
        S.table_kind = 2;
    }
    __syncwarp();
    return CE_OK;
}

// the fixed code of RFC 1951 3.2.6
__device__ void build_fixed(WarpSmem& S, int lane) {
    for (int s = lane; s < 320; s += 32)
        S.lens[s] = (uint8_t)(s < 144 ? 8 : s < 256 ? 9 : s < 280 ? 7 : s < 288 ? 8 : 5);
    __syncwarp();
    CodeInfo ci = build_code(S, S.lens, 288, S.lfirst, S.lcount, S.loff, S.lsym, lane);
    __syncwarp();
    fill_lut<LB>(S.lit, S.lfirst, S.lcount, S.loff, S.lsym, ci.maxlen, K_LONG << 28,
                 LitMake{S.lfirst, S.lcount, S.loff, S.lsym}, lane);
    if (lane == 0) S.lmax = (uint32_t)ci.maxlen;
    ci = build_code(S, S.lens + 288, 32, S.dfirst, S.dcount, S.doff, S.dsym, lane);
    __syncwarp();
    fill_lut<DB>(S.dist, S.dfirst, S.dcount, S.doff, S.dsym, ci.maxlen, DK_LONG << 8, DistMake(), lane);
    if (lane == 0) {
        S.dmax = (uint32_t)ci.maxlen;
        S.table_kind = 1;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// symbol output of one part
// ---------------------------------------------------------------------------
struct OutState {
    uint16_t* sym;     // the part's symbols; also its window
    uint64_t cap;
    uint64_t n;        // symbols so far (uniform)
    bool known;        // the context before the part is empty (member start)
    bool neg;          // this lane copied from before the part start (a placeholder source)
    // The determined tail (Section "Undetermined context propagation technique": a placeholder is only ever
    // copied, so once the last 32 KiB of output hold none, no later symbol can be one): symbols from det on
    // are stored as bytes, symbol k at byte det + k of the part's buffer (det is a multiple of 8, so a lane's
    // 8 positions are all below it or all at or above it).  ~0: no tail yet.
    uint32_t det = 0xffffffffu;
    uint32_t last_ph = 0;   // at or after one past the last placeholder written (uniform; kept in kTail mode)
};

__device__ __forceinline__ uint8_t* tail_bytes(const OutState& o) { return reinterpret_cast<uint8_t*>(o.sym) + o.det; }

__device__ __forceinline__ void cp_async4(uint32_t dst_shared, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst_shared), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// the symbol at part position q: q < 0 lies in the symbolic context.  Part
// positions are 32-bit (a part holds fewer than 2^31 symbols).
__device__ __forceinline__ uint16_t sym_at(const uint16_t* out, int32_t q) {
    return q >= 0 ? out[(uint32_t)q] : (uint16_t)(kPH | (uint32_t)((int32_t)kWin + q));
}
// the same with the determined tail: a position at or after o.det is a byte
__device__ __forceinline__ uint16_t sym_get(const OutState& o, int32_t q) {
    if (q >= 0 && (uint32_t)q >= o.det) return tail_bytes(o)[(uint32_t)q];
    return sym_at(o.sym, q);
}
// an upper bound on one past the part's last placeholder: the end of any pass of 256 positions (from A) that
// wrote one (uniform)
__device__ __forceinline__ void track_placeholders(OutState& o, const uint32_t* e, uint32_t A, uint32_t end) {
    uint32_t any = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) any |= e[u];
    if (__any_sync(0xffffffffu, (any & kPH) != 0)) o.last_ph = max(o.last_ph, min(A + 256u, end));
}

// Writes the symbols of a batch of tokens (lane t holds token t < ntok):
// token = (1 << 16) | byte for a literal, bit 31 | length << 16 | (distance-1)
// for a match.  Output-parallel: lane j produces output positions j, j + 32,
// ... of the batch.  A position inside a match follows the copy to its source;
// a source inside the batch is resolved in registers (the covering token is
// found by binary search over the tokens' starts, an overlapping copy folds
// back by the distance), so only sources before the batch are loaded from the
// part's output (or are placeholders U_j before the part start).  All loads of
// up to 256 positions are issued before their stores.
__device__ __forceinline__ int exec_batch(OutState& o, uint32_t tok, int ntok, int lane, uint64_t& block_n) {
    const bool valid = lane < ntok;
    const uint32_t len = valid ? ((tok >> 16) & 0x1ffu) : 0u;
    uint32_t incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t base = (uint32_t)o.n;
    if ((uint64_t)base + total > o.cap) return CE_OVERFLOW;
    const uint32_t st = incl - len;          // start of my token, relative to the batch
    uint16_t* out = o.sym;
    bool bad = false;
    for (uint32_t r0 = 0; r0 < total; r0 += 256) {
        uint32_t val[8];
        int32_t src[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            uint32_t rel = r0 + 32u * r + (uint32_t)lane;
            bool need = rel < total;
            val[r] = 0;
            src[r] = INT32_MIN;
            while (__any_sync(FULL, need)) {
                int t = 0;
#pragma unroll
                for (int sft = 16; sft; sft >>= 1) {
                    const uint32_t x = __shfl_sync(FULL, st, (t + sft) & 31);
                    if (t + sft < ntok && x <= rel) t += sft;
                }
                const uint32_t tk = __shfl_sync(FULL, tok, t), sk = __shfl_sync(FULL, st, t);
                if (need) {
                    if (!(tk >> 31)) {
                        val[r] = tk & 0xffu;
                        need = false;
                    } else {
                        const uint32_t dk = (tk & 0xffffu) + 1u;
                        int32_t q = (int32_t)rel - (int32_t)dk;
                        if (q >= (int32_t)sk) q = (int32_t)sk - (int32_t)dk + (int32_t)((rel - sk) % dk);
                        if (q < 0) {
                            src[r] = (int32_t)base + q;     // before the batch: final, or a placeholder
                            need = false;
                        } else {
                            rel = (uint32_t)q;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (src[r] != INT32_MIN) {
                if (src[r] < 0) {
                    if (o.known) bad = true;
                    o.neg = true;
                }
                val[r] = sym_at(out, src[r]);
            }
        }
        if (__any_sync(FULL, bad)) return CE_DIST;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint32_t rel = r0 + 32u * r + (uint32_t)lane;
            if (rel < total) out[base + rel] = (uint16_t)val[r];
        }
    }
    __syncwarp();
    o.n = base + total;
    block_n += total;
    return CE_OK;
}

__device__ __forceinline__ bool allowed_has(const uint32_t* a, uint32_t b) { return (a[b >> 5] >> (b & 31)) & 1u; }

// Up to 32 tokens of a Huffman block; lane t keeps token t.  SAFE: every
// word this batch can read lies inside the member (no bounds checks).
template <bool SAFE, bool CHECK>
__device__ __forceinline__ int decode_batch(WarpSmem& S, BitIn& br, int lane, uint32_t& mytok, int& ntok, bool& eob) {
#pragma unroll 1
    while (ntok < 32) {
        br.refill<SAFE>();
        uint32_t e = S.lit[br.lo & ((1u << LB) - 1u)];
        uint32_t k = e >> 28;
        if (k <= K_LIT2) {
            const uint32_t b = (e >> 8) & 0xffu;
            if (k == K_LIT2 && ntok < 31) {
                const uint32_t b2 = (e >> 16) & 0xffu;
                if (CHECK && !(allowed_has(S.allowed, b) && allowed_has(S.allowed, b2))) return CE_BYTE;
                br.drop(e & 31u);
                if (lane == ntok) mytok = 0x10000u | b;
                if (lane == ntok + 1) mytok = 0x10000u | b2;
                ntok += 2;
                continue;
            }
            if (CHECK && !allowed_has(S.allowed, b)) return CE_BYTE;
            br.drop(k == K_LIT ? (e & 31u) : ((e >> 24) & 15u));
            if (lane == ntok) mytok = 0x10000u | b;
            ++ntok;
            continue;
        }
        if (k >= K_LONG) {
            uint32_t L = 0;
            const int s = k == K_LONG
                              ? decode_long(br.peek(15), LB, S.lfirst, S.lcount, S.loff, S.lsym, (int)S.lmax, L)
                              : -1;
            if (s < 0) return CE_DATA;
            e = lit_entry((uint32_t)s, L, 0);
            k = e >> 28;
            if (k == K_BAD) return CE_DATA;
            if (k == K_LIT) {
                const uint32_t b = (e >> 8) & 0xffu;
                if (CHECK && !allowed_has(S.allowed, b)) return CE_BYTE;
                br.drop(e & 31u);
                if (lane == ntok) mytok = 0x10000u | b;
                ++ntok;
                continue;
            }
        }
        if (k == K_EOB) {
            br.drop(e & 31u);
            eob = true;
            return CE_OK;
        }
        uint32_t len = (e >> 8) & 0x1ffu, dn = e & 31u;
        if (k == K_LENX) {
            const uint32_t eb = (e >> 17) & 7u;
            len += (br.lo >> dn) & ((1u << eb) - 1u);
            dn += eb;
        }
        br.drop(dn);
        br.refill<SAFE>();
        uint32_t d = S.dist[br.lo & ((1u << DB) - 1u)];
        if (d & 0x300u) {
            if ((d & 0x300u) != (DK_LONG << 8)) return CE_DATA;
            uint32_t L = 0;
            const int s = decode_long(br.peek(15), DB, S.dfirst, S.dcount, S.doff, S.dsym, (int)S.dmax, L);
            if (s < 0) return CE_DATA;
            d = dist_entry((uint32_t)s, L);
            if (d & 0x300u) return CE_DATA;
        }
        const uint32_t dl = d & 15u, de = (d >> 4) & 15u;
        const uint32_t dist = (d >> 16) + ((br.lo >> dl) & ((1u << de) - 1u));
        br.drop(dl + de);
        if (lane == ntok) mytok = 0x80000000u | (len << 16) | (dist - 1u);
        ++ntok;
    }
    return CE_OK;
}

constexpr int CE_MORE = 100;   // internal: the token limit was reached inside the block

__device__ int huff_block(WarpSmem& S, BitIn& br, OutState& o, bool check, uint64_t max_block, uint64_t end_bit,
                          uint64_t& block_n, int lane, uint32_t tok_limit = 0) {
    uint32_t done = 0;
    for (;;) {
        uint32_t mytok = 0;
        int ntok = 0;
        bool eob = false;
        const int st = check ? decode_batch<false, true>(S, br, lane, mytok, ntok, eob)
                             : decode_batch<false, false>(S, br, lane, mytok, ntok, eob);
        if (st) return st;
        if (ntok) {
            const int e = exec_batch(o, mytok, ntok, lane, block_n);
            if (e) return e;
        }
        if (br.pos() > end_bit) return CE_TRUNC;
        if (max_block && block_n >= max_block) return CE_SIZE;
        if (eob) return CE_OK;
        done += (uint32_t)ntok;
        if (tok_limit && done >= tok_limit) return CE_MORE;
    }
}

// ---------------------------------------------------------------------------
// parallel decoding of one Huffman block by the 32 lanes of a warp.
// Round: lane k decodes its own kSeg-bit segment from bit start + k*kSeg with
// the block's codes (a guess: it may begin inside a code), storing its tokens
// and marking its token starts among the first kSyncW bits.  Lane k then
// continues into segment k+1 until its parse meets a token start of lane
// k+1's parse: from there the two parses are identical (Huffman codes
// resynchronise), so lane k+1's tokens from that bit on are the block's.
// Lane 0 starts at a known token start, so the chain of meeting points gives
// the true token sequence; the warp then writes those tokens in order.  A
// lane that does not meet its successor within kSyncW bits ends the round
// there; the next round starts at that known position.
// ---------------------------------------------------------------------------
constexpr uint32_t kSeg = 2048;      // bits per lane per round
constexpr uint32_t kSyncW = 1024;    // bits at the head of a segment where meeting points are looked for
constexpr uint32_t kTokCap = 512;    // tokens a lane may keep per round (own segment + continuation)
constexpr uint64_t kTokPerPart = 32ull * kTokCap;   // token buffer of one part (one warp)

enum : int { LT_ONE = 0, LT_TWO = 1, LT_EOB = 2, LT_ERR = 3 };

// one token by one lane: t0 (and t1 for two literals, the first l1 bits long)
template <bool SAFE>
__device__ __forceinline__ int lane_token(const WarpSmem& S, BitIn& b, uint32_t& t0, uint32_t& t1, uint32_t& l1) {
    b.refill<SAFE>();
    uint32_t e = S.lit[b.lo & ((1u << LB) - 1u)];
    uint32_t k = e >> 28;
    if (k == K_LIT2) {
        t0 = 0x10000u | ((e >> 8) & 0xffu);
        t1 = 0x10000u | ((e >> 16) & 0xffu);
        l1 = (e >> 24) & 15u;
        b.drop(e & 31u);
        return LT_TWO;
    }
    if (k >= K_LONG) {
        uint32_t L = 0;
        const int s = k == K_LONG ? decode_long(b.peek(15), LB, S.lfirst, S.lcount, S.loff, S.lsym, (int)S.lmax, L) : -1;
        if (s < 0) return LT_ERR;
        e = lit_entry((uint32_t)s, L, 0);
        k = e >> 28;
        if (k == K_BAD) return LT_ERR;
    }
    if (k == K_LIT) {
        t0 = 0x10000u | ((e >> 8) & 0xffu);
        b.drop(e & 31u);
        return LT_ONE;
    }
    if (k == K_EOB) {
        b.drop(e & 31u);
        return LT_EOB;
    }
    uint32_t len = (e >> 8) & 0x1ffu, dn = e & 31u;
    if (k == K_LENX) {
        const uint32_t eb = (e >> 17) & 7u;
        len += (b.lo >> dn) & ((1u << eb) - 1u);
        dn += eb;
    }
    b.drop(dn);
    b.refill<SAFE>();
    uint32_t d = S.dist[b.lo & ((1u << DB) - 1u)];
    if (d & 0x300u) {
        if ((d & 0x300u) != (DK_LONG << 8)) return LT_ERR;
        uint32_t L = 0;
        const int s = decode_long(b.peek(15), DB, S.dfirst, S.dcount, S.doff, S.dsym, (int)S.dmax, L);
        if (s < 0) return LT_ERR;
        d = dist_entry((uint32_t)s, L);
        if (d & 0x300u) return LT_ERR;
    }
    const uint32_t dl = d & 15u, de = (d >> 4) & 15u;
    const uint32_t dist = (d >> 16) + ((b.lo >> dl) & ((1u << de) - 1u));
    b.drop(dl + de);
    t0 = 0x80000000u | (len << 16) | (dist - 1u);
    return LT_ONE;
}

enum : uint32_t { PS_OK = 0, PS_EOB = 1, PS_ERR = 2, PS_CAP = 3, PS_SYNC = 4, PS_NOSYNC = 5 };

__device__ __forceinline__ void mark(uint32_t& mw, uint32_t& mwi, uint32_t* m, uint32_t rel) {
    const uint32_t wi = rel >> 5;
    if (wi != mwi) {
        m[mwi] = mw;
        mw = 0;
        mwi = wi;
    }
    mw |= 1u << (rel & 31);
}

// own segment: tokens from `my0` while the token start lies before my0 + kSeg.
// The loop runs in lock step over the warp (one token per lane per step).
__device__ uint32_t seg_own(const WarpSmem& S, BitIn& b, uint64_t my0, uint32_t* m, uint32_t* tb, uint32_t& n,
                            uint64_t& stop, uint32_t& ev) {
    uint32_t mw = 0, mwi = 0;
    uint32_t st = PS_OK;
    const uint32_t p0 = (uint32_t)my0;
    bool go = true;
    while (__any_sync(FULL, go)) {
        if (!go) continue;
        const uint32_t rel = (uint32_t)(b.wi * 32u - b.cnt) - p0;
        if (rel >= kSeg) {
            go = false;
            continue;
        }
        if (rel < kSyncW) mark(mw, mwi, m, rel);
        if (n + 2 > kTokCap) {
            st = PS_CAP;
            go = false;
            continue;
        }
        uint32_t t0, t1, l1;
        const int r = lane_token<false>(S, b, t0, t1, l1);
        if (r <= LT_TWO) {
            tb[n++] = t0;
            if (r == LT_TWO) {
                if (rel + l1 < kSyncW) mark(mw, mwi, m, rel + l1);
                tb[n++] = t1;
            }
        } else {
            st = r == LT_EOB ? PS_EOB : PS_ERR;
            ev = n;
            go = false;
        }
    }
    m[mwi] = mw;
    stop = b.pos();
    return st;
}

// continuation into the next segment until the parse meets one of its token
// starts (lock step; lanes with nothing to do idle)
__device__ uint32_t seg_next(const WarpSmem& S, BitIn& b, bool active, uint64_t nx0, const uint32_t* nm, uint32_t* tb,
                             uint32_t n, uint32_t& n2, uint64_t& q, uint32_t& ev) {
    const uint32_t p0 = (uint32_t)nx0;
    uint32_t st = PS_NOSYNC;
    bool go = active;
    while (__any_sync(FULL, go)) {
        if (!go) continue;
        const uint32_t rel = (uint32_t)(b.wi * 32u - b.cnt) - p0;
        if (rel >= kSyncW || n + n2 + 2 > kTokCap) {
            st = PS_NOSYNC;
            go = false;
            continue;
        }
        if ((nm[rel >> 5] >> (rel & 31)) & 1u) {
            st = PS_SYNC;
            go = false;
            continue;
        }
        uint32_t t0, t1, l1;
        const int r = lane_token<false>(S, b, t0, t1, l1);
        if (r <= LT_TWO) {
            tb[n + n2++] = t0;
            if (r == LT_TWO) tb[n + n2++] = t1;
        } else {
            ev = n2;
            st = r == LT_EOB ? PS_EOB : PS_ERR;
            go = false;
        }
    }
    q = b.pos();
    return st;
}

// Stage entries of exec_range: kEntryRes | symbol when resolved; else the
// index of the source in the same pass, or kEntryCross | its index in the
// previous pass.
constexpr uint32_t kEntryRes = 0x10000u, kEntryCross = 0x20000u;

struct PassMasks {
    uint32_t am, hm, cm, om;   // bit u: async copy, its upper half, cross entry, open in-pass pointer
    uint32_t neg;              // a source lies before the part start (a placeholder)
    uint32_t bm, bx;           // bit u: the async copy holds a tail byte; bits 2u, 2u+1: its byte in the word
};

// The entries of the pass at A (positions A + 8 lane .. + 7) into stage buffer
// b; positions before fin are final in the part's output and are copied
// asynchronously into their entries (the 32-bit word holding the symbol).
template <bool TAIL>
__device__ __forceinline__ PassMasks build_pass(uint32_t* masks, const uint32_t* tokS, const uint32_t* stS,
                                                uint32_t ntok, uint32_t base, uint32_t end, const uint16_t* out,
                                                uint32_t det, uint32_t A, uint32_t fin, int b, int lane) {
    PassMasks m{0, 0, 0, 0, 0, 0, 0};
    uint32_t* buf = masks + 256 * b;
    const uint32_t p0 = A + 8u * (uint32_t)lane;
    if (!(p0 + 8u > base && p0 < end)) {
#pragma unroll
        for (int u = 0; u < 8; ++u) buf[8u * lane + u] = kEntryRes;
        return m;
    }
    const uint32_t sh = (uint32_t)__cvta_generic_to_shared(buf);
    const uint32_t r0 = (p0 > base ? p0 : base) - base;
    uint32_t lo = 0, hi = ntok - 1;                        // last token starting at or before r0
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (stS[mid] <= r0) lo = mid;
        else hi = mid - 1;
    }
    uint32_t ti = lo;
    uint32_t next = ti + 1 < ntok ? stS[ti + 1] : 0xffffffffu;
    uint32_t tk = tokS[ti];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const uint32_t P = p0 + (uint32_t)u;
        const uint32_t slot = 8u * lane + u;
        if (P < base || P >= end) {
            buf[slot] = kEntryRes;
            continue;
        }
        if (P - base >= next) {                            // the next token (tokens are at least 1 long)
            ++ti;
            next = ti + 1 < ntok ? stS[ti + 1] : 0xffffffffu;
            tk = tokS[ti];
        }
        if (!(tk >> 31)) {
            buf[slot] = kEntryRes | (tk & 0xffu);
            continue;
        }
        const int32_t src = (int32_t)P - (int32_t)((tk & 0xffffu) + 1u);
        if (src < 0) {                                     // a placeholder U_j before the part start
            m.neg = 1;
            buf[slot] = kEntryRes | sym_at(out, src);
        } else if ((uint32_t)src < fin) {                  // final: copy its word into the entry
            if (TAIL && (uint32_t)src >= det) {            // a byte of the determined tail
                const uint32_t bo = det + (uint32_t)src;
                cp_async4(sh + 4u * slot, reinterpret_cast<const uint8_t*>(out) + (bo & ~3u));
                m.bm |= 1u << u;
                m.bx |= (bo & 3u) << (2 * u);
            } else {
                cp_async4(sh + 4u * slot, reinterpret_cast<const uint32_t*>(out) + ((uint32_t)src >> 1));
                m.hm |= ((uint32_t)src & 1u) << u;
            }
            m.am |= 1u << u;
        } else if ((uint32_t)src < A) {                    // inside the previous pass
            buf[slot] = kEntryCross | ((uint32_t)src - (A - 256u));
            m.cm |= 1u << u;
        } else {                                           // inside this pass
            buf[slot] = (uint32_t)src - A;
            m.om |= 1u << u;
        }
    }
    return m;
}

// Execution modes of a part's blocks: kPlain, u16 symbols only; kTail, with the determined tail: an upper
// bound on the part's last placeholder is kept, and positions at or after OutState::det (once set) are
// bytes.  Two instantiations keep the tail's checks out of the plain decoding loop; one instantiation serves
// every block of the tail option, so warps in different parts run the same code.
enum : int { kPlain = 0, kTail = 1 };

// A lane's 8 resolved entries (positions p0 .. p0 + 7; the low 16 bits are the symbols) into the part's
// output, the positions inside [base, end) only: one 16-byte store of u16 symbols, or one 8-byte store of
// bytes in the determined tail.
template <bool TAIL>
__device__ __forceinline__ void store8(const OutState& o, uint16_t* out, const uint32_t* e, uint32_t p0, uint32_t base,
                                       uint32_t end) {
    const bool all = p0 >= base && p0 + 8u <= end;
    if (TAIL && p0 >= o.det) {
        uint8_t* t = tail_bytes(o);
        if (all) {
            uint2 v;
            v.x = (e[0] & 0xffu) | ((e[1] & 0xffu) << 8) | ((e[2] & 0xffu) << 16) | (e[3] << 24);
            v.y = (e[4] & 0xffu) | ((e[5] & 0xffu) << 8) | ((e[6] & 0xffu) << 16) | (e[7] << 24);
            *reinterpret_cast<uint2*>(t + p0) = v;
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t P = p0 + (uint32_t)u;
                if (P >= base && P < end) t[P] = (uint8_t)e[u];
            }
        }
    } else if (all) {
        uint4 v;
        v.x = (e[0] & 0xffffu) | (e[1] << 16);
        v.y = (e[2] & 0xffffu) | (e[3] << 16);
        v.z = (e[4] & 0xffffu) | (e[5] << 16);
        v.w = (e[6] & 0xffffu) | (e[7] << 16);
        *reinterpret_cast<uint4*>(out + p0) = v;
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t P = p0 + (uint32_t)u;
            if (P >= base && P < end) out[P] = (uint16_t)e[u];
        }
    }
}

// Writes up to 256 consecutive tokens of the block (lane j loads tokens
// 8j..8j+7).  Output positions go in passes of 256, lane l taking 8
// consecutive ones (one 16-byte store); a position inside a match takes its
// source: a source before the pass (the part's output so far,
// or a placeholder U_j before the part start) is loaded; a source inside the
// pass is resolved by pointer jumping over the pass's entries in shared memory
// (overlapping copies included, with no division).
// PIPE: the passes are pipelined (the next pass's final sources copied
// asynchronously while a pass resolves); else one pass at a time with direct
// loads.  k_sync always takes the second (its block-start search leaves fewer
// registers); k_inflate takes either (KParams::pipe): which is faster depends
// on the data (how far back the sources lie), so the autotuner can choose.
template <bool PIPE, int MODE>
__device__ __forceinline__ int exec_range(WarpSmem& S, OutState& o, const uint32_t* tks, uint32_t ntok, bool check,
                                          uint64_t& block_n, int lane) {
    uint32_t t[8], L[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t idx = 8u * lane + i;
        t[i] = idx < ntok ? tks[idx] : 0u;
        L[i] = idx < ntok ? ((t[i] >> 16) & 0x1ffu) : 0u;
        sum += L[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t x = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += x;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t base = (uint32_t)o.n;
    if ((uint64_t)base + total > o.cap) return CE_OVERFLOW;
    if (check) {
        bool bad = false;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (L[i] && !(t[i] >> 31) && !allowed_has(S.allowed, t[i] & 0xffu)) bad = true;
        if (__any_sync(FULL, bad)) return CE_BYTE;
    }
    if (total == 0) return CE_OK;
    uint32_t* tokS = S.masks + 512;                        // the batch's tokens
    uint32_t* stS = S.masks + 768;                         // their output offsets from base
    uint32_t s0 = incl - sum;
    uint16_t* out = o.sym;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t idx = 8u * lane + i;
        if (idx < ntok) {
            tokS[idx] = t[i];
            stS[idx] = s0;
            // a match's source before the batch is final already: bring its line toward L2 now, so the
            // passes below find it there
            const int32_t src = (int32_t)(base + s0) - (int32_t)((t[i] & 0xffffu) + 1u);
            if ((t[i] >> 31) && src >= 0 && (uint32_t)src < base) {
                const void* a = (MODE == kTail && (uint32_t)src >= o.det) ? (const void*)(tail_bytes(o) + src)
                                                                         : (const void*)(out + src);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
        }
        s0 += L[i];
    }
    __syncwarp();
    bool bad = false;
    const uint32_t end = base + total;
    if constexpr (PIPE) {
    // Passes over [A, A + 256) with A a multiple of 8; lane l takes positions A + 8l .. A + 8l + 7.  A pass's
    // entries live in one of two stage buffers of 256 words: kRes | symbol when resolved, else the index of
    // the source inside the same pass (strictly earlier), or kCross | index of the source in the previous
    // pass.  While pass j is resolved, pass j + 1 is built: each of its sources that is final already (before
    // pass j: earlier passes and batches) is copied asynchronously -- the 32-bit word holding the symbol,
    // straight into the source's entry -- so those loads overlap pass j's work.  Pointer jumping (each entry
    // replaced by the entry it points to) then resolves a pass; its successor's cross entries are read from
    // it next, before its buffer is reused.
    constexpr uint32_t kRes = kEntryRes;
    int cur = 0;
    uint32_t A = base & ~7u;
    const uint32_t det = o.det;
    PassMasks m = build_pass<MODE == kTail>(S.masks, tokS, stS, ntok, base, end, out, det, A, base, cur, lane);
    uint32_t neg = m.neg;
    cp_async_commit();
    for (;;) {
        const uint32_t A1 = A + 256u;
        const bool more = A1 < end;
        PassMasks m1{0, 0, 0, 0, 0, 0, 0};
        if (more)
            m1 = build_pass<MODE == kTail>(S.masks, tokS, stS, ntok, base, end, out, det, A1, A > base ? A : base,
                                           cur ^ 1, lane);
        neg |= m1.neg;
        cp_async_commit();
        cp_async_wait<1>();                                // this pass's copies (this lane's) have landed
        uint32_t* buf = S.masks + 256 * cur;
        const uint32_t p0 = A + 8u * (uint32_t)lane;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if ((m.am >> u) & 1u) {
                const uint32_t w = buf[8u * lane + u];
                const uint32_t v = (MODE == kTail && ((m.bm >> u) & 1u))
                                       ? ((w >> (8u * ((m.bx >> (2 * u)) & 3u))) & 0xffu)
                                       : (((m.hm >> u) & 1u) ? (w >> 16) : (w & 0xffffu));
                buf[8u * lane + u] = kRes | v;
            }
        __syncwarp();
        uint32_t e[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) e[u] = buf[8u * lane + u];
        uint32_t open = m.om;
        while (__any_sync(FULL, open != 0)) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if ((open >> u) & 1u) e[u] = buf[e[u]];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if ((open >> u) & 1u) {
                    buf[8u * lane + u] = e[u];
                    if (e[u] & kRes) open &= ~(1u << u);
                }
            __syncwarp();
        }
        if (more) {                                        // the next pass's sources in this one
            uint32_t* nb = S.masks + 256 * (cur ^ 1);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if ((m1.cm >> u) & 1u) nb[8u * lane + u] = buf[nb[8u * lane + u] & 0xffu];
        }
        store8<MODE == kTail>(o, out, e, p0, base, end);
        if (MODE == kTail && o.det == 0xffffffffu) track_placeholders(o, e, A, end);
        __syncwarp();                                      // this pass is final; its buffer may be reused
        if (!more) break;
        A = A1;
        cur ^= 1;
        m = m1;
    }
    cp_async_wait<0>();
    if (neg) {
        o.neg = true;
        if (o.known) bad = true;
    }
    } else {
    uint32_t* stage = S.masks;                             // 256 entries: the positions of one pass
    // passes over [A, A + 256) with A a multiple of 8; lane l takes positions A + 8l .. A + 8l + 7.  A source
    // before max(A, base) is final (earlier passes, earlier batches, or a placeholder before the part start)
    // and is loaded; a source inside the pass is a pointer to its stage entry, strictly earlier, so pointer
    // jumping (each entry replaced by the entry it points to) ends with every entry a symbol.  An entry is
    // 0x10000 | symbol when resolved, else the pass index of its source.
    for (uint32_t A = base & ~7u; A < end; A += 256u) {
        const uint32_t p0 = A + 8u * (uint32_t)lane;
        const uint32_t lo_pos = A > base ? A : base;       // first position of the pass that is this batch's
        uint32_t e[8];
        uint32_t open = 0;                                 // bit u: e[u] still a pointer
        if (p0 + 8u > base && p0 < end) {
            const uint32_t r0 = (p0 > base ? p0 : base) - base;
            uint32_t lo = 0, hi = ntok - 1;                // last token starting at or before r0
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (stS[mid] <= r0) lo = mid;
                else hi = mid - 1;
            }
            uint32_t ti = lo;
            uint32_t next = ti + 1 < ntok ? stS[ti + 1] : 0xffffffffu;
            uint32_t tk = tokS[ti];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t P = p0 + (uint32_t)u;
                e[u] = 0x10000u;
                if (P < base || P >= end) continue;
                if (P - base >= next) {                    // the next token (tokens are at least 1 long)
                    ++ti;
                    next = ti + 1 < ntok ? stS[ti + 1] : 0xffffffffu;
                    tk = tokS[ti];
                }
                if (!(tk >> 31)) {
                    e[u] = 0x10000u | (tk & 0xffu);
                    continue;
                }
                const int32_t src = (int32_t)P - (int32_t)((tk & 0xffffu) + 1u);
                if (src < (int32_t)lo_pos) {
                    if (src < 0) {
                        if (o.known) bad = true;
                        o.neg = true;
                    }
                    e[u] = 0x10000u | (MODE == kTail ? sym_get(o, src) : sym_at(out, src));
                } else {
                    e[u] = (uint32_t)src - A;
                    open |= 1u << u;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) e[u] = 0x10000u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) stage[8u * lane + u] = e[u];
        __syncwarp();
        while (__any_sync(FULL, open != 0)) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if ((open >> u) & 1u) e[u] = stage[e[u]];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if ((open >> u) & 1u) {
                    stage[8u * lane + u] = e[u];
                    if (e[u] & 0x10000u) open &= ~(1u << u);
                }
            __syncwarp();
        }
        store8<MODE == kTail>(o, out, e, p0, base, end);
        if (MODE == kTail && o.det == 0xffffffffu) track_placeholders(o, e, A, end);
        __syncwarp();                                      // this pass is final for the next one
    }
    }
    if (__any_sync(FULL, bad)) return CE_DIST;
    o.n = base + total;
    block_n += total;
    return CE_OK;
}

template <bool PIPE, int MODE>
__device__ int par_block(WarpSmem& S, uint32_t* tokbuf, BitIn& br, OutState& o, bool check, uint64_t max_block,
                         uint64_t end_bit, uint64_t& block_n, int lane) {
    uint32_t* tb = tokbuf + (uint64_t)lane * kTokCap;
    uint32_t* mymask = S.masks + 32 * lane;
    for (;;) {
        const uint64_t start = br.pos();
        const uint64_t my0 = start + (uint64_t)lane * kSeg;
#pragma unroll
        for (int w = 0; w < 32; ++w) mymask[w] = 0;
        {   // bring the lane's segment (and the continuation window) into L1
            const uint64_t b0 = my0 >> 3, b1 = (my0 + kSeg + kSyncW + 128) >> 3;
            for (uint64_t a = b0 & ~127ull; a < b1; a += 128)
                if (a < br.nbytes) asm volatile("prefetch.global.L1 [%0];" ::"l"(br.b + a));
        }
        BitIn b = br;
        b.seek(my0);
        uint32_t n = 0, ev1 = 0, ev2 = 0, n2 = 0;
        uint64_t stop = 0, q = 0;
        const uint32_t st1 = seg_own(S, b, my0, mymask, tb, n, stop, ev1);
        __syncwarp();
        const uint32_t st2 = seg_next(S, b, st1 == PS_OK && lane < 31, my0 + kSeg, S.masks + 32 * ((lane + 1) & 31), tb,
                                      n, n2, q, ev2);
        __syncwarp();
        // the chain of meeting points, lane by lane (uniform)
        uint32_t skip = 0, my_vs = 0, my_ve = 0;
        int last = -1;
        bool block_end = false;
        int err = CE_OK;
        uint64_t round_end = 0;
        for (int k = 0; k < 32; ++k) {
            const uint32_t s1 = __shfl_sync(FULL, st1, k), nk = __shfl_sync(FULL, n, k);
            uint32_t ve;
            bool stop_here = true;
            if (s1 == PS_EOB) {
                ve = __shfl_sync(FULL, ev1, k);
                block_end = true;
                round_end = shfl64(stop, k);
            } else if (s1 == PS_ERR) {
                err = CE_DATA;
                ve = skip;
            } else if (s1 == PS_CAP || k == 31) {
                ve = nk;
                round_end = shfl64(stop, k);
            } else {
                const uint32_t s2 = __shfl_sync(FULL, st2, k), n2k = __shfl_sync(FULL, n2, k);
                const uint64_t qk = shfl64(q, k);
                if (s2 == PS_EOB) {
                    ve = nk + __shfl_sync(FULL, ev2, k);
                    block_end = true;
                    round_end = qk;
                } else if (s2 == PS_ERR) {
                    err = CE_DATA;
                    ve = skip;
                } else if (s2 == PS_NOSYNC) {
                    ve = nk + n2k;
                    round_end = qk;
                } else {                                   // met lane k+1 at qk
                    ve = nk + n2k;
                    stop_here = false;
                }
                if (!stop_here) {
                    // lane k+1's tokens that start before qk are not the block's
                    const uint32_t rel = (uint32_t)(qk - (start + (uint64_t)(k + 1) * kSeg));
                    const uint32_t w = S.masks[32 * (k + 1) + lane];
                    const uint32_t below = (uint32_t)lane < (rel >> 5) ? __popc(w)
                                         : ((uint32_t)lane == (rel >> 5) ? __popc(w & ((1u << (rel & 31)) - 1u)) : 0u);
                    const uint32_t nskip = __reduce_add_sync(FULL, below);
                    if (lane == k) {
                        my_vs = skip;
                        my_ve = ve;
                    }
                    skip = nskip;
                    continue;
                }
            }
            if (lane == k) {
                my_vs = skip;
                my_ve = ve;
            }
            last = k;
            break;
        }
        if (err) return err;
        // the block's tokens of this round, in order: lane ranges one after another
        for (int k = 0; k <= last; ++k) {
            const uint32_t vs = __shfl_sync(FULL, my_vs, k), ve = __shfl_sync(FULL, my_ve, k);
            const uint32_t* rng = tokbuf + (uint64_t)k * kTokCap;
            for (uint32_t x = vs; x < ve; x += 256) {
                const int e = exec_range<PIPE, MODE>(S, o, rng + x, ve - x < 256 ? ve - x : 256, check, block_n, lane);
                if (e) return e;
                if (max_block && block_n >= max_block) return CE_SIZE;
            }
        }
        __syncwarp();
        if (round_end > end_bit) return CE_TRUNC;
        br.seek(round_end);
        if (block_end) return CE_OK;
    }
}

__device__ int stored_block(BitIn& br, OutState& o, bool check, const uint32_t* allowed, uint64_t end_bit,
                            uint64_t& block_n, int lane) {
    const uint64_t p = (br.pos() + 7) & ~7ull;
    if (p + 32 > end_bit) return CE_TRUNC;
    const uint64_t byte = p >> 3;
    const uint8_t* g = br.b;
    const uint32_t len = (uint32_t)__ldg(g + byte) | ((uint32_t)__ldg(g + byte + 1) << 8);
    const uint32_t nlen = (uint32_t)__ldg(g + byte + 2) | ((uint32_t)__ldg(g + byte + 3) << 8);
    if ((len ^ 0xffffu) != nlen) return CE_DATA;
    if (p + 32 + 8ull * len > end_bit) return CE_TRUNC;
    if (o.n + len > o.cap) return CE_OVERFLOW;
    bool bad = false;
    for (uint32_t j = lane; j < len; j += 32) {
        const uint32_t v = __ldg(g + byte + 4 + j);
        if (check && !allowed_has(allowed, v)) bad = true;
        const uint64_t P = o.n + j;
        if (P >= o.det) tail_bytes(o)[P] = (uint8_t)v;
        else o.sym[P] = (uint16_t)v;
    }
    if (__any_sync(FULL, bad)) return CE_BYTE;
    o.n += len;
    block_n += len;
    br.seek(p + 32 + 8ull * len);
    __syncwarp();
    return CE_OK;
}

// one block.  candidate: the block must be a non-final dynamic block (the
// block-start checks); min/max_block bound its size; check: its literals must
// be allowed bytes.  Huffman blocks are decoded by the whole warp in parallel
// (par_block); a candidate block start first runs a short serial prefix, so
// that false candidates fail after a few tokens.
template <bool PIPE, int MODE = kPlain>
__device__ int one_block(WarpSmem& S, uint32_t* tokbuf, BitIn& br, OutState& o, bool check, uint64_t min_block,
                         uint64_t max_block, bool candidate, uint64_t end_bit, uint32_t& final, int lane) {
    br.refill();
    final = br.peek(1);
    const uint32_t type = br.peek(3) >> 1;
    br.drop(3);
    if (br.pos() > end_bit) return CE_TRUNC;
    if (candidate) {
        if (final) return CE_FINAL;
        if (type != 2) return CE_TYPE;
    }
    uint64_t block_n = 0;
    int st;
    if (type == 0) {
        st = stored_block(br, o, check, S.allowed, end_bit, block_n, lane);
    } else if (type == 3) {
        st = CE_DATA;
    } else {
        if (type == 1) {
            if (S.table_kind != 1) build_fixed(S, lane);
            st = CE_OK;
        } else {
            st = read_dynamic<false>(S, br, lane);
            if (st == CE_OK && br.pos() > end_bit) st = CE_TRUNC;
        }
        if (st == CE_OK && candidate) {
            st = huff_block(S, br, o, check, max_block, end_bit, block_n, lane, 64);
            st = st == CE_MORE ? CE_MORE : (st == CE_OK ? CE_OK + 1000 : st);
        }
        if (st == CE_OK || st == CE_MORE)
            st = par_block<PIPE, MODE>(S, tokbuf, br, o, check, max_block, end_bit, block_n, lane);
        else if (st == CE_OK + 1000)
            st = CE_OK;
    }
    if (st == CE_OK && max_block && block_n >= max_block) st = CE_SIZE;
    if (st == CE_OK && block_n < min_block) st = CE_SIZE;
    return st;
}

// ---------------------------------------------------------------------------
// block-start candidates.  Per bit offset p, in order of cost:
//  1. BFINAL = 0, BTYPE = 10, HLIT <= 29, HDIST <= 29: bit-parallel over the
//     32 offsets of a lane;
//  2. the code-length code is complete: sum of 2^-l over its lengths is 1,
//     from a 512-entry table of three-field sums;
//  3. the whole dynamic header is valid (the checks of read_dynamic<true>),
//     32 listed offsets at a time, one per lane (hdr_ok_lane).
// The full block decode then follows in k_sync, lowest offset first.  Stages
// 1-3 are implied by the complete checks, so no offset that passes those is
// dropped here.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi, uint32_t s) { return __funnelshift_r(lo, hi, s); }

// 3-field Kraft sums in units of 2^-7: kraft3[a | b << 3 | c << 6]
__device__ __forceinline__ uint32_t kraft1(uint32_t l) { return l ? (128u >> l) : 0u; }

__device__ uint32_t cl_complete(const uint16_t* kraft3, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t k) {
    // bits of the window from offset k + 13 (HCLEN) onward; k < 32
    const uint32_t q = k + 13;                   // < 45
    const uint32_t a0 = q < 32 ? fsr(w0, w1, q) : fsr(w1, w2, q - 32);
    const uint32_t hclen = (a0 & 15u) + 4;
    const uint32_t q1 = q + 4, q2 = q + 34;      // 10 fields, then 9 fields
    const uint32_t f1 = q1 < 32 ? fsr(w0, w1, q1) : fsr(w1, w2, q1 - 32);
    const uint32_t f2 = q2 < 64 ? fsr(w1, w2, q2 - 32) : fsr(w2, w3, q2 - 64);
    const uint64_t fields = (uint64_t)(f1 & 0x3fffffffu) | ((uint64_t)(f2 & 0x7ffffffu) << 30);
    const uint64_t x = fields & ((1ull << (3 * hclen)) - 1ull);
    uint32_t kr = 0;
#pragma unroll
    for (int g = 0; g < 7; ++g) kr += kraft3[(x >> (9 * g)) & 511u];
    return kr == 128u;
}

// The whole dynamic-header check of one candidate by one lane, with no
// shared state (the checks of read_dynamic<true>): the code-length code is
// decoded canonically from its lengths -- code length by comparing the next
// 7 bits (MSB first) against the left-aligned limits of lengths 1..6, symbol
// from the lengths' offsets and the symbols sorted by (length, value) -- and
// the literal/length and distance length sets are checked as they are read.
// The caller has already checked that the code-length code is complete.
__device__ bool hdr_ok_lane(const FileDesc& F, uint64_t p) {
    BitIn br;
    br.setup(F.gz, F.gz_len);
    br.seek(p + 3);
    br.refill();
    const uint32_t hlit = br.peek(5) + 257;
    br.drop(5);
    const uint32_t hdist = br.peek(5) + 1;
    br.drop(5);
    const uint32_t hclen = br.peek(4) + 4;
    br.drop(4);
    if (hlit > 286 || hdist > 30) return false;
    uint64_t lens = 0;                                     // 3 bits per code-length symbol 0..18
    br.refill();
#pragma unroll
    for (uint32_t k = 0; k < 19; ++k) {
        if (k == 10) br.refill();
        if (k < hclen) {
            lens |= (uint64_t)br.peek(3) << (3 * c_clorder[k]);
            br.drop(3);
        }
    }
    uint64_t cnt8 = 0;                                     // symbols of each length (8 bits per length)
#pragma unroll
    for (int t = 0; t < 19; ++t) {
        const uint32_t l = (uint32_t)(lens >> (3 * t)) & 7u;
        if (l) cnt8 += 1ull << (8 * l);
    }
    uint32_t first = 0, offs = 0, limA = 0, limB = 0xffff0000u;
    uint64_t base8 = 0, next8 = 0;
#pragma unroll
    for (int l = 1; l <= 7; ++l) {
        const uint32_t cprev = (uint32_t)(cnt8 >> (8 * (l - 1))) & 0xffu, c = (uint32_t)(cnt8 >> (8 * l)) & 0xffu;
        first = (first + cprev) << 1;                     // first code of length l
        const uint32_t lim = (first + c) << (7 - l);      // left-aligned end of the length-l codes
        if (l <= 4) limA |= (lim > 255u ? 255u : lim) << (8 * (l - 1));
        else if (l <= 6) limB |= (lim > 255u ? 255u : lim) << (8 * (l - 5));
        base8 |= (uint64_t)((offs - first + 128u) & 0xffu) << (8 * l);
        next8 |= (uint64_t)offs << (8 * l);
        offs += c;
    }
    uint64_t slo = 0, shi = 0;                             // symbols sorted by (length, value), 5 bits each
#pragma unroll
    for (int t = 0; t < 19; ++t) {
        const uint32_t l = (uint32_t)(lens >> (3 * t)) & 7u;
        if (l) {
            const uint32_t i = (uint32_t)(next8 >> (8 * l)) & 0xffu;
            next8 += 1ull << (8 * l);
            if (i < 12) slo |= (uint64_t)t << (5 * i);
            else shi |= (uint64_t)t << (5 * (i - 12));
        }
    }
    const uint32_t total = hlit + hdist;
    uint32_t i = 0, prev = 0, kl = 0, kd = 0, nl = 0, nd = 0, ml = 0, md = 0;
    bool eob = false;
    while (i < total) {
        br.refill();
        const uint32_t v = __brev(br.peek(7)) >> 25;      // the next 7 bits, first bit most significant
        const uint32_t vv = v * 0x01010101u;
        const uint32_t l = 1u + ((__popc(__vcmpgeu4(vv, limA)) + __popc(__vcmpgeu4(vv, limB))) >> 3);
        const uint32_t ix = ((uint32_t)(base8 >> (8 * l)) & 0xffu) - 128u + (v >> (7 - l));
        const uint32_t sym = ix < 12 ? (uint32_t)(slo >> (5 * ix)) & 31u : (uint32_t)(shi >> (5 * (ix - 12))) & 31u;
        br.drop(l);
        uint32_t rep = 1, val;
        if (sym < 16) {
            val = sym;
            prev = sym;
        } else if (sym == 16) {
            if (i == 0) return false;
            val = prev;
            rep = 3 + br.peek(2);
            br.drop(2);
        } else if (sym == 17) {
            val = 0;
            rep = 3 + br.peek(3);
            br.drop(3);
            prev = 0;
        } else {
            val = 0;
            rep = 11 + br.peek(7);
            br.drop(7);
            prev = 0;
        }
        if (i + rep > total) return false;
        if (val) {
            const uint32_t e2 = i + rep;
            const uint32_t nlit = i < hlit ? ((e2 < hlit ? e2 : hlit) - i) : 0u;
            const uint32_t ndst = rep - nlit;
            kl += nlit * (32768u >> val);
            kd += ndst * (32768u >> val);
            nl += nlit;
            nd += ndst;
            if (nlit && val > ml) ml = val;
            if (ndst && val > md) md = val;
            if (i <= 256 && 256 < e2) eob = true;
            if (kl > 32768u || kd > 32768u) return false;
        }
        i += rep;
    }
    if (!eob) return false;
    if (!(kl == 32768u || (nl == 1 && ml == 1))) return false;
    if (!(kd == 32768u || nd == 0 || (nd == 1 && md == 1))) return false;
    return br.pos() <= F.end_bit;
}

// Search state of a part, kept by the caller between candidates: the next
// window to filter, and a list of up to 32 filtered offsets (one per lane,
// relative to the part's scan start) whose header checks are done.
struct ScanState {
    uint64_t next;       // first bit not yet filtered
    uint64_t mine;       // this lane's list entry
    uint32_t pass;       // list entries whose whole header passed, not yet returned
};

__device__ __forceinline__ void scan_begin(ScanState& st, uint64_t lo) {
    st.next = lo;
    st.mine = 0;
    st.pass = 0;
}

// The next block-start candidate at or after the state's position, lowest
// first: windows of 1024 bits are filtered (each lane tests 32 offsets with
// bit masks, then the completeness of the code-length code); the survivors
// are gathered, one per lane, until 32 are listed or the range ends, and then
// all whole-header checks of the list run at once, one per lane.
__device__ uint64_t find_candidate(const uint16_t* kraft3, const FileDesc& F, uint64_t lo, uint64_t hi, int lane,
                                   ScanState& st) {
    BitIn w;
    w.setup(F.gz, F.gz_len);
    if (hi > F.end_bit) hi = F.end_bit;
    for (;;) {
        if (st.pass) {
            const int k = __ffs(st.pass) - 1;
            st.pass &= st.pass - 1;
            return lo + shfl64(st.mine, k);
        }
        if (st.next >= hi) return kNone;
        uint32_t n = 0;                                    // entries listed
        while (n < 32 && st.next < hi) {
            const uint64_t T = st.next & ~1023ull;
            const uint64_t base = T + 32ull * (uint64_t)lane;
            const uint64_t wi = base >> 5;
            const uint32_t w0 = w.word(wi), w1 = w.word(wi + 1), w2 = w.word(wi + 2), w3 = w.word(wi + 3);
            const uint64_t x = (uint64_t)w0 | ((uint64_t)w1 << 32);
            uint64_t y = ~x & ~(x >> 1) & (x >> 2);                // BFINAL = 0, BTYPE = 10
            y &= ~((x >> 4) & (x >> 5) & (x >> 6) & (x >> 7));     // HLIT <= 29
            y &= ~((x >> 9) & (x >> 10) & (x >> 11) & (x >> 12));  // HDIST <= 29
            uint32_t m = (uint32_t)y;
            if (base < st.next) {
                const uint64_t d = st.next - base;
                m = d >= 32 ? 0u : (m & (~0u << d));
            }
            if (base + 32 > hi) m = base >= hi ? 0u : (m & ((1u << (uint32_t)(hi - base)) - 1u));
            uint32_t c = 0;
            for (uint32_t mm = m; mm; mm &= mm - 1) {
                const uint32_t k = __ffs(mm) - 1;
                if (cl_complete(kraft3, w0, w1, w2, w3, k)) c |= 1u << k;
            }
            // list the survivors lowest first (lanes cover increasing offsets) while there is room
            uint64_t resume = T + 1024;
            for (uint32_t bl = __ballot_sync(FULL, c != 0); bl; bl = __ballot_sync(FULL, c != 0)) {
                const int l = __ffs(bl) - 1;
                const uint32_t cl = __shfl_sync(FULL, c, l);
                const uint32_t k = __ffs(cl) - 1;
                const uint64_t pos = T + 32ull * (uint64_t)l + k;
                if (n == 32) {                            // full: this window resumes here
                    resume = pos;
                    break;
                }
                if (lane == l) c &= c - 1;
                if ((uint32_t)lane == n) st.mine = pos - lo;
                ++n;
            }
            st.next = resume < hi ? resume : hi;
        }
        const bool ok = (uint32_t)lane < n && hdr_ok_lane(F, lo + st.mine);
        st.pass = __ballot_sync(FULL, ok);
    }
}

__device__ __forceinline__ WarpSmem& warp_smem() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<WarpSmem*>(smem_raw)[threadIdx.x >> 5];
}

__device__ __forceinline__ void init_smem(WarpSmem& S, const KParams& p, int lane) {
    if (lane < 8) S.allowed[lane] = p.allowed[lane];
    if (lane == 0) S.table_kind = 0;
    __syncwarp();
}

// pass-1 CTA shapes: warps per block and the blocks per SM the register
// budget is set for (about 20 resident warps per SM, 96 registers a thread)
constexpr int pass1_min_blocks(int wpb) { return wpb == 2 ? 10 : (wpb == 4 ? 5 : 2); }

// Work queue of the pass-1 kernels: each resident warp takes the next queue
// position until the parts run out, so parts of uneven work (many members of
// different sizes in one launch) balance over the warps.  Position q holds
// part order[q] (the parts with the most expected output first, so that the
// short ones fill the end of the launch), or part q without an order.  The
// counter is zeroed on the stream before each launch.
__device__ __forceinline__ int next_part(uint32_t* queue, int lane) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(queue, 1u);
    return (int)min(__shfl_sync(FULL, c, 0), 0x7fffffffu);
}

// ---------------------------------------------------------------------------
// k_sync: block start of each part and its first block; k_inflate: the rest of each part
// ---------------------------------------------------------------------------
// The block start of part c and its first block (Section "Detection of DEFLATE block start positions").
__device__ void sync_part(const uint16_t* kraft3, WarpSmem& S, uint32_t* tok, const FileDesc& F, ChunkDesc& C,
                          uint16_t* symbuf, const KParams& p, int lane) {
    init_smem(S, p, lane);
    OutState o{symbuf + C.sym_base, C.cap, 0, C.index == 0 && C.lo <= F.s0_bit, false};
    BitIn br;
    br.setup(F.gz, F.gz_len);
    uint32_t state = CS_EMPTY, err = CE_OK, final = 0;
    uint64_t sync = kNone, resume = 0;
    if (C.disabled) {
        state = CS_EMPTY;
    } else if (o.known || C.given) {          // the member start (empty context) or a known block start
        br.seek(C.lo);
        const int st = one_block<false>(S, tok, br, o, false, 0, 0, false, F.end_bit, final, lane);
        sync = C.lo;
        resume = br.pos();
        if (st) {
            state = CS_ERROR;
            err = (uint32_t)st;
        } else {
            state = CS_FOUND;
        }
    } else {
        ScanState scan;
        scan_begin(scan, C.lo);
        for (;;) {
            const uint64_t cand = find_candidate(kraft3, F, C.lo, C.hi, lane, scan);
            if (cand == kNone) break;
            br.seek(cand);
            o.n = 0;
            o.neg = false;
            const int st = one_block<false>(S, tok, br, o, true, p.min_block, p.max_block, true, F.end_bit, final,
                                            lane);
            if (st == CE_OK) {
                state = CS_FOUND;
                sync = cand;
                resume = br.pos();
                break;
            }
            if (st == CE_OVERFLOW) {             // the candidate's block does not fit: cannot judge it here
                state = CS_ERROR;
                err = CE_OVERFLOW;
                sync = cand;
                break;
            }
        }
    }
    const bool neg = __any_sync(FULL, o.neg);
    if (lane == 0) {
        C.err = err;
        C.sync = sync;
        C.resume = resume;
        C.n = state == CS_FOUND ? o.n : 0;
        C.nph = 0;
        // a bound on one past the last placeholder: the first block's end (the member start has none)
        C.last_ph = (state == CS_FOUND && !o.known) ? o.n : 0;
        C.det = kNone;
        C.anyph = neg && state == CS_FOUND;
        C.blocks = state == CS_FOUND ? 1u : 0u;
        C.final = final && state == CS_FOUND;
        C.confirmed = (state == CS_FOUND && (o.known || C.given || final || p.confirm_blocks == 0)) ? 1u : 0u;
        C.end = resume;
        C.state = state;
    }
    __syncwarp();
}

// Where part c's decoding stops: the start of the next part that holds one (`sync` is final after k_sync and
// never written by k_inflate, whose other warps rewrite `state`); parts merged into their predecessor hold
// none.
__device__ __forceinline__ uint64_t find_stop(const FileDesc& F, const ChunkDesc* chunks, int c, uint64_t stop_hint) {
    for (int j = c + 1; j < F.chunk0 + F.nchunks; ++j) {
        const uint64_t sj = chunks[j].sync;
        if (sj != kNone) return sj;
    }
    return stop_hint;
}

// Pass 1 of part c from the end of its first block up to the next part's block start.
template <bool PIPE>
__device__ void inflate_part(WarpSmem& S, uint32_t* tok, const FileDesc* __restrict__ files, ChunkDesc* chunks, int c,
                             uint16_t* symbuf, const KParams& p, int lane) {
    ChunkDesc& C = chunks[c];
    if (C.state != CS_FOUND) return;
    if (C.probe) {                    // a streamed segment's end: the block start found is all it gives
        if (lane == 0) {
            C.state = CS_DONE;
            C.n = 0;
            C.anyph = 0;
            C.blocks = 0;
            C.final = 0;
            C.confirmed = 0;
            C.end = C.sync;
        }
        __syncwarp();
        return;
    }
    const FileDesc& F = files[C.file];
    const uint64_t stop = find_stop(F, chunks, c, C.stop_hint);
    OutState o{symbuf + C.sym_base, C.cap, C.n, C.index == 0 && C.sync == F.s0_bit, false};
    o.det = C.det == kNone ? 0xffffffffu : (uint32_t)C.det;
    o.last_ph = (uint32_t)C.last_ph;
    // the determined tail when the configuration asks for it; decoding from a bit offset keeps every symbol
    // as u16 (its caller asks for the symbols themselves)
    const bool tail_ok = p.tail && F.mode != 1;
    uint32_t blocks = C.blocks, final = C.final, err = CE_OK, confirmed = C.confirmed;
    uint64_t end = C.resume;
    // the confirmation (Section "Detection of DEFLATE block start positions") covers the start's block and
    // the confirm_blocks blocks after it; they are decoded with the literal checks
    const uint32_t window = (uint32_t)p.confirm_blocks + 1u;
    if (final) {
        if (stop != kNone && !F.open_end) err = CE_CHAIN;
    } else if (!(stop != kNone && C.resume == stop) || (C.confirm_ext && !confirmed)) {
        init_smem(S, p, lane);
        BitIn br;
        br.setup(F.gz, F.gz_len);
        br.seek(C.resume);
        // past the stop (confirm_ext): blocks decoded only to finish the confirmation; the part's own
        // output, end and status are those at the stop
        bool past = false;
        uint32_t err_stop = CE_OK;
        uint64_t n_stop = 0, end_stop = 0;
        for (;;) {
            const uint64_t pos = br.pos();
            if (!past && stop != kNone && pos >= stop) {
                err_stop = pos != stop ? (uint32_t)CE_CHAIN : (uint32_t)CE_OK;
                if (!C.confirm_ext || blocks >= window) {
                    err = err_stop;
                    break;
                }
                past = true;
                n_stop = o.n;
                end_stop = pos;
            }
            if (past && blocks >= window) break;
            // no placeholder among the last 32 KiB: none can follow; the rest goes out as bytes
            if (tail_ok && !past && o.det == 0xffffffffu && o.n >= (uint64_t)o.last_ph + kWin)
                o.det = (uint32_t)((o.n + 7) & ~7ull);
            const bool check = !o.known && blocks < window;
            uint32_t fin = 0;
            const int st = tail_ok ? one_block<PIPE, kTail>(S, tok, br, o, check, 0, 0, false, F.end_bit, fin, lane)
                                   : one_block<PIPE, kPlain>(S, tok, br, o, check, 0, 0, false, F.end_bit, fin, lane);
            if (st) {
                err = (check && st != CE_OVERFLOW) ? (uint32_t)CE_CONFIRM : (uint32_t)st;
                break;
            }
            ++blocks;
            if (fin) {
                if (blocks <= window) confirmed = 1;
                if (past) break;
                final = 1;
                if (stop != kNone && !F.open_end) err = CE_CHAIN;   // an open member may end before the next part
                break;
            }
        }
        end = br.pos();
        if (blocks >= window && err != CE_CONFIRM) confirmed = 1;
        if (past) {
            if (err == CE_OK) err = err_stop;
            if (err != CE_CONFIRM && err != CE_OVERFLOW) {
                o.n = n_stop;
                end = end_stop;
            }
        }
    }
    const bool neg = __any_sync(FULL, o.neg);
    if (err == CE_OK && final && F.mode != 2 && !F.open_end) {   // the trailer must follow the final block
        if (((end + 7) >> 3) + 8 != F.gz_len) err = CE_TRAIL;
    }
    if (lane == 0) {
        C.state = err ? CS_ERROR : CS_DONE;
        C.err = err;
        C.n = o.n;
        C.anyph = C.anyph | (neg ? 1u : 0u);
        C.blocks = blocks;
        C.final = final;
        C.confirmed = confirmed;
        C.end = end;
        C.last_ph = o.last_ph;
        C.det = o.det < o.n ? (uint64_t)o.det : kNone;
    }
    __syncwarp();
}

// Work queue over the parts (one per warp at a time), for both kernels.
template <int WPB>
__global__ void __launch_bounds__(32 * WPB, pass1_min_blocks(WPB))
    k_sync(const FileDesc* __restrict__ files, ChunkDesc* chunks, int nchunks, uint16_t* symbuf, uint32_t* tokbuf,
           uint32_t* queue, const uint32_t* __restrict__ order, KParams p) {
    __shared__ uint16_t kraft3[512];
    for (uint32_t v = threadIdx.x; v < 512; v += blockDim.x)
        kraft3[v] = (uint16_t)(kraft1(v & 7) + kraft1((v >> 3) & 7) + kraft1(v >> 6));
    __syncthreads();
    WarpSmem& S = warp_smem();
    const int lane = threadIdx.x & 31;
    uint32_t* tok = tokbuf + (uint64_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kTokPerPart;
    for (;;) {
        const int q = next_part(queue, lane);
        if (q >= nchunks) return;
        const int c = order ? (int)__ldg(order + q) : q;
        sync_part(kraft3, S, tok, files[chunks[c].file], chunks[c], symbuf, p, lane);
    }
}

template <int WPB, bool PIPE>
__global__ void __launch_bounds__(32 * WPB, pass1_min_blocks(WPB))
    k_inflate(const FileDesc* __restrict__ files, ChunkDesc* chunks, int nchunks, uint16_t* symbuf, uint32_t* tokbuf,
              uint32_t* queue, const uint32_t* __restrict__ order, KParams p) {
    WarpSmem& S = warp_smem();
    const int lane = threadIdx.x & 31;
    uint32_t* tok = tokbuf + (uint64_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kTokPerPart;
    for (;;) {
        const int q = next_part(queue, lane);
        if (q >= nchunks) return;
        const int c = order ? (int)__ldg(order + q) : q;
        inflate_part<PIPE>(S, tok, files, chunks, c, symbuf, p, lane);
    }
}

// ---------------------------------------------------------------------------
// k_plan: output offsets, error aggregation, length checks (one block per member)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_plan(FileDesc* files, ChunkDesc* chunks) {
    FileDesc& F = files[blockIdx.x];
    __shared__ uint64_t part[1024];
    __shared__ uint32_t bad, fin;
    __shared__ int any_final;
    const int t = threadIdx.x;
    if (t == 0) {
        bad = 0xffffffffu;
        fin = 0xffffffffu;
        any_final = 0;
    }
    __syncthreads();
    // an open member ends with the first part that decoded its final block; the parts after it lie in
    // what follows the member (the next member, or other data) and are dropped
    if (F.open_end)
        for (int i = t; i < F.nchunks; i += 1024) {
            const ChunkDesc& C = chunks[F.chunk0 + i];
            if (C.state == CS_DONE && C.final) atomicMin(&fin, (uint32_t)i);
        }
    __syncthreads();
    uint64_t carry = F.out_base;
    for (int b0 = 0; b0 < F.nchunks; b0 += 1024) {
        const int c = F.chunk0 + b0 + t;
        uint64_t n = 0;
        if (b0 + t < F.nchunks && (uint32_t)(b0 + t) > fin) {
            chunks[c].state = CS_EMPTY;
        } else if (b0 + t < F.nchunks) {
            ChunkDesc& C = chunks[c];
            if (C.state == CS_DONE) {
                n = C.n;
                if (C.final) atomicOr(&any_final, 1);
            } else if (C.state == CS_ERROR) {
                atomicMin(&bad, (uint32_t)(b0 + t));
            }
        }
        part[t] = n;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {          // inclusive scan
            const uint64_t v = t >= d ? part[t - d] : 0;
            __syncthreads();
            part[t] += v;
            __syncthreads();
        }
        if (b0 + t < F.nchunks) chunks[c].out_off = carry + part[t] - n;
        carry += part[1023];
        __syncthreads();
    }
    if (t == 0) {
        const uint64_t total = carry - F.out_base;
        F.total = total;
        F.bad_chunk = bad;
        F.crc_acc = 0;
        F.member_end = F.gz_len;
        uint32_t st = PGZ_OK;
        if (F.open_end && fin != 0xffffffffu && bad == 0xffffffffu) {   // the member's own trailer
            const uint64_t me = ((chunks[F.chunk0 + fin].end + 7) >> 3) + 8;
            if (me > F.gz_len) {
                st = PGZ_E_DATA;
            } else {
                const uint8_t* tr = F.gz + me - 8;
                F.crc_expect = tr[0] | ((uint32_t)tr[1] << 8) | ((uint32_t)tr[2] << 16) | ((uint32_t)tr[3] << 24);
                F.isize_expect = tr[4] | ((uint32_t)tr[5] << 8) | ((uint32_t)tr[6] << 16) | ((uint32_t)tr[7] << 24);
                F.member_end = me;
            }
        }
        if (st == PGZ_OK) {
            if (bad != 0xffffffffu) {
                F.bad_err = chunks[F.chunk0 + bad].err;
                st = F.bad_err == CE_TRAIL ? PGZ_E_UNSUPPORTED : PGZ_E_DATA;
            } else if (!any_final && (F.mode == 0 || F.mode == 1 || (F.mode == 3 && F.last_seg))) {
                st = PGZ_E_DATA;
            } else if (F.mode != 2 && total > F.out_cap) {
                st = PGZ_E_CAPACITY;
            } else if (F.mode == 0 && (uint32_t)total != F.isize_expect) {
                st = PGZ_E_ISIZE;
            } else if (F.mode == 3 && F.last_seg && (uint32_t)(F.out_before + total) != F.isize_expect) {
                st = PGZ_E_ISIZE;
            }
        }
        F.status = st;
    }
}

// ---------------------------------------------------------------------------
// pass 2a: the window chain
// map of part c: entry k of w_{c+1} is D_c[n-32768+k] if that exists (a byte
// or U_j -> w_c[j]), else w_c[k+n]
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t map_entry(const uint16_t* d, uint64_t n, uint64_t det, uint32_t k) {
    const int64_t t = (int64_t)n - (int64_t)kWin + (int64_t)k;
    if (t < 0) return (uint16_t)(kPH | (uint32_t)(k + n));
    return (uint64_t)t >= det ? reinterpret_cast<const uint8_t*>(d)[det + (uint64_t)t] : d[t];   // det: the tail
}

// Every thread handles entries tid + 1024*j; eight loads are in flight at once.
__global__ void __launch_bounds__(1024) k_chain_compose(const FileDesc* __restrict__ files,
                                                        const ChunkDesc* __restrict__ chunks, const int32_t* g0,
                                                        const int32_t* gn, const int32_t* gfile,
                                                        const uint16_t* __restrict__ sym, uint16_t* gmaps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t* acc = reinterpret_cast<uint16_t*>(smem_raw);
    uint16_t* tmp = acc + kWin;
    const int g = blockIdx.x;
    if (files[gfile[g]].status != PGZ_OK) return;
    const uint32_t tid = threadIdx.x;
    bool have = false;
    for (int c = g0[g]; c < g0[g] + gn[g]; ++c) {
        const ChunkDesc& C = chunks[c];
        if (C.state != CS_DONE || C.n == 0) continue;
        const uint16_t* d = sym + C.sym_base;
        const uint64_t n = C.n;
        for (uint32_t j0 = 0; j0 < kWin / 1024; j0 += 8) {
            uint16_t m[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) m[u] = map_entry(d, n, C.det, tid + 1024u * (j0 + u));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint16_t e = m[u];
                if (have && (e & kPH)) e = acc[e & (kWin - 1)];
                tmp[tid + 1024u * (j0 + u)] = e;
            }
        }
        __syncthreads();
        uint16_t* x = acc;
        acc = tmp;
        tmp = x;
        have = true;
    }
    uint16_t* dst = gmaps + (uint64_t)g * kWin;
    for (uint32_t k = tid; k < kWin; k += 1024) dst[k] = have ? acc[k] : (uint16_t)(kPH | k);
}

__global__ void __launch_bounds__(1024) k_chain_walk(const FileDesc* __restrict__ files, const uint16_t* __restrict__ gmaps,
                                                     uint8_t* wstart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint8_t* W = smem_raw;
    uint8_t* W2 = smem_raw + kWin;
    const FileDesc& F = files[blockIdx.x];
    if (F.status != PGZ_OK) return;
    const uint32_t tid = threadIdx.x;
    for (uint32_t k = tid; k < kWin; k += 1024) W[k] = F.win0 ? F.win0[k] : 0;   // before the member: never referenced
    __syncthreads();
    for (int g = F.group0; g < F.group0 + F.ngroups; ++g) {
        uint8_t* ws = wstart + (uint64_t)g * kWin;
        const uint16_t* m = gmaps + (uint64_t)g * kWin;
        for (uint32_t j0 = 0; j0 < kWin / 1024; j0 += 8) {
            uint16_t e[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) e[u] = m[tid + 1024u * (j0 + u)];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t k = tid + 1024u * (j0 + u);
                ws[k] = W[k];
                W2[k] = (e[u] & kPH) ? W[e[u] & (kWin - 1)] : (uint8_t)e[u];
            }
        }
        __syncthreads();
        uint8_t* x = W;
        W = W2;
        W2 = x;
    }
}

__global__ void __launch_bounds__(1024) k_chain_expand(const FileDesc* __restrict__ files,
                                                       const ChunkDesc* __restrict__ chunks, const int32_t* g0,
                                                       const int32_t* gn, const int32_t* gfile,
                                                       const uint16_t* __restrict__ sym, const uint8_t* wstart,
                                                       uint8_t* windows) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint8_t* W = smem_raw;
    uint8_t* W2 = smem_raw + kWin;
    const int g = blockIdx.x;
    if (files[gfile[g]].status != PGZ_OK) return;
    const uint32_t tid = threadIdx.x;
    const uint8_t* ws = wstart + (uint64_t)g * kWin;
    for (uint32_t k = tid; k < kWin / 16; k += 1024)
        reinterpret_cast<uint4*>(W)[k] = reinterpret_cast<const uint4*>(ws)[k];
    __syncthreads();
    for (int c = g0[g]; c < g0[g] + gn[g]; ++c) {
        const ChunkDesc& C = chunks[c];
        uint4* wc = reinterpret_cast<uint4*>(windows + (uint64_t)c * kWin);
        for (uint32_t k = tid; k < kWin / 16; k += 1024) wc[k] = reinterpret_cast<const uint4*>(W)[k];
        if (C.state != CS_DONE || C.n == 0) continue;
        const uint16_t* d = sym + C.sym_base;
        const uint64_t n = C.n;
        for (uint32_t j0 = 0; j0 < kWin / 1024; j0 += 8) {
            uint16_t m[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) m[u] = map_entry(d, n, C.det, tid + 1024u * (j0 + u));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint16_t e = m[u];
                W2[tid + 1024u * (j0 + u)] = (e & kPH) ? W[e & (kWin - 1)] : (uint8_t)e;
            }
        }
        __syncthreads();
        uint8_t* x = W;
        W = W2;
        W2 = x;
    }
}

// ---------------------------------------------------------------------------
// pass 2b: translation U_j -> w_i[j], 8 symbols per thread per step
// ---------------------------------------------------------------------------

// Persistent: block b translates parts b, b + gridDim.x, ...; the part's
// window w_i is copied into shared memory (only if the part produced a
// placeholder) while the block's previous part is translated (two tables).  The shared table is the window followed by the 256 byte
// values, so a symbol s (a byte b < 0x100, or 0x8000 | j for U_j) becomes
// T[s ^ 0x8000]: window byte j for a placeholder, b for a byte, with no
// branch.  Parts without any placeholder pack their bytes with byte
// permutations.
//
// A warp writes a contiguous run of slices of 512 symbols, a lane 16
// symbols (two 16-byte loads) of each; the loads of the next slice are in
// flight while a slice is translated.
// Output bytes P..P+15 of a lane (P = out_off + symbol index) go out as the
// two aligned 8-byte words from P - m (m = out_off mod 8); the m bytes before
// P come from the previous lane (lane 31's from the previous slice), the m
// bytes after P + 15 - m are the next lane's first word.  Partial slices and
// the first slice of a warp's run take byte stores where a neighbour is
// missing.
constexpr int kTransThreads = 512;
constexpr uint32_t kTransSlice = 512;                  // symbols per slice (16 per lane)
constexpr size_t kTransSmem = 2 * (kWin + 256);         // two window tables

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// 8 symbols -> 8 bytes (symbols past nv are taken as byte 0)
__device__ __forceinline__ uint64_t translate8(const uint8_t* T, uint4 q, uint32_t nv, bool ph) {
    uint32_t w4[4] = {q.x, q.y, q.z, q.w};
    if (nv < 8) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (2u * k >= nv) w4[k] = 0;
            else if (2u * k + 1 >= nv) w4[k] &= 0xffffu;
        }
    }
    uint32_t b0, b1;
    if (!ph) {
        b0 = __byte_perm(w4[0], w4[1], 0x6420);
        b1 = __byte_perm(w4[2], w4[3], 0x6420);
    } else {
        uint32_t pr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = w4[k] ^ 0x80008000u;
            pr[k] = (uint32_t)T[w & 0xffffu] | ((uint32_t)T[w >> 16] << 8);
        }
        b0 = __byte_perm(pr[0], pr[1], 0x5410);
        b1 = __byte_perm(pr[2], pr[3], 0x5410);
    }
    return (uint64_t)b0 | ((uint64_t)b1 << 32);
}

// 8 bytes of the determined tail as they are (bytes past nv taken as 0)
__device__ __forceinline__ uint64_t tail8(uint4 q, uint32_t nv) {
    const uint64_t v = (uint64_t)q.x | ((uint64_t)q.y << 32);
    return nv >= 8 ? v : (nv ? v & (~0ull >> (64 - 8 * nv)) : 0ull);
}

__global__ void __launch_bounds__(kTransThreads, 2) k_translate(const FileDesc* __restrict__ files, ChunkDesc* chunks,
                                                                int nchunks, const uint16_t* __restrict__ sym,
                                                                const uint8_t* __restrict__ windows,
                                                                const uint8_t* __restrict__ fillw) {
    extern __shared__ __align__(16) uint8_t Wbuf[];      // two tables of kWin + 256 bytes (kTransSmem)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x < 256) {
        Wbuf[kWin + threadIdx.x] = (uint8_t)threadIdx.x;
        Wbuf[2 * kWin + 256 + threadIdx.x] = (uint8_t)threadIdx.x;
    }
    // the window of part c goes into table `buf` by asynchronous copies, one group per part
    auto fetch = [&](int c, int buf) {
        if (c < nchunks) {
            const ChunkDesc& C = chunks[c];
            if (files[C.file].status == PGZ_OK && C.state == CS_DONE && C.n != 0 && C.anyph) {
                const uint8_t* src = fillw ? fillw : windows + (uint64_t)c * kWin;
                const uint32_t dst = smem_u32(Wbuf + buf * (kWin + 256));
                for (uint32_t k = threadIdx.x; k < kWin / 16; k += blockDim.x) cp_async16(dst + 16 * k, src + 16 * k);
            }
        }
        cp_async_commit();
    };
    fetch(blockIdx.x, 0);
    int buf = 0;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x, buf ^= 1) {
        fetch(c + gridDim.x, buf ^ 1);                    // the next part's window, while this part runs
        cp_async_wait<1>();                               // this part's window (this thread's copies) ...
        __syncthreads();                                  // ... and everyone else's
        const uint8_t* W = Wbuf + buf * (kWin + 256);
        const ChunkDesc& C = chunks[c];
        const FileDesc& F = files[C.file];
        const bool ph = C.anyph != 0;
        if (F.status == PGZ_OK && C.state == CS_DONE && C.n != 0) {   // uniform per block
        const uint16_t* s = sym + C.sym_base;
        // output byte P of the member goes to out[P - out_lo] when out_lo <= P < out_hi
        uint8_t* out = F.out;
        const uint64_t lo = F.out_lo, hi = F.out_hi;
        const bool vec = F.out_lo == 0 && F.out_hi == kNone && ((reinterpret_cast<uintptr_t>(out) & 7) == 0);
        const uint32_t m = (uint32_t)(C.out_off & 7), sh = 8u * m;
        const uint32_t n32 = (uint32_t)C.n;
        const uint32_t nsl = (n32 + kTransSlice - 1) / kTransSlice, per = (nsl + nwarp - 1) / nwarp;
        const uint32_t j0 = min(nsl, per * (uint32_t)warp), j1 = min(nsl, per * (uint32_t)(warp + 1));
        // the determined tail (symbols from det32 on are bytes at byte det32 + k; det32 is a multiple of 8, so
        // each 8-symbol half lies wholly before or wholly inside it): copied, not translated
        const uint32_t det32 = C.det < (uint64_t)n32 ? (uint32_t)C.det : 0xffffffffu;
        const uint8_t* tb = reinterpret_cast<const uint8_t*>(s) + (det32 == 0xffffffffu ? 0u : det32);
        auto load_half = [&](uint32_t j, uint32_t i0, uint4& a) {
            if (!(j < j1 && i0 < n32)) {
                a = make_uint4(0, 0, 0, 0);
            } else if (i0 >= det32) {
                const uint2 v = *reinterpret_cast<const uint2*>(tb + i0);
                a = make_uint4(v.x, v.y, 0, 0);
            } else {
                a = *reinterpret_cast<const uint4*>(s + i0);
            }
        };
        // loads of slice j + 1 are in flight while slice j is translated
        auto load = [&](uint32_t j, uint4& a, uint4& b) {
            const uint32_t i = j * kTransSlice + 16u * (uint32_t)lane;
            load_half(j, i, a);
            load_half(j, i + 8, b);
        };
        uint4 n0, n1;
        load(j0, n0, n1);
        uint64_t carry = 0;                               // lane 31's second word of the previous slice
        for (uint32_t j = j0; j < j1; ++j) {
            const uint4 q0 = n0, q1 = n1;
            load(j + 1, n0, n1);
            const uint32_t i = j * kTransSlice + 16u * (uint32_t)lane;
            const bool full = (j + 1) * kTransSlice <= n32;   // uniform: every lane holds 16 symbols
            const uint32_t nv = full ? 16u : (i < n32 ? min(n32 - i, 16u) : 0u);
            const uint64_t v0 = i >= det32 ? tail8(q0, nv < 8 ? nv : 8u) : translate8(W, q0, nv < 8 ? nv : 8u, ph);
            const uint64_t v1 = i + 8 >= det32 ? tail8(q1, nv > 8 ? nv - 8 : 0u)
                                               : translate8(W, q1, nv > 8 ? nv - 8 : 0u, ph);
            const uint64_t P = C.out_off + i;
            if (!vec || !full) {          // each lane stores its own bytes (clipped to [lo, hi) when !vec)
                for (uint32_t k = 0; k < nv; ++k) {
                    const uint64_t q = P + k;
                    if (q >= lo && q < hi) out[q - lo] = (uint8_t)((k < 8 ? v0 : v1) >> (8 * (k & 7)));
                }
                continue;
            }
            if (m == 0) {
                *reinterpret_cast<uint64_t*>(out + P) = v0;
                *reinterpret_cast<uint64_t*>(out + P + 8) = v1;
                continue;
            }
            uint64_t prev = __shfl_up_sync(FULL, v1, 1);
            if (lane == 0) prev = carry;
            carry = shfl64(v1, 31);
            const bool have_prev = lane > 0 || j > j0;    // the previous slice of this run was full
            if (have_prev) {
                *reinterpret_cast<uint64_t*>(out + P - m) = (v0 << sh) | (prev >> (64 - sh));
            } else {
                for (uint32_t k = 0; k < 8 - m; ++k) out[P + k] = (uint8_t)(v0 >> (8 * k));
            }
            *reinterpret_cast<uint64_t*>(out + P + 8 - m) = (v1 << sh) | (v0 >> (64 - sh));
            // my last m bytes start the next lane's first word; lane 31 writes them itself unless
            // the next slice is full and in this run
            if (lane == 31) {
                const bool next_full = j + 1 < j1 && (j + 2) * kTransSlice <= n32;
                if (!next_full)
                    for (uint32_t k = 16 - m; k < 16; ++k) out[P + k] = (uint8_t)(v1 >> (8 * (k - 8)));
            }
        }
        }
        __syncthreads();                                  // table `buf` is refilled two parts later
    }
    cp_async_wait<0>();
}

// placeholder count of every part and one past its last placeholder (for
// statistics and inspection; not on the decompression path)
__global__ void __launch_bounds__(256) k_count_ph(ChunkDesc* chunks, int nchunks, const uint16_t* __restrict__ sym) {
    __shared__ unsigned long long s_n, s_last;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        ChunkDesc& C = chunks[c];
        __syncthreads();
        if (threadIdx.x == 0) {
            s_n = 0;
            s_last = 0;
        }
        __syncthreads();
        const uint64_t n0 = C.state == CS_DONE ? C.n : 0;
        const uint64_t n = n0 < C.det ? n0 : C.det;        // a determined tail holds no placeholder
        const uint16_t* p = sym + C.sym_base;
        unsigned long long cnt = 0, last = 0;
        for (uint64_t i = threadIdx.x; i < n; i += blockDim.x)
            if (p[i] & kPH) {
                ++cnt;
                last = i + 1;
            }
        for (int d = 16; d; d >>= 1) {
            cnt += __shfl_xor_sync(FULL, cnt, d);
            last = max(last, __shfl_xor_sync(FULL, last, d));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_n, cnt);
            atomicMax(&s_last, last);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            C.nph = s_n;
            C.last_ph = s_last;
        }
    }
}

// ---------------------------------------------------------------------------
// CRC-32 in GF(2): reflected representation, bit 31-k = coefficient of x^k
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t gf2_mul(uint32_t a, uint32_t b) {
    uint32_t p = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        p ^= b & (0u - ((a >> (31 - k)) & 1u));
        b = (b >> 1) ^ (kPoly & (0u - (b & 1u)));
    }
    return p;
}

__device__ uint32_t xpow8(uint64_t n) {       // x^(8n) mod P
    uint64_t e = n << 3;
    uint32_t r = 0x80000000u;
    for (int k = 0; e; ++k, e >>= 1)
        if (e & 1) r = gf2_mul(r, c_x2k[k]);
    return r;
}

constexpr uint32_t kPiece = 32;       // bytes per lane and segment
constexpr uint32_t kCrcSeg = 32 * kPiece;   // bytes per warp step (one piece per lane)
constexpr int kCrcAhead = 3;          // segments whose loads are in flight while one is folded
constexpr int kCrcThreads = 1024;     // one block per SM
// four byte tables with one copy per lane (128 KiB), then the segment shift's four byte tables, shared (4 KiB)
constexpr size_t kCrcSmem = (4 * 256 * 32 + 4 * 256) * sizeof(uint32_t);

// Slicing by four (four table lookups per 32-bit word, RFC 1952 CRC in the
// reflected form): with x = r ^ w, the register after the word's four bytes
// is T3[x0] ^ T2[x1] ^ T1[x2] ^ T0[x3], where Tk is the byte table followed
// by k zero bytes.  Each lane reads its own copy of the tables (entry b of
// table k of lane l at word 32 * (256 k + b) + l), so the lookups of a warp
// never share a bank.
__device__ __forceinline__ uint32_t crc_word(const uint32_t* Tl, uint32_t r, uint32_t w) {
    const uint32_t x = r ^ w;
    return Tl[32u * (768u + (x & 0xffu))] ^ Tl[32u * (512u + ((x >> 8) & 0xffu))] ^
           Tl[32u * (256u + ((x >> 16) & 0xffu))] ^ Tl[32u * (x >> 24)];
}

// raw CRC register (zero start) of a whole piece held in registers
__device__ __forceinline__ uint32_t crc_piece(const uint32_t* Tl, const uint4 (&v)[kPiece / 16]) {
    uint32_t r = 0;
#pragma unroll
    for (int q = 0; q < (int)(kPiece / 16); ++q) {
        r = crc_word(Tl, r, v[q].x);
        r = crc_word(Tl, r, v[q].y);
        r = crc_word(Tl, r, v[q].z);
        r = crc_word(Tl, r, v[q].w);
    }
    return r;
}

// raw CRC register (zero start) of n bytes at p, byte by byte
__device__ __forceinline__ uint32_t crc_bytes(const uint32_t* Tl, const uint8_t* p, uint64_t n) {
    uint32_t r = 0;
    for (uint64_t i = 0; i < n; ++i) r = Tl[32u * ((r ^ p[i]) & 0xffu)] ^ (r >> 8);
    return r;
}

// r times x^(8 kCrcSeg) mod P: by linearity, the XOR of the products of r's four bytes, each looked up in
// its own table (Y + 256 j: byte j of the register, in place, times the constant)
__device__ __forceinline__ uint32_t crc_shift_seg(const uint32_t* Y, uint32_t r) {
    return Y[r & 0xffu] ^ Y[256u + ((r >> 8) & 0xffu)] ^ Y[512u + ((r >> 16) & 0xffu)] ^ Y[768u + (r >> 24)];
}

// Each warp takes a contiguous run of segments and walks the members it
// covers.  Within a member, lane l's pieces (bytes 32 l .. 32 l + 31 of each
// segment) are folded across the run's full segments by Horner's rule,
// acc_l <- acc_l x^(8 kCrcSeg) + R(piece), so that at the end acc_l
// x^(8 kPiece (31 - l)), summed over the lanes, is the raw CRC of those
// segments (R(A||B) = R(A) x^(8|B|) + R(B)); that sum is shifted to the end
// of the member once and XOR-accumulated there.  The loads of the next
// kCrcAhead segments are in flight while a segment is folded (a warp's
// 32-byte pieces are one 1 KiB stretch, so each load instruction reads few
// lines).  A member's last segment, when shorter, is done byte by byte with
// per-lane shifts, and so is a member whose output is not 16-byte aligned.
__global__ void __launch_bounds__(kCrcThreads, 1) k_crc(FileDesc* files, int nfiles, uint64_t total_seg,
                                                        const uint64_t* seg0, uint64_t segs_per_warp) {
    extern __shared__ uint32_t T[];                       // 4 x 256 x 32 words, then 4 x 256 (the segment shift)
    __shared__ uint32_t LS[32];
    for (int k = threadIdx.x; k < 4 * 256 * 32; k += blockDim.x) T[k] = c_crc_tab[k >> 13][(k >> 5) & 255];
    uint32_t* Y = T + 4 * 256 * 32;
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) Y[k] = c_seg_shift[k >> 8][k & 255];
    if (threadIdx.x < 32) LS[threadIdx.x] = c_lane_shift[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t* Tl = T + lane;
    const uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t s_begin = w * segs_per_warp;
    if (s_begin >= total_seg) return;
    const uint64_t s_end = s_begin + segs_per_warp < total_seg ? s_begin + segs_per_warp : total_seg;
    int f;
    {
        int lo = 0, hi = nfiles - 1;                      // member holding the run's first segment
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg0[mid] <= s_begin) lo = mid;
            else hi = mid - 1;
        }
        f = lo;
    }
    // this lane's part of a raw CRC that ends `shift` bytes before the end of member f: summed over the warp,
    // shifted to the end, accumulated
    auto add = [&](uint32_t r, uint64_t shift) {
        for (int d = 16; d; d >>= 1) r ^= __shfl_xor_sync(FULL, r, d);
        if (lane == 0) atomicXor(&files[f].crc_acc, shift ? gf2_mul(r, xpow8(shift)) : r);
    };
    for (uint64_t sg = s_begin; sg < s_end; ++f) {        // one member of the run per step
        const uint64_t m_end = f + 1 < nfiles ? seg0[f + 1] : ~0ull;
        if (sg >= m_end) continue;                        // a member with no segment
        const uint64_t g_end = m_end < s_end ? m_end : s_end;
        const FileDesc& F = files[f];
        const uint64_t i0 = sg - seg0[f], i1 = g_end - seg0[f];   // the member's segments [i0, i1) in this run
        sg = g_end;
        if (F.status != PGZ_OK || (F.mode != 0 && F.mode != 3)) continue;
        const uint64_t D = F.total;
        const uint8_t* out = F.out;
        const uint64_t nfull = D / kCrcSeg;
        const uint64_t ie = i1 < nfull ? i1 : nfull;      // full segments [i0, ie)
        const uint8_t* base = out + (uint64_t)kPiece * lane;
        if (i0 < ie) {
            uint32_t acc = 0;
            if ((reinterpret_cast<uintptr_t>(out) & 15) == 0) {
                uint4 v[kCrcAhead + 1][kPiece / 16];
                auto load = [&](uint64_t i, uint4 (&dst)[kPiece / 16]) {
                    if (i < ie) {
                        const uint4* p = reinterpret_cast<const uint4*>(base + i * kCrcSeg);
#pragma unroll
                        for (int q = 0; q < (int)(kPiece / 16); ++q) dst[q] = p[q];
                    }
                };
#pragma unroll
                for (int k = 0; k < kCrcAhead; ++k) load(i0 + k, v[k]);
                for (uint64_t i = i0; i < ie; i += kCrcAhead + 1) {
#pragma unroll
                    for (int k = 0; k <= kCrcAhead; ++k) {
                        if (i + k < ie) {
                            load(i + k + kCrcAhead, v[(k + kCrcAhead) % (kCrcAhead + 1)]);
                            const uint32_t r = crc_piece(Tl, v[k]);
                            acc = i + k > i0 ? crc_shift_seg(Y, acc) ^ r : r;
                        }
                    }
                }
            } else {
                for (uint64_t i = i0; i < ie; ++i) {
                    const uint32_t r = crc_bytes(Tl, base + i * kCrcSeg, kPiece);
                    acc = i > i0 ? crc_shift_seg(Y, acc) ^ r : r;
                }
            }
            add(gf2_mul(acc, LS[31 - lane]), D - ie * kCrcSeg);
        }
        if (i0 <= nfull && nfull < i1 && D > nfull * kCrcSeg) {   // the member's last segment, shorter
            const uint64_t pa = nfull * kCrcSeg + (uint64_t)kPiece * lane;
            const uint64_t pb = pa + kPiece < D ? pa + kPiece : D;
            uint32_t r = 0;
            if (pa < pb) r = gf2_mul(crc_bytes(Tl, out + pa, pb - pa), xpow8(D - pb));
            add(r, 0);
        }
    }
}

__global__ void k_finalize(FileDesc* files, int nfiles) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfiles) return;
    FileDesc& F = files[f];
    if (F.status != PGZ_OK) return;
    if (F.mode == 3) {
        // register after the segment, from the register the earlier segments left (R_I(M) = I x^(8|M|) + R_0(M))
        const uint32_t reg = F.crc_acc ^ gf2_mul(F.crc_in, xpow8(F.total));
        F.crc = reg;
        if (F.last_seg && (reg ^ 0xffffffffu) != F.crc_expect) F.status = PGZ_E_CRC;
        return;
    }
    if (F.mode != 0) return;
    // register after D bytes from the initial all-ones register, then inverted
    const uint32_t crc = F.crc_acc ^ gf2_mul(0xffffffffu, xpow8(F.total)) ^ 0xffffffffu;
    F.crc = crc;
    if (crc != F.crc_expect) F.status = PGZ_E_CRC;
}

// ---------------------------------------------------------------------------
// DNA sequences in a block with undetermined characters (Appendix "Heuristic
// extraction of DNA sequences in DEFLATE block"): the maximal non-overlapping
// substrings matching T D+ (U+ D+)* T, T a newline or an undetermined
// character, D a nucleotide, U an undetermined character.  Within a maximal
// run of D/U symbols there is at most one: from the first D preceded by a T
// to the last D followed by a T (outside the run, only a newline is a T), if
// the first comes before the last.  Each thread takes the runs that start in
// its segment of kSeqSeg symbols (following a run past the segment's end).
// ---------------------------------------------------------------------------
constexpr uint32_t kSeqSeg = 1024;

__device__ __forceinline__ uint32_t seq_class(uint16_t s) {      // 0 other, 1 D, 2 U, 3 newline
    if (s & kPH) return 2;
    const uint32_t b = s & 0xffu;
    if (b == 'A' || b == 'C' || b == 'G' || b == 'T' || b == 'N') return 1;
    return b == '\n' ? 3 : 0;
}

__global__ void __launch_bounds__(256) k_sequences(const uint16_t* __restrict__ sym, uint64_t n, uint32_t min_len,
                                                   uint64_t* spans, uint64_t max_spans, unsigned long long* counts) {
    const uint64_t a = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kSeqSeg;
    if (a >= n) return;
    const uint64_t b = a + kSeqSeg < n ? a + kSeqSeg : n;
    uint64_t p = a;
    if (a > 0 && seq_class(sym[a - 1]) - 1u < 2u)                  // a run that began in an earlier segment
        while (p < n && seq_class(sym[p]) - 1u < 2u) ++p;
    while (p < b) {
        uint32_t c = seq_class(sym[p]);
        if (c - 1u >= 2u) {
            ++p;
            continue;
        }
        const uint64_t r0 = p;
        const bool open_left = r0 > 0 && seq_class(sym[r0 - 1]) == 3;
        uint64_t first = ~0ull, last = ~0ull, u_first = 0, u_last = 0, nu = 0;
        uint32_t prev = 0;
        for (; p < n; ++p) {
            c = seq_class(sym[p]);
            if (c - 1u >= 2u) break;
            const uint32_t nx = p + 1 < n ? seq_class(sym[p + 1]) : 0u;
            if (c == 1) {
                if (first == ~0ull && (p == r0 ? open_left : prev == 2)) {
                    first = p;
                    u_first = nu;
                }
                if (nx == 2 || nx == 3) {                          // followed by a T
                    last = p;
                    u_last = nu;
                }
            } else {
                ++nu;
            }
            prev = c;
        }
        if (first != ~0ull && last != ~0ull && last >= first && last - first + 1 >= min_len) {
            const unsigned long long k = atomicAdd(&counts[0], 1ull);
            const bool und = u_last > u_first;
            if (und) atomicAdd(&counts[1], 1ull);
            if (k < max_spans) {
                spans[2 * k] = first;
                spans[2 * k + 1] = (last - first + 1) | (und ? (1ull << 63) : 0ull);
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
void launch_sequences(const uint16_t* sym, uint64_t n, uint32_t min_len, uint64_t* spans, uint64_t max_spans,
                      unsigned long long* counts, cudaStream_t s) {
    cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
    if (n == 0) return;
    const uint64_t threads = (n + kSeqSeg - 1) / kSeqSeg;
    k_sequences<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(sym, n, min_len, spans, max_spans, counts);
}

static size_t warp_smem_bytes() { return sizeof(WarpSmem); }

static int wpb_of(const KParams& p) { return p.wpb == 2 || p.wpb == 8 ? p.wpb : 4; }
static int wpb_slot(int wpb) { return wpb == 2 ? 0 : (wpb == 4 ? 1 : 2); }

// resident blocks of the pass-1 kernels of a CTA shape on the current device
// (both kernels have the same launch bounds and shared memory); also raises
// the kernels' dynamic shared-memory limit once
template <int WPB>
static int pass1_resident_blocks_t() {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = dev >= 0 && dev < 64 ? dev : 0;
    if (!cached[slot]) {
        const int smem = (int)(WPB * warp_smem_bytes());
        int sms = 0, per_sm_a = 0, per_sm_b = 0, per_sm_c = 0;
        const bool ok =
            cudaFuncSetAttribute(k_sync<WPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
            cudaFuncSetAttribute(k_inflate<WPB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_inflate<WPB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, k_sync<WPB>, 32 * WPB, smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_inflate<WPB, true>, 32 * WPB, smem) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, k_inflate<WPB, false>, 32 * WPB, smem) ==
                cudaSuccess;
        const int per_sm_sync = per_sm_a, per_sm_inflate = std::min(per_sm_b, per_sm_c);
        const int v = std::max(1, sms) * std::max(1, std::min(per_sm_sync, per_sm_inflate));
        if (!ok) {
            cudaGetLastError();
            return v;                            // not cached: asked again once a device answers
        }
        cached[slot] = v;
    }
    return cached[slot];
}

static int pass1_resident_blocks(int wpb) {
    switch (wpb_slot(wpb)) {
        case 0: return pass1_resident_blocks_t<2>();
        case 1: return pass1_resident_blocks_t<4>();
        default: return pass1_resident_blocks_t<8>();
    }
}

int pass1_warps(int nchunks, int wpb) {
    if (nchunks <= 0) return 0;
    wpb = wpb == 2 || wpb == 8 ? wpb : 4;
    const int blocks = std::min((nchunks + wpb - 1) / wpb, pass1_resident_blocks(wpb));
    return blocks * wpb;
}

template <int WPB>
static void launch_pass1_t(bool sync, const FileDesc* files, ChunkDesc* chunks, int nchunks, uint16_t* sym,
                         uint32_t* tok, uint32_t* queue, const uint32_t* order, const KParams& p, cudaStream_t s) {
    const int grid = pass1_warps(nchunks, WPB) / WPB;
    const size_t smem = WPB * warp_smem_bytes();
    if (sync) k_sync<WPB><<<grid, 32 * WPB, smem, s>>>(files, chunks, nchunks, sym, tok, queue, order, p);
    else if (p.pipe)
        k_inflate<WPB, true><<<grid, 32 * WPB, smem, s>>>(files, chunks, nchunks, sym, tok, queue, order, p);
    else k_inflate<WPB, false><<<grid, 32 * WPB, smem, s>>>(files, chunks, nchunks, sym, tok, queue, order, p);
}

static void launch_pass1_any(bool sync, const FileDesc* files, ChunkDesc* chunks, int nchunks, uint16_t* sym,
                             uint32_t* tok, uint32_t* queue, const uint32_t* order, const KParams& p,
                             cudaStream_t s) {
    if (nchunks <= 0) return;
    cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
    switch (wpb_slot(wpb_of(p))) {
        case 0: launch_pass1_t<2>(sync, files, chunks, nchunks, sym, tok, queue, order, p, s); break;
        case 1: launch_pass1_t<4>(sync, files, chunks, nchunks, sym, tok, queue, order, p, s); break;
        default: launch_pass1_t<8>(sync, files, chunks, nchunks, sym, tok, queue, order, p, s); break;
    }
}

void launch_sync(const FileDesc* files, ChunkDesc* chunks, int nchunks, uint16_t* sym, uint32_t* tok,
                 uint32_t* queue, const uint32_t* order, const KParams& p, cudaStream_t s) {
    launch_pass1_any(true, files, chunks, nchunks, sym, tok, queue, order, p, s);
}

void launch_inflate(const FileDesc* files, ChunkDesc* chunks, int nchunks, uint16_t* sym, uint32_t* tok,
                    uint32_t* queue, const uint32_t* order, const KParams& p, cudaStream_t s) {
    launch_pass1_any(false, files, chunks, nchunks, sym, tok, queue, order, p, s);
}

uint64_t token_words_per_part() { return kTokPerPart; }

void launch_plan(FileDesc* files, ChunkDesc* chunks, int nfiles, cudaStream_t s) {
    if (nfiles <= 0) return;
    k_plan<<<nfiles, 1024, 0, s>>>(files, chunks);
}

void launch_chain(const FileDesc* files, const ChunkDesc* chunks, int nfiles, int ngroups,
                  const int32_t* g0, const int32_t* gn, const int32_t* gfile, const uint16_t* sym,
                  uint16_t* gmaps, uint8_t* wstart, uint8_t* windows, cudaStream_t s) {
    if (ngroups <= 0) return;
    static bool attr[64] = {};                            // the shared-memory limits are raised per device
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = dev >= 0 && dev < 64 ? dev : 0;
    if (!attr[slot]) {
        attr[slot] =
            cudaFuncSetAttribute(k_chain_compose, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kWin) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_chain_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kWin) == cudaSuccess &&
            cudaFuncSetAttribute(k_chain_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kWin) == cudaSuccess;
    }
    k_chain_compose<<<ngroups, 1024, 4 * kWin, s>>>(files, chunks, g0, gn, gfile, sym, gmaps);
    k_chain_walk<<<nfiles, 1024, 2 * kWin, s>>>(files, gmaps, wstart);
    k_chain_expand<<<ngroups, 1024, 2 * kWin, s>>>(files, chunks, g0, gn, gfile, sym, wstart, windows);
}

void launch_translate(const FileDesc* files, ChunkDesc* chunks, int nchunks, uint64_t max_cap,
                      const uint16_t* sym, const uint8_t* windows, const uint8_t* fillw, cudaStream_t s) {
    if (nchunks <= 0) return;
    (void)max_cap;
    static int resident[64] = {};                         // blocks of k_translate that fit on the device at once
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = dev >= 0 && dev < 64 ? dev : 0;
    if (!resident[slot]) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaFuncSetAttribute(k_translate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTransSmem) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_translate, kTransThreads, kTransSmem) == cudaSuccess &&
            sms > 0 && per_sm > 0)
            resident[slot] = sms * per_sm;
        else
            cudaGetLastError();
    }
    const int cap = resident[slot] ? resident[slot] : 152 * 2;
    const int grid = nchunks < cap ? nchunks : cap;
    k_translate<<<grid, kTransThreads, kTransSmem, s>>>(files, chunks, nchunks, sym, windows, fillw);
}

uint64_t crc_segment_bytes() { return kCrcSeg; }

void launch_count_ph(ChunkDesc* chunks, int nchunks, const uint16_t* sym, cudaStream_t s) {
    if (nchunks <= 0) return;
    k_count_ph<<<nchunks < 1216 ? nchunks : 1216, 256, 0, s>>>(chunks, nchunks, sym);
}

void launch_crc(FileDesc* files, int nfiles, uint64_t total_seg, const uint64_t* seg0, cudaStream_t s) {
    if (nfiles <= 0 || total_seg == 0) return;
    static int sms[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = dev >= 0 && dev < 64 ? dev : 0;
    if (!sms[slot]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0) sms[slot] = n;
        else cudaGetLastError();
        cudaFuncSetAttribute(k_crc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCrcSmem);
    }
    const uint64_t wpb = kCrcThreads / 32;
    const uint64_t target = (uint64_t)(sms[slot] ? sms[slot] : 152) * wpb;   // one block per SM
    const uint64_t spw = (total_seg + target - 1) / target;
    const uint64_t warps = (total_seg + spw - 1) / spw;
    k_crc<<<(unsigned)((warps + wpb - 1) / wpb), kCrcThreads, kCrcSmem, s>>>(files, nfiles, total_seg, seg0, spw);
}

void launch_finalize(FileDesc* files, int nfiles, cudaStream_t s) {
    if (nfiles <= 0) return;
    k_finalize<<<(nfiles + 127) / 128, 128, 0, s>>>(files, nfiles);
}

int kernels_per_run() { return 9; }

// CRC-32 constants from the polynomial (RFC 1952 section 8)
static uint32_t h_mul(uint32_t a, uint32_t b) {
    uint32_t p = 0;
    for (int k = 0; k < 32; ++k) {
        if ((a >> (31 - k)) & 1u) p ^= b;
        b = (b & 1u) ? (b >> 1) ^ kPoly : (b >> 1);
    }
    return p;
}

void upload_crc_tables() {
    uint32_t tab[4][256], x2k[64], ls[32];
    for (uint32_t b = 0; b < 256; ++b) {
        uint32_t r = b;
        for (int k = 0; k < 8; ++k) r = (r & 1u) ? (r >> 1) ^ kPoly : (r >> 1);
        tab[0][b] = r;
    }
    for (int k = 1; k < 4; ++k)                // k further zero bytes
        for (uint32_t b = 0; b < 256; ++b) tab[k][b] = (tab[k - 1][b] >> 8) ^ tab[0][tab[k - 1][b] & 0xffu];
    x2k[0] = 0x40000000u;                      // x
    for (int k = 1; k < 64; ++k) x2k[k] = h_mul(x2k[k - 1], x2k[k - 1]);
    for (int l = 0; l < 32; ++l) {             // x^(8*kPiece*l)
        uint64_t e = 8ull * kPiece * (uint64_t)l;
        uint32_t r = 0x80000000u;
        for (int k = 0; e; ++k, e >>= 1)
            if (e & 1) r = h_mul(r, x2k[k]);
        ls[l] = r;
    }
    uint32_t xseg = 0x80000000u;
    {
        uint64_t e = 8ull * kCrcSeg;
        for (int k = 0; e; ++k, e >>= 1)
            if (e & 1) xseg = h_mul(xseg, x2k[k]);
    }
    uint32_t seg[4][256];                      // multiplication by x^(8*kCrcSeg), byte by byte (it is linear)
    for (int j = 0; j < 4; ++j)
        for (uint32_t b = 0; b < 256; ++b) seg[j][b] = h_mul(b << (8 * j), xseg);
    cudaMemcpyToSymbol(c_crc_tab, tab, sizeof tab);
    cudaMemcpyToSymbol(c_x2k, x2k, sizeof x2k);
    cudaMemcpyToSymbol(c_lane_shift, ls, sizeof ls);
    cudaMemcpyToSymbol(c_seg_shift, seg, sizeof seg);
}

}  // namespace pgz
