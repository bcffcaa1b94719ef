// pgz_internal.h -- structures shared by the host planner and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pgz {

constexpr uint32_t kWin = 32768;          // DEFLATE window (RFC 1951 2; Section "DEFLATE algorithm")
constexpr uint32_t kPH = 0x8000u;         // symbol flag: placeholder U_j, j in the low 15 bits
constexpr uint64_t kNone = ~0ull;

// chunk states after the sync / inflate kernels
enum ChunkState : uint32_t {
    CS_PENDING = 0,
    CS_FOUND = 1,      // block start accepted, its block decoded
    CS_EMPTY = 2,      // no accepted block start in the scan range
    CS_DONE = 3,       // pass 1 finished for this part
    CS_ERROR = 4       // see ChunkDesc::err
};

// device-side error codes of a part (ChunkDesc::err)
enum ChunkErr : uint32_t {
    CE_OK = 0,
    CE_DATA = 1,       // invalid DEFLATE content
    CE_TRUNC = 2,      // read past the compressed data
    CE_DIST = 3,       // distance beyond the start of the member
    CE_OVERFLOW = 4,   // symbol capacity of the part exceeded
    CE_CHAIN = 5,      // did not end exactly on the next part's block start
    CE_CONFIRM = 6,    // a confirmation block failed
    CE_TRAIL = 7,      // data after the member's final block
    CE_BYTE = 8,       // literal outside the allowed set (sync checks)
    CE_SIZE = 9,       // block size outside the bounds (sync checks)
    CE_FINAL = 10,     // BFINAL set at a candidate
    CE_TYPE = 11       // not a dynamic block at a candidate
};

struct KParams {
    uint32_t allowed[8];   // 256-bit set of literal bytes accepted at a block start
    uint32_t min_block;
    uint32_t max_block;
    int confirm_blocks;
    int wpb;               // warps per block of the pass-1 kernels: 2, 4 or 8 (0: 4)
    int pipe;              // k_inflate executes tokens in pipelined passes (1) or one pass at a time (0)
    int tail;              // k_inflate stores a part's determined tail as bytes (1) or keeps u16 symbols (0)
};

// one gzip member
struct FileDesc {
    const uint8_t* gz;
    uint64_t gz_len;
    uint8_t* out;
    uint64_t out_cap;
    uint64_t s0_bit;       // first bit of the DEFLATE data
    uint64_t end_bit;      // (gz_len - 8) * 8: the trailer is not DEFLATE data
    uint32_t crc_expect;
    uint32_t isize_expect;
    int32_t chunk0, nchunks;
    int32_t group0, ngroups;
    uint64_t seg0, nseg;   // 4 KiB CRC segments of the output
    uint32_t mode;         // 0 whole member; 1 from a bit offset (no CRC/ISIZE); 2 byte range of the output;
                           // 3 one segment of a streamed member (bit positions relative to the segment's bytes)
    uint32_t open_end;     // mode 0: more members may follow; the member ends after its final block, and its
                           // trailer (CRC-32, ISIZE) is read there
    uint64_t out_base;     // output offset of the first part (mode 2: from the index)
    uint64_t out_lo, out_hi;  // member output bytes [out_lo, out_hi) go to out[P - out_lo]
    // results
    uint64_t total;        // output bytes
    uint32_t crc_acc;      // XOR of position-shifted raw CRCs of the segments
    uint32_t crc;          // finished CRC-32
    uint32_t status;       // pgz_status
    uint32_t bad_chunk;    // first part with an error (for recovery), or ~0
    uint32_t bad_err;
    uint32_t pad1;
    uint64_t member_end;   // mode 0: one past the member's trailer, in bytes of gz
    // mode 3 (streamed member): what the earlier segments left
    const uint8_t* win0;   // resolved 32 KiB window before the segment's first part (null: the member start)
    uint64_t out_before;   // output bytes of the member before the segment
    uint32_t crc_in;       // CRC-32 register after those bytes (all-ones start, not inverted)
    uint32_t last_seg;     // the segment reaches the member's end: its final block and trailer are in it
};

// one part of a member
struct ChunkDesc {
    // plan
    uint64_t lo, hi;       // scan range of the block start, bits [lo, hi)
    uint64_t sym_base;     // offset of the part's symbols in the scratch (u16 units)
    uint64_t cap;          // symbol capacity
    int32_t file;
    int32_t index;         // part number within the member
    uint32_t disabled;     // 1: treated as empty (merged into the previous part)
    uint32_t given;        // 1: lo is a known block start (no search)
    uint64_t stop_hint;    // block start after the last part of the plan (range decoding), else kNone
    // results
    uint64_t sync;         // block start (bit), kNone if none
    uint64_t resume;       // bit after the first block
    uint64_t n;            // symbols produced
    uint64_t nph;          // placeholder symbols produced (counted by the translation)
    uint64_t last_ph;      // one past the last placeholder symbol (pass 1 keeps it up to date; the statistics
                           // kernel recounts it)
    uint64_t det;          // the determined tail: symbols from det on are stored as bytes (u8 at byte offset
                           // det + k of the part's buffer for symbol k), kNone if the part has no such tail
    uint64_t end;          // bit where pass 1 stopped
    uint64_t out_off;      // output offset of the part
    uint32_t state;
    uint32_t err;
    uint32_t blocks;
    uint32_t final;        // the part decoded the member's final block
    uint32_t anyph;        // pass 1 produced at least one placeholder
    uint32_t probe;        // 1: only the block start is searched (the end of a streamed segment); no output
    uint32_t confirm_ext;  // plan: when the part reaches the next part's start before its confirmation blocks
                           // are all decoded, it decodes on past that start until they are (output unchanged)
    uint32_t confirmed;    // result: the start's block and the confirm_blocks blocks after it (or up to a
                           // final block) decoded with the checks; always 1 for a known start
};

// host-side launch wrappers (pgz_kernels.cu)
// tok: token_words_per_part() u32 of parallel-block-decoder scratch for each of
//      pass1_warps(nchunks, p.wpb) warps (at most nchunks rounded up to p.wpb);
// queue: one u32 work counter per kernel (zeroed by the launcher on the stream);
// order (nullable): the parts in the order the work queue hands them out (nchunks entries).
void launch_sync(const FileDesc* files, ChunkDesc* chunks, int nchunks, uint16_t* sym, uint32_t* tok,
                 uint32_t* queue, const uint32_t* order, const KParams& p, cudaStream_t s);
void launch_inflate(const FileDesc* files, ChunkDesc* chunks, int nchunks, uint16_t* sym, uint32_t* tok,
                    uint32_t* queue, const uint32_t* order, const KParams& p, cudaStream_t s);
uint64_t token_words_per_part();
int pass1_warps(int nchunks, int wpb);
void launch_plan(FileDesc* files, ChunkDesc* chunks, int nfiles, cudaStream_t s);
void launch_chain(const FileDesc* files, const ChunkDesc* chunks, int nfiles, int ngroups,
                  const int32_t* group_chunk0, const int32_t* group_n, const int32_t* group_file,
                  const uint16_t* sym, uint16_t* gmaps, uint8_t* wstart, uint8_t* windows, cudaStream_t s);
void launch_translate(const FileDesc* files, ChunkDesc* chunks, int nchunks, uint64_t max_cap,
                      const uint16_t* sym, const uint8_t* windows, const uint8_t* fill_window, cudaStream_t s);
// total_seg: CRC segments of crc_segment_bytes() output bytes over all members (FileDesc::seg0, nseg)
uint64_t crc_segment_bytes();
void launch_crc(FileDesc* files, int nfiles, uint64_t total_seg, const uint64_t* seg0, cudaStream_t s);
void launch_finalize(FileDesc* files, int nfiles, cudaStream_t s);
// DNA sequences among n u16 symbols: spans[2k] = start, spans[2k+1] = length | bit 63 if undetermined
// symbols lie inside; counts[0] = spans found (may exceed max_spans), counts[1] = those with undetermined
void launch_sequences(const uint16_t* sym, uint64_t n, uint32_t min_len, uint64_t* spans, uint64_t max_spans,
                      unsigned long long* counts, cudaStream_t s);
// ChunkDesc::nph and last_ph from the symbols of every finished part (statistics and inspection only)
void launch_count_ph(ChunkDesc* chunks, int nchunks, const uint16_t* sym, cudaStream_t s);
int kernels_per_run();
void upload_crc_tables();

// Recovery after a failed run (pgz_host.cu), shared by every entry point.  For the member F whose parts are
// plan[F.chunk0 .. F.chunk0 + F.nchunks) with the run's results res[...], it changes the plan for a re-run:
//  - every searched start whose confirmation failed is searched again from the bit after it (Section
//    "Detection of DEFLATE block start positions"): the lowest start that passes both the block checks and
//    the confirmation is the one taken;
//  - then the first failing part, in order, decides: a part that did not end exactly on the next part's
//    start shows that start is not on the member's chain of blocks, and that part is merged into its
//    predecessor (if its confirmation is not settled yet, it first decodes past its stop to settle it);
//    another decoding error of a searched start merges its part too.
// Returns kRecoverRerun, kRecoverGrow (*grow = a part that needs more symbol capacity; the caller decides
// how to give it) or kRecoverStop (the error is final).
constexpr int kRecoverStop = 0, kRecoverRerun = 1, kRecoverGrow = 2;
int recover_member(const FileDesc& F, ChunkDesc* plan, const ChunkDesc* res, int confirm_blocks,
                   uint64_t* false_syncs, int* grow);

}  // namespace pgz
