// pgz_noalloc.cu -- pgz_decompress_noalloc: whole-member decompression that
// allocates nothing.
//
// Some callers cannot let a library allocate device memory: applications
// that hand all GPU memory to their own pool or caching allocator at start-up
// and forbid allocations behind its back, services with a hard device-memory
// budget fixed in advance, and latency-critical loops where cudaFree (which
// synchronises the whole device) is not acceptable.  For them this entry point
// runs the same kernels as pgz_decompress with all scratch memory (plan
// arrays, pass-1 symbols, windows) taken from one file-scope __device__ array
// of fixed size, so it calls no cudaMalloc, cudaFree, cudaMallocHost or any
// other allocating routine.  The array exists on every GPU that loads the
// library, for the life of the process.
//
// Limits: the member's output (ISIZE) must be at most kNaMaxOut bytes, its
// compressed size at most kNaMaxIn bytes, and its gzip header at most
// kNaMaxHeader bytes; larger inputs are rejected with PGZ_E_ARG.
//
// The first call on a device resolves the array's device address
// (cudaGetSymbolAddress, with that device current) and uploads the CRC-32
// constants; make that first call before any stream capture on the device.
// All calls share the array, so calls that overlap on the GPU (on different
// streams, or from different host threads) race with each other: serialise
// them.  Every call rewrites all of the scratch it reads.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "pgz_internal.h"
#include "../../include/pgz.h"

namespace {
using namespace pgz;

constexpr uint64_t kNaMaxOut = 4ull << 20;          // largest output (ISIZE) accepted
constexpr uint64_t kNaMaxIn = kNaMaxOut + (kNaMaxOut >> 6) + 4096;   // stored blocks cost ~0.03 %
constexpr uint64_t kNaMaxHeader = 4096;
constexpr int kNaMaxParts = 64;
constexpr int kNaMaxGroups = 8;
constexpr uint64_t kNaSymbols = 2 * kNaMaxOut;       // u16 symbols shared by the parts
constexpr uint64_t kNaPartBytes = 32 << 10;          // compressed bytes per part
constexpr int kNaMaxRetries = 32;

constexpr size_t a256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffFiles = 0;
constexpr size_t kOffChunks = a256(kOffFiles + sizeof(FileDesc));
constexpr size_t kOffG0 = a256(kOffChunks + kNaMaxParts * sizeof(ChunkDesc));
constexpr size_t kOffGn = a256(kOffG0 + kNaMaxGroups * sizeof(int32_t));
constexpr size_t kOffGfile = a256(kOffGn + kNaMaxGroups * sizeof(int32_t));
constexpr size_t kOffSeg0 = a256(kOffGfile + kNaMaxGroups * sizeof(int32_t));
constexpr size_t kOffWindows = a256(kOffSeg0 + sizeof(uint64_t));
constexpr size_t kOffGmaps = a256(kOffWindows + (size_t)kNaMaxParts * kWin);
constexpr size_t kOffWstart = a256(kOffGmaps + (size_t)kNaMaxGroups * kWin * sizeof(uint16_t));
constexpr size_t kOffSym = a256(kOffWstart + (size_t)kNaMaxGroups * kWin);
constexpr size_t kTokWords = 32 * 512;                // token buffer of one part (parallel block decoder)
constexpr size_t kOffTok = a256(kOffSym + kNaSymbols * sizeof(uint16_t));
constexpr size_t kOffQueue = a256(kOffTok + (size_t)kNaMaxParts * kTokWords * sizeof(uint32_t));
constexpr size_t kScratchBytes = a256(kOffQueue + 2 * sizeof(uint32_t));   // about 23 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// device address of the array on the current device (set-up on first use)
int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PGZ_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PGZ_E_CUDA;
        upload_crc_tables();
        if (cudaGetLastError() != cudaSuccess) return PGZ_E_CUDA;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return PGZ_OK;
}

uint32_t crc32_bitwise(const uint8_t* p, size_t n) {
    uint32_t c = 0xffffffffu;
    for (size_t i = 0; i < n; ++i) {
        c ^= p[i];
        for (int k = 0; k < 8; ++k) c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : (c >> 1);
    }
    return ~c;
}

// RFC 1952 member header inside the first hlen bytes: offset of the DEFLATE data
int header_offset(const uint8_t* h, uint64_t hlen, uint64_t gz_len, uint64_t* s0) {
    if (gz_len < 18 || hlen < 10) return PGZ_E_HEADER;
    if (h[0] != 0x1f || h[1] != 0x8b || h[2] != 8 || (h[3] & 0xe0)) return PGZ_E_HEADER;
    const uint8_t flg = h[3];
    uint64_t pos = 10;
    if (flg & 4) {
        if (pos + 2 > hlen) return PGZ_E_ARG;
        pos += 2 + (h[pos] | ((uint64_t)h[pos + 1] << 8));
    }
    for (int f = 8; f <= 16; f <<= 1) {
        if (flg & f) {
            while (pos < hlen && h[pos]) ++pos;
            if (pos >= hlen) return hlen < gz_len ? PGZ_E_ARG : PGZ_E_HEADER;
            ++pos;
        }
    }
    if (flg & 2) {
        if (pos + 2 > hlen) return PGZ_E_ARG;
        if ((crc32_bitwise(h, pos) & 0xffffu) != (h[pos] | ((uint32_t)h[pos + 1] << 8))) return PGZ_E_HEADER;
        pos += 2;
    }
    if (pos > hlen) return PGZ_E_ARG;
    if (pos + 8 > gz_len) return PGZ_E_HEADER;
    *s0 = pos;
    return PGZ_OK;
}

}  // namespace

extern "C" int pgz_decompress_noalloc(const uint8_t* gz, uint64_t gz_len, uint8_t* out, uint64_t out_cap,
                                      uint64_t* out_len, void* cuda_stream) {
    if (!gz || !out_len || (!out && out_cap) || (reinterpret_cast<uintptr_t>(gz) & 3)) return PGZ_E_ARG;
    *out_len = 0;
    if (gz_len < 18) return PGZ_E_HEADER;
    if (gz_len > kNaMaxIn) return PGZ_E_ARG;
    unsigned char* base = nullptr;
    int e = scratch_for_current_device(&base);
    if (e) return e;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // header and trailer (pageable host copies: no staging allocation of ours)
    uint8_t hdr[kNaMaxHeader + 8];
    const uint64_t hlen = gz_len < kNaMaxHeader ? gz_len : kNaMaxHeader;
    if (cudaMemcpyAsync(hdr, gz, hlen, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hdr + hlen, gz + gz_len - 8, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PGZ_E_CUDA;
    uint64_t s0 = 0;
    e = header_offset(hdr, hlen, gz_len, &s0);
    if (e) return e;
    const uint8_t* t = hdr + hlen;
    const uint32_t crc = t[0] | ((uint32_t)t[1] << 8) | ((uint32_t)t[2] << 16) | ((uint32_t)t[3] << 24);
    const uint32_t isize = t[4] | ((uint32_t)t[5] << 8) | ((uint32_t)t[6] << 16) | ((uint32_t)t[7] << 24);
    if (isize > kNaMaxOut) return PGZ_E_ARG;

    FileDesc* d_files = reinterpret_cast<FileDesc*>(base + kOffFiles);
    ChunkDesc* d_chunks = reinterpret_cast<ChunkDesc*>(base + kOffChunks);
    int32_t* d_g0 = reinterpret_cast<int32_t*>(base + kOffG0);
    int32_t* d_gn = reinterpret_cast<int32_t*>(base + kOffGn);
    int32_t* d_gfile = reinterpret_cast<int32_t*>(base + kOffGfile);
    uint64_t* d_seg0 = reinterpret_cast<uint64_t*>(base + kOffSeg0);
    uint8_t* d_windows = base + kOffWindows;
    uint16_t* d_gmaps = reinterpret_cast<uint16_t*>(base + kOffGmaps);
    uint8_t* d_wstart = base + kOffWstart;
    uint16_t* d_sym = reinterpret_cast<uint16_t*>(base + kOffSym);
    uint32_t* d_tok = reinterpret_cast<uint32_t*>(base + kOffTok);
    uint32_t* d_queue = reinterpret_cast<uint32_t*>(base + kOffQueue);
    if (token_words_per_part() != kTokWords || pass1_warps(kNaMaxParts, 4) > kNaMaxParts) return PGZ_E_ARG;

    KParams kp{};
    pgz_config cfg;
    pgz_config_init(&cfg);
    for (int b = 0; b < 256; ++b)
        if ((cfg.allowed[b >> 3] >> (b & 7)) & 1) kp.allowed[b >> 5] |= 1u << (b & 31);
    kp.min_block = cfg.min_block;
    kp.max_block = cfg.max_block;
    kp.confirm_blocks = cfg.confirm_blocks;
    kp.wpb = 4;
    kp.pipe = 0;

    const uint64_t csize = gz_len - 8 - s0, end_bit = (gz_len - 8) * 8;
    uint64_t n = (csize + kNaPartBytes - 1) / kNaPartBytes;
    n = n < 1 ? 1 : (n > (uint64_t)kNaMaxParts ? (uint64_t)kNaMaxParts : n);
    ChunkDesc plan[kNaMaxParts], res[kNaMaxParts];
    FileDesc F, R;
    bool replan = true;
    uint64_t false_syncs = 0;
    for (int attempt = 0; attempt <= kNaMaxRetries; ++attempt) {
        if (replan) {                                  // n parts of equal compressed size
            const uint64_t per = (csize + n - 1) / n;
            const uint64_t cap = (kNaSymbols / n) / 8 * 8;
            memset(plan, 0, sizeof plan);
            for (uint64_t i = 0; i < n; ++i) {
                ChunkDesc& C = plan[i];
                C.lo = (s0 + i * per) * 8;
                C.hi = (s0 + (i + 1) * per) * 8 < end_bit ? (s0 + (i + 1) * per) * 8 : end_bit;
                C.sym_base = i * cap;
                C.cap = cap;
                C.index = (int32_t)i;
                C.disabled = (i > 0 && C.lo >= end_bit) ? 1u : 0u;
                C.stop_hint = kNone;
                C.sync = kNone;
            }
            replan = false;
        }
        uint64_t gsz = 1;
        while (gsz * gsz < n) ++gsz;
        int32_t g0[kNaMaxGroups], gn[kNaMaxGroups], gfile[kNaMaxGroups];
        int ng = 0;
        for (uint64_t a = 0; a < n; a += gsz, ++ng) {
            g0[ng] = (int32_t)a;
            gn[ng] = (int32_t)(gsz < n - a ? gsz : n - a);
            gfile[ng] = 0;
        }
        memset(&F, 0, sizeof F);
        F.gz = gz;
        F.gz_len = gz_len;
        F.out = out;
        F.out_cap = out_cap;
        F.s0_bit = s0 * 8;
        F.end_bit = end_bit;
        F.crc_expect = crc;
        F.isize_expect = isize;
        F.chunk0 = 0;
        F.nchunks = (int32_t)n;
        F.group0 = 0;
        F.ngroups = ng;
        F.seg0 = 0;
        F.nseg = ((out_cap < (uint64_t)kNaMaxOut ? out_cap : (uint64_t)kNaMaxOut) + crc_segment_bytes() - 1) /
                 crc_segment_bytes();
        F.out_hi = kNone;
        F.bad_chunk = 0xffffffffu;
        const uint64_t seg0 = 0;
        cudaMemcpyAsync(d_files, &F, sizeof F, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_chunks, plan, n * sizeof(ChunkDesc), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_g0, g0, ng * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_gn, gn, ng * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_gfile, gfile, ng * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_seg0, &seg0, sizeof seg0, cudaMemcpyHostToDevice, s);
        launch_sync(d_files, d_chunks, (int)n, d_sym, d_tok, d_queue, nullptr, kp, s);
        launch_inflate(d_files, d_chunks, (int)n, d_sym, d_tok, d_queue + 1, nullptr, kp, s);
        launch_plan(d_files, d_chunks, 1, s);
        launch_chain(d_files, d_chunks, 1, ng, d_g0, d_gn, d_gfile, d_sym, d_gmaps, d_wstart, d_windows, s);
        launch_translate(d_files, d_chunks, (int)n, plan[0].cap, d_sym, d_windows, nullptr, s);
        launch_crc(d_files, 1, F.nseg, d_seg0, s);
        launch_finalize(d_files, 1, s);
        if (cudaGetLastError() != cudaSuccess) return PGZ_E_CUDA;
        if (cudaMemcpyAsync(&R, d_files, sizeof R, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PGZ_E_CUDA;
        *out_len = R.total;
        if (R.status == PGZ_OK || R.bad_chunk == 0xffffffffu) return (int)R.status;
        // a part failed: adjust the plan as pgz_decompress does, within the fixed scratch
        if (cudaMemcpyAsync(res, d_chunks, n * sizeof(ChunkDesc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PGZ_E_CUDA;
        // the same recovery as pgz_decompress, within the fixed scratch: a part that needs more symbol
        // capacity makes the plan use fewer parts, each with a larger share of the symbol array
        F.nchunks = (int32_t)n;
        int grow = -1;
        const int a = recover_member(F, plan, res, kp.confirm_blocks, &false_syncs, &grow);
        if (a == kRecoverGrow) {
            if (n == 1) return PGZ_E_CAPACITY;
            n = (n + 1) / 2;
            replan = true;
        } else if (a != kRecoverRerun) {
            return (int)R.status;
        }
    }
    return PGZ_E_DATA;
}
