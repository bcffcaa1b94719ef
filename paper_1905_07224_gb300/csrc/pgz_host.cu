// pgz_host.cu -- the C ABI of libpgz (include/pgz.h): gzip header parsing,
// part planning, the launch sequence of the two passes, recovery from false
// block starts, batches replayed as CUDA graphs, and the random-access index.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "pgz_internal.h"
#include "../../include/pgz.h"

using namespace pgz;

namespace pgz {

namespace {

// a part whose block start was searched (not the member start, not a known start, not a segment-end probe)
bool searched_start(const FileDesc& F, const ChunkDesc& C, const ChunkDesc& R) {
    return !C.given && !C.probe && !C.disabled && R.sync != kNone && !(C.index == 0 && C.lo <= F.s0_bit);
}

// the part that holds the next block start after part c (the part k_inflate stopped at), or -1
int next_start(const FileDesc& F, const ChunkDesc* res, int c) {
    for (int j = c + 1; j < F.chunk0 + F.nchunks; ++j)
        if (res[j].sync != kNone) return j;
    return -1;
}

// The confirmation of part c's start: its block and the confirm_blocks blocks after it must decode with the
// checks (Section "Detection of DEFLATE block start positions").  A part checks the blocks it decodes itself;
// when it ends exactly on the next part's start before the window is complete, the blocks of that part are
// the same chain's next blocks, and their checks (made by that part) continue the window.  Returns the
// 1-based position of the first failing block in the window, 0 if the window passed, -1 if the run's results
// do not settle it.
int confirm_failure(const FileDesc& F, const ChunkDesc* res, int c, int confirm_blocks) {
    const int window = confirm_blocks + 1;
    int before = 0;                                  // blocks of the window decoded by earlier parts
    for (;;) {
        const ChunkDesc& R = res[c];
        if (R.confirmed) return 0;
        if (R.state == CS_ERROR && R.err == CE_CONFIRM) {
            const int k = before + (int)R.blocks + 1;
            return k <= window ? k : 0;
        }
        if (R.state != CS_DONE) return -1;
        before += (int)R.blocks;
        if (before >= window) return 0;
        const int j = next_start(F, res, c);
        if (j < 0 || res[j].sync != R.end) return -1;
        c = j;
    }
}

}  // namespace

int recover_member(const FileDesc& F, ChunkDesc* plan, const ChunkDesc* res, int confirm_blocks,
                   uint64_t* false_syncs, int* grow) {
    const int c0 = F.chunk0, c1 = F.chunk0 + F.nchunks;
    // a streamed segment whose probe found no block start: its last part ran to the end of the segment's
    // bytes; only a longer look-ahead helps (the caller's decision)
    if (F.mode == 3 && !F.last_seg && res[c1 - 1].state == CS_EMPTY) return kRecoverStop;
    // 1. starts that failed their confirmation: the search goes on from the bit after each
    bool again = false;
    if (confirm_blocks > 0)
        for (int c = c0; c < c1; ++c) {
            if (!searched_start(F, plan[c], res[c])) continue;
            if (confirm_failure(F, res, c, confirm_blocks) > 0) {
                plan[c].lo = res[c].sync + 1;
                plan[c].confirm_ext = 0;
                again = true;
            }
        }
    if (again) return kRecoverRerun;
    // 2. the first failing part, in order: every part before it ended on the next start, so its own start
    // lies on the member's chain of blocks
    for (int c = c0; c < c1; ++c) {
        const ChunkDesc& R = res[c];
        if (R.state != CS_ERROR) continue;
        ChunkDesc& C = plan[c];
        if (R.err == CE_OVERFLOW) {
            *grow = c;
            return kRecoverGrow;
        }
        if (R.err == CE_TRAIL) return kRecoverStop;
        if (R.err == CE_CHAIN) {
            const int j = next_start(F, res, c);
            if (j < 0) return kRecoverStop;
            if (res[j].state == CS_ERROR && res[j].err == CE_OVERFLOW) {
                *grow = j;
                return kRecoverGrow;
            }
            if (plan[j].probe) {                  // a false block start at the segment's end: search on after it
                plan[j].lo = res[j].sync + 1;
                ++*false_syncs;
                return kRecoverRerun;
            }
            // the start of part j is not on the chain.  Its confirmation decides between the next start of
            // its search (failed, handled above) and no start in its range (passed: merge); when the run left
            // it open, part j first decodes past its stop to settle it
            if (confirm_blocks > 0 && searched_start(F, plan[j], res[j]) && !plan[j].confirm_ext &&
                confirm_failure(F, res, j, confirm_blocks) < 0) {
                plan[j].confirm_ext = 1;
                return kRecoverRerun;
            }
            plan[j].disabled = 1;
            ++*false_syncs;
            return kRecoverRerun;
        }
        if (C.index == 0 && C.lo <= F.s0_bit) return kRecoverStop;
        if (C.given) return kRecoverStop;
        if (R.err == CE_CONFIRM && R.sync != kNone) {
            C.lo = R.sync + 1;
            C.confirm_ext = 0;
            return kRecoverRerun;
        }
        C.disabled = 1;
        ++*false_syncs;
        return kRecoverRerun;
    }
    return kRecoverStop;
}

}  // namespace pgz

namespace {

constexpr uint64_t kMaxPartSymbols = (1ull << 31) - 256;   // part positions are 32-bit in the kernels
constexpr int kMaxRetries = 32;

struct DBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

struct PBuf {   // pinned host staging
    void* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMallocHost(&p, bytes);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// CRC-32 of RFC 1952 section 8 (host; used for the optional header CRC only)
uint32_t host_crc32(const uint8_t* p, size_t n) {
    uint32_t c = 0xffffffffu;
    for (size_t i = 0; i < n; ++i) {
        c ^= p[i];
        for (int k = 0; k < 8; ++k) c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : (c >> 1);
    }
    return ~c;
}

// RFC 1952 2.3 member header.  Returns PGZ_OK and the offset of the DEFLATE
// data, PGZ_E_HEADER, or -1 if the header runs past the hlen bytes given.
int parse_header(const uint8_t* h, uint64_t hlen, uint64_t gz_len, uint64_t* s0) {
    if (gz_len < 18 || hlen < 10) return PGZ_E_HEADER;
    if (h[0] != 0x1f || h[1] != 0x8b || h[2] != 8 || (h[3] & 0xe0)) return PGZ_E_HEADER;
    const uint8_t flg = h[3];
    uint64_t pos = 10;
    if (flg & 4) {
        if (pos + 2 > hlen) return -1;
        pos += 2 + (h[pos] | ((uint64_t)h[pos + 1] << 8));
    }
    for (int f = 8; f <= 16; f <<= 1) {
        if (flg & f) {
            while (pos < hlen && h[pos]) ++pos;
            if (pos >= hlen) return hlen < gz_len ? -1 : PGZ_E_HEADER;
            ++pos;
        }
    }
    if (flg & 2) {
        if (pos + 2 > hlen) return -1;
        const uint32_t c = host_crc32(h, pos) & 0xffffu;
        if (c != (h[pos] | ((uint32_t)h[pos + 1] << 8))) return PGZ_E_HEADER;
        pos += 2;
    }
    if (pos > hlen) return -1;
    if (pos + 8 > gz_len) return PGZ_E_HEADER;
    *s0 = pos;
    return PGZ_OK;
}

struct MemberInfo {
    uint64_t s0;
    uint32_t crc, isize;
};

// a planned set of members and their parts, with device buffers
struct Plan {
    std::vector<FileDesc> files;
    std::vector<ChunkDesc> chunks;
    std::vector<int32_t> g0, gn, gfile;
    std::vector<uint64_t> seg0;
    std::vector<uint32_t> order;  // the parts in the order the pass-1 work queue hands them out
    uint64_t sym_total = 0, max_cap = 0, total_seg = 0;
    bool chain = true, translate = true, crc = true;
    bool results_valid = false;   // the device chunk array holds the last run's results
    int wpb = 4;                  // warps per block of the pass-1 kernels (sizes the token scratch)
    const uint8_t* fill = nullptr;   // device window of fill bytes (mode 1)
    DBuf d_files, d_chunks, d_g0, d_gn, d_gfile, d_seg0, d_sym, d_windows, d_gmaps, d_wstart, d_tok, d_queue, d_order;
    PBuf h_files, h_chunks, h_static;
    cudaGraphExec_t graph = nullptr;
    void release() {
        d_files.release();
        d_chunks.release();
        d_g0.release();
        d_gn.release();
        d_gfile.release();
        d_seg0.release();
        d_sym.release();
        d_windows.release();
        d_gmaps.release();
        d_wstart.release();
        d_tok.release();
        d_queue.release();
        d_order.release();
        h_files.release();
        h_chunks.release();
        h_static.release();
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
};

}  // namespace

struct pgz_ctx {
    pgz_config cfg;
    KParams kp;
    cudaStream_t stream = nullptr;
    Plan plan;                 // the last call's plan (kept for inspection)
    PBuf hdr;                  // header / trailer staging
    DBuf in_buf, out_buf, fill_buf;
    DBuf carry_win;            // streaming: the resolved window a segment leaves for the next
    DBuf sin[2], sout[2];      // streaming: compressed bytes and output of two segments in flight
    PBuf stage[2];             // streaming: pinned output of two segments
    uint64_t launches = 0;
    cudaEvent_t ev[8] = {};
    // host-buffer batches: device copies of the jobs, and one plan per group of jobs in flight
    static constexpr int kHostGroups = 4;
    DBuf hb_in, hb_out;
    Plan hb_plan[kHostGroups];
    cudaStream_t hb_up = nullptr, hb_down = nullptr;
    cudaEvent_t hb_ev_up[kHostGroups] = {}, hb_ev_run[kHostGroups] = {};
};

struct pgz_batch {
    pgz_ctx* ctx;
    Plan plan;
    std::vector<pgz_job> jobs;
};

struct pgz_index {
    const uint8_t* gz;
    uint64_t gz_len;
    uint64_t total;
    std::vector<uint64_t> sync, off, n, stop;   // per non-empty part
    std::vector<MemberInfo> info;
    DBuf windows;                                // resolved w_i, 32 KiB each
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PGZ_OK : (e == cudaErrorMemoryAllocation ? PGZ_E_NOMEM : PGZ_E_CUDA); }

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// header and trailer of a member in device memory
int read_member(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, MemberInfo* mi) {
    if (gz_len < 18) return PGZ_E_HEADER;
    uint64_t want = std::min<uint64_t>(gz_len, 4096);
    for (;;) {
        if (cuda_status(ctx->hdr.ensure(want + 8))) return PGZ_E_NOMEM;
        uint8_t* h = ctx->hdr.as<uint8_t>();
        if (cudaMemcpyAsync(h, gz, want, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
        if (cudaMemcpyAsync(h + want, gz + gz_len - 8, 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            return PGZ_E_CUDA;
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
        uint64_t s0 = 0;
        const int r = parse_header(h, want, gz_len, &s0);
        if (r == -1 && want < gz_len) {
            want = std::min<uint64_t>(gz_len, want * 4);
            continue;
        }
        if (r != PGZ_OK) return PGZ_E_HEADER;
        const uint8_t* t = h + want;
        mi->s0 = s0;
        mi->crc = t[0] | ((uint32_t)t[1] << 8) | ((uint32_t)t[2] << 16) | ((uint32_t)t[3] << 24);
        mi->isize = t[4] | ((uint32_t)t[5] << 8) | ((uint32_t)t[6] << 16) | ((uint32_t)t[7] << 24);
        return PGZ_OK;
    }
}

// parts of one member: equal compressed size (Section "Full file decompression
// in two passes": n roughly equal parts)
void plan_member(pgz_ctx* ctx, Plan& P, const uint8_t* gz, uint64_t gz_len, uint8_t* out, uint64_t out_cap,
                 const MemberInfo& mi, uint32_t mode) {
    FileDesc F{};
    F.gz = gz;
    F.gz_len = gz_len;
    F.out = out;
    F.out_cap = out_cap;
    F.s0_bit = mi.s0 * 8;
    F.end_bit = (gz_len - 8) * 8;
    F.crc_expect = mi.crc;
    F.isize_expect = mi.isize;
    F.mode = mode;
    F.out_hi = kNone;
    const uint64_t csize = gz_len - 8 - mi.s0;
    uint64_t n;
    if (ctx->cfg.n_chunks > 0) n = (uint64_t)ctx->cfg.n_chunks;
    else n = std::max<uint64_t>(1, (csize + ctx->cfg.chunk_bytes - 1) / ctx->cfg.chunk_bytes);
    n = std::max<uint64_t>(1, std::min<uint64_t>(n, std::max<uint64_t>(1, csize / 64)));
    const uint64_t per = (csize + n - 1) / n;
    // symbols expected per part: ISIZE is exact below 4 GiB; 2x the compressed size bounds text otherwise
    const uint64_t d_est = std::max<uint64_t>(mi.isize, 2 * csize);
    const uint64_t cap = std::min<uint64_t>(round_up(2 * d_est / n + 65536, 8), kMaxPartSymbols);
    F.chunk0 = (int32_t)P.chunks.size();
    F.nchunks = (int32_t)n;
    for (uint64_t i = 0; i < n; ++i) {
        ChunkDesc C{};
        C.lo = (mi.s0 + i * per) * 8;
        C.hi = std::min<uint64_t>((mi.s0 + (i + 1) * per) * 8, F.end_bit);
        C.file = (int32_t)P.files.size();
        C.index = (int32_t)i;
        C.disabled = (i > 0 && C.lo >= F.end_bit) ? 1u : 0u;
        C.cap = cap;
        C.stop_hint = kNone;
        C.sync = kNone;
        P.chunks.push_back(C);
    }
    // window-chain groups of about sqrt(n) parts
    const uint64_t gsz = std::max<uint64_t>(1, (uint64_t)std::ceil(std::sqrt((double)n)));
    F.group0 = (int32_t)P.g0.size();
    F.ngroups = 0;
    for (uint64_t a = 0; a < n; a += gsz) {
        P.g0.push_back(F.chunk0 + (int32_t)a);
        P.gn.push_back((int32_t)std::min<uint64_t>(gsz, n - a));
        P.gfile.push_back((int32_t)P.files.size());
        F.ngroups++;
    }
    P.files.push_back(F);
}

// symbol offsets, CRC segments, device buffers
int layout(Plan& P) {
    uint64_t base = 0, mx = 0;
    for (auto& C : P.chunks) {
        C.cap = round_up(C.cap, 8);
        C.sym_base = base;
        base += C.cap;
        mx = std::max(mx, C.cap);
    }
    P.sym_total = base;
    P.max_cap = mx;
    P.seg0.clear();
    uint64_t seg = 0;
    for (auto& F : P.files) {
        uint64_t cap_sum = 0;
        for (int c = F.chunk0; c < F.chunk0 + F.nchunks; ++c) cap_sum += P.chunks[c].cap;
        const uint64_t bound = std::min(F.out_cap, cap_sum);
        F.seg0 = seg;
        F.nseg = (bound + crc_segment_bytes() - 1) / crc_segment_bytes();
        P.seg0.push_back(seg);
        seg += F.nseg;
    }
    P.total_seg = seg;
    // longest expected work first: a part's symbol capacity is planned from its member's expected output per
    // part (ranges: the indexed part's length), so parts with more output to produce start earlier and the
    // short ones fill the end of the persistent launches; parts that will not run go last
    P.order.resize(P.chunks.size());
    for (size_t c = 0; c < P.order.size(); ++c) P.order[c] = (uint32_t)c;
    std::stable_sort(P.order.begin(), P.order.end(), [&](uint32_t a, uint32_t b) {
        const ChunkDesc &A = P.chunks[a], &B = P.chunks[b];
        const uint64_t wa = A.disabled ? 0 : A.cap, wb = B.disabled ? 0 : B.cap;
        return wa > wb;
    });
    const size_t nf = P.files.size(), nc = P.chunks.size(), ng = P.g0.size();
    cudaError_t e = cudaSuccess;
    if (!e) e = P.d_files.ensure(nf * sizeof(FileDesc));
    if (!e) e = P.d_chunks.ensure(nc * sizeof(ChunkDesc));
    if (!e) e = P.d_g0.ensure(ng * sizeof(int32_t));
    if (!e) e = P.d_gn.ensure(ng * sizeof(int32_t));
    if (!e) e = P.d_gfile.ensure(ng * sizeof(int32_t));
    if (!e) e = P.d_seg0.ensure(nf * sizeof(uint64_t));
    if (!e) e = P.d_sym.ensure(P.sym_total * sizeof(uint16_t));
    if (!e) e = P.d_tok.ensure((size_t)pass1_warps((int)nc, P.wpb) * token_words_per_part() * sizeof(uint32_t));
    if (!e) e = P.d_queue.ensure(2 * sizeof(uint32_t));
    if (!e) e = P.d_order.ensure(nc * sizeof(uint32_t));
    if (!e && P.chain) e = P.d_windows.ensure(nc * (size_t)kWin);
    if (!e && P.chain) e = P.d_gmaps.ensure(ng * (size_t)kWin * sizeof(uint16_t));
    if (!e && P.chain) e = P.d_wstart.ensure(ng * (size_t)kWin);
    if (!e) e = P.h_files.ensure(nf * sizeof(FileDesc));
    if (!e) e = P.h_chunks.ensure(nc * sizeof(ChunkDesc));
    if (!e) e = P.h_static.ensure(3 * round_up(ng * sizeof(int32_t), 16) + round_up(nf * sizeof(uint64_t), 16) +
                                  round_up(nc * sizeof(uint32_t), 16));
    return cuda_status(e);
}

// the device-resident part of a run: uploads, every stage, result download
// the plan's static arrays (outside any graph capture), staged in pinned memory: a copy from pageable memory
// is staged by the driver and may reach the copy engine after pinned copies issued later (the next group of
// compressed bytes of a host-buffer batch), so that the run would wait for them
void upload_static(Plan& P, cudaStream_t s) {
    const size_t nf = P.files.size(), ng = P.g0.size(), nc = P.order.size();
    uint8_t* h = P.h_static.as<uint8_t>();
    size_t off = 0;
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (bytes) {
            memcpy(h + off, src, bytes);
            cudaMemcpyAsync(dst, h + off, bytes, cudaMemcpyHostToDevice, s);
        }
        off += round_up(bytes, 16);
    };
    put(P.d_g0.p, P.g0.data(), ng * sizeof(int32_t));
    put(P.d_gn.p, P.gn.data(), ng * sizeof(int32_t));
    put(P.d_gfile.p, P.gfile.data(), ng * sizeof(int32_t));
    put(P.d_seg0.p, P.seg0.data(), nf * sizeof(uint64_t));
    put(P.d_order.p, P.order.data(), nc * sizeof(uint32_t));
}

// up/up_done (optional): the plan's uploads go on stream `up` instead, and the run waits for them (event
// up_done); see pgz_decompress_batch_host
int enqueue(pgz_ctx* ctx, Plan& P, cudaStream_t s, bool timed, cudaStream_t up = nullptr,
            cudaEvent_t up_done = nullptr) {
    const size_t nf = P.files.size(), nc = P.chunks.size(), ng = P.g0.size();
    const cudaStream_t u = up ? up : s;
    memcpy(P.h_files.p, P.files.data(), nf * sizeof(FileDesc));
    memcpy(P.h_chunks.p, P.chunks.data(), nc * sizeof(ChunkDesc));
    cudaMemcpyAsync(P.d_files.p, P.h_files.p, nf * sizeof(FileDesc), cudaMemcpyHostToDevice, u);
    cudaMemcpyAsync(P.d_chunks.p, P.h_chunks.p, nc * sizeof(ChunkDesc), cudaMemcpyHostToDevice, u);
    if (up && (cudaEventRecord(up_done, up) != cudaSuccess || cudaStreamWaitEvent(s, up_done, 0) != cudaSuccess))
        return PGZ_E_CUDA;
    FileDesc* df = P.d_files.as<FileDesc>();
    ChunkDesc* dc = P.d_chunks.as<ChunkDesc>();
    uint16_t* sym = P.d_sym.as<uint16_t>();
    int k = 0;
    if (timed) cudaEventRecord(ctx->ev[0], s);
    launch_sync(df, dc, (int)nc, sym, P.d_tok.as<uint32_t>(), P.d_queue.as<uint32_t>(), P.d_order.as<uint32_t>(),
                ctx->kp, s);
    if (cudaPeekAtLastError() != cudaSuccess) return PGZ_E_CUDA;
    if (timed) cudaEventRecord(ctx->ev[1], s);
    launch_inflate(df, dc, (int)nc, sym, P.d_tok.as<uint32_t>(), P.d_queue.as<uint32_t>() + 1,
                   P.d_order.as<uint32_t>(), ctx->kp, s);
    if (cudaPeekAtLastError() != cudaSuccess) return PGZ_E_CUDA;
    launch_plan(df, dc, (int)nf, s);
    k += 3;
    if (timed) cudaEventRecord(ctx->ev[2], s);
    if (P.chain) {
        launch_chain(df, dc, (int)nf, (int)ng, P.d_g0.as<int32_t>(), P.d_gn.as<int32_t>(), P.d_gfile.as<int32_t>(),
                     sym, P.d_gmaps.as<uint16_t>(), P.d_wstart.as<uint8_t>(), P.d_windows.as<uint8_t>(), s);
        k += 3;
    }
    if (timed) cudaEventRecord(ctx->ev[3], s);
    if (P.translate) {
        launch_translate(df, dc, (int)nc, P.max_cap, sym, P.d_windows.as<uint8_t>(), P.fill, s);
        k += 1;
    }
    if (timed) cudaEventRecord(ctx->ev[4], s);
    if (P.crc) {
        launch_crc(df, (int)nf, P.total_seg, P.d_seg0.as<uint64_t>(), s);
        launch_finalize(df, (int)nf, s);
        k += 2;
    }
    if (timed) cudaEventRecord(ctx->ev[5], s);
    cudaMemcpyAsync(P.h_files.p, P.d_files.p, nf * sizeof(FileDesc), cudaMemcpyDeviceToHost, s);
    ctx->launches += (uint64_t)k;
    return cuda_status(cudaGetLastError());
}

int read_chunks(pgz_ctx* ctx, Plan& P) {
    cudaMemcpyAsync(P.h_chunks.p, P.d_chunks.p, P.chunks.size() * sizeof(ChunkDesc), cudaMemcpyDeviceToHost,
                    ctx->stream);
    return cuda_status(cudaStreamSynchronize(ctx->stream));
}

// placeholder counts of the last run's parts (after the run; not timed), then the results
int count_and_read_chunks(pgz_ctx* ctx, Plan& P) {
    launch_count_ph(P.d_chunks.as<ChunkDesc>(), (int)P.chunks.size(), P.d_sym.as<uint16_t>(), ctx->stream);
    if (cudaPeekAtLastError() != cudaSuccess) return PGZ_E_CUDA;
    return read_chunks(ctx, P);
}

// Adjusts the plan after a failed run; returns true if a re-run may succeed (an overflowing part gets twice
// its symbol capacity; the rest is recover_member's).
bool recover(pgz_ctx* ctx, Plan& P, int f, const ChunkDesc* res, uint64_t* false_syncs) {
    int grow = -1;
    const int a = recover_member(P.files[f], P.chunks.data(), res, ctx->kp.confirm_blocks, false_syncs, &grow);
    if (a == kRecoverGrow) {
        ChunkDesc& C = P.chunks[grow];
        if (C.cap >= kMaxPartSymbols) return false;
        C.cap = std::min<uint64_t>(C.cap * 2, kMaxPartSymbols);
        return true;
    }
    return a == kRecoverRerun;
}

void reset_results(Plan& P) {
    for (auto& C : P.chunks) {
        C.sync = kNone;
        C.state = CS_PENDING;
        C.err = 0;
        C.n = C.nph = C.last_ph = C.end = C.out_off = C.resume = 0;
        C.det = kNone;
        C.blocks = C.final = 0;
    }
    for (auto& F : P.files) {
        F.total = 0;
        F.crc_acc = F.crc = 0;
        F.status = PGZ_OK;
        F.bad_chunk = 0xffffffffu;
        F.bad_err = 0;
    }
}

void fill_stats(pgz_ctx* ctx, const Plan& P, pgz_stats* st, uint64_t retries, uint64_t false_syncs, bool timed,
                const ChunkDesc* res) {
    if (!st) return;
    memset(st, 0, sizeof *st);
    for (const auto& F : P.files) {
        st->in_bytes += F.gz_len;
    }
    const FileDesc* hf = P.h_files.as<FileDesc>();
    for (size_t f = 0; f < P.files.size(); ++f) st->out_bytes += hf[f].total;
    st->chunks = P.chunks.size();
    st->retries = retries;
    st->false_syncs = false_syncs;
    if (res) {
        for (size_t c = 0; c < P.chunks.size(); ++c) {
            if (res[c].state == CS_EMPTY) st->empty_chunks++;
            st->placeholders += res[c].nph;
            st->symbols += res[c].n;
            if (res[c].state == CS_DONE && res[c].det < res[c].n) st->determined += res[c].n - res[c].det;
        }
    }
    if (timed) {
        cudaEventElapsedTime(&st->ms_sync, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&st->ms_inflate, ctx->ev[1], ctx->ev[2]);
        cudaEventElapsedTime(&st->ms_chain, ctx->ev[2], ctx->ev[3]);
        cudaEventElapsedTime(&st->ms_translate, ctx->ev[3], ctx->ev[4]);
        cudaEventElapsedTime(&st->ms_crc, ctx->ev[4], ctx->ev[5]);
        cudaEventElapsedTime(&st->ms_total, ctx->ev[0], ctx->ev[5]);
    }
}

// the first half of a run of a plan: buffers, uploads and every launch, all asynchronous on the context's
// stream
int start_run(pgz_ctx* ctx, Plan& P, bool timed, cudaStream_t up = nullptr, cudaEvent_t up_done = nullptr) {
    P.wpb = ctx->kp.wpb;
    reset_results(P);
    int e = layout(P);
    if (e) return e;
    upload_static(P, up ? up : ctx->stream);
    return enqueue(ctx, P, ctx->stream, timed, up, up_done);
}

// the second half: waits for the run, then re-runs with recovery until the plan succeeds or cannot
int finish_run(pgz_ctx* ctx, Plan& P, pgz_stats* st) {
    uint64_t retries = 0, false_syncs = 0;
    const bool timed = st != nullptr;
    int status = PGZ_OK;
    for (;;) {
        int e = PGZ_OK;
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
        const FileDesc* hf = P.h_files.as<FileDesc>();
        bool again = false;
        status = PGZ_OK;
        bool need_chunks = false;
        for (size_t f = 0; f < P.files.size(); ++f)
            if (hf[f].bad_chunk != 0xffffffffu) need_chunks = true;
        if (need_chunks || st) {
            e = st ? count_and_read_chunks(ctx, P) : read_chunks(ctx, P);
            if (e) return e;
        }
        P.results_valid = true;
        const ChunkDesc* res = P.h_chunks.as<ChunkDesc>();
        for (size_t f = 0; f < P.files.size(); ++f) {
            P.files[f].total = hf[f].total;
            P.files[f].member_end = hf[f].member_end;
            P.files[f].status = hf[f].status;
            if (hf[f].status == PGZ_OK) continue;
            if (hf[f].bad_chunk != 0xffffffffu && retries < (uint64_t)kMaxRetries &&
                recover(ctx, P, (int)f, res, &false_syncs)) {
                again = true;
            } else if (status == PGZ_OK) {
                status = (int)hf[f].status;
            }
        }
        if (again) {
            ++retries;
            e = start_run(ctx, P, timed);
            if (e) return e;
            continue;
        }
        if (need_chunks || st) {
            for (size_t c = 0; c < P.chunks.size(); ++c) {   // keep the results for inspection
                P.chunks[c].sync = res[c].sync;
                P.chunks[c].n = res[c].n;
                P.chunks[c].nph = res[c].nph;
                P.chunks[c].last_ph = res[c].last_ph;
                P.chunks[c].state = res[c].state;
                P.chunks[c].out_off = res[c].out_off;
            }
        }
        fill_stats(ctx, P, st, retries, false_syncs, timed, (need_chunks || st) ? res : nullptr);
        return status;
    }
}

// runs a plan to completion, with recovery re-runs
int execute(pgz_ctx* ctx, Plan& P, pgz_stats* st) {
    const int e = start_run(ctx, P, st != nullptr);
    if (e) return e;
    return finish_run(ctx, P, st);
}

// a byte range [d_off, d_off + len) of an indexed member as a mode-2 member of P:
// the indexed parts covering it, each from its known block start, the last one
// up to the next indexed start; wins receives (part in P, indexed part) pairs
// whose windows come from the index
void plan_range(Plan& P, const pgz_index* idx, uint64_t d_off, uint64_t len, uint8_t* out,
                std::vector<std::pair<size_t, size_t>>& wins) {
    const size_t np = idx->sync.size();
    size_t a = 0;
    while (a + 1 < np && idx->off[a + 1] <= d_off) ++a;
    size_t b = a;
    while (b + 1 < np && idx->off[b + 1] < d_off + len) ++b;
    const MemberInfo& mi = idx->info[0];
    FileDesc F{};
    F.gz = idx->gz;
    F.gz_len = idx->gz_len;
    F.out = out;
    F.out_cap = len;
    F.s0_bit = mi.s0 * 8;
    F.end_bit = (idx->gz_len - 8) * 8;
    F.mode = 2;
    F.out_base = idx->off[a];
    F.out_lo = d_off;
    F.out_hi = d_off + len;
    F.chunk0 = (int32_t)P.chunks.size();
    F.nchunks = (int32_t)(b - a + 1);
    F.group0 = (int32_t)P.g0.size();
    F.ngroups = 0;
    for (size_t k = a; k <= b; ++k) {
        ChunkDesc C{};
        C.lo = idx->sync[k];
        C.hi = idx->sync[k] + 1;
        C.file = (int32_t)P.files.size();
        C.index = (int32_t)k;
        C.given = 1;
        C.stop_hint = (k == b) ? idx->stop[k] : kNone;
        C.sync = kNone;
        C.cap = round_up(idx->n[k] + 8, 8);
        wins.emplace_back(P.chunks.size(), k);
        P.chunks.push_back(C);
    }
    P.files.push_back(F);
}

void copy_range_windows(Plan& P, const pgz_index* idx, const std::vector<std::pair<size_t, size_t>>& wins,
                        cudaStream_t s) {
    for (const auto& w : wins)
        cudaMemcpyAsync(P.d_windows.as<uint8_t>() + w.first * kWin, idx->windows.as<uint8_t>() + w.second * kWin, kWin,
                        cudaMemcpyDeviceToDevice, s);
}

// One segment of a streamed member as a mode-3 member of P.  The device holds the member's bytes
// [win_lo, win_lo + win_len) at win; bit positions are relative to win_lo.  Part 0 starts at the known
// block start b (the member's first block when first); parts 1.. search equal shares of [b, seg_end);
// unless the segment is the last, a probe part searches [seg_end, probe_hi) for the block start where the
// next segment begins, and the last part stops there.  The last segment's bytes end with the trailer.
void plan_segment(pgz_ctx* ctx, Plan& P, const uint8_t* win, uint64_t win_len, uint64_t b, uint64_t seg_end,
                  uint64_t probe_hi, bool first, bool last, const uint8_t* win0, uint64_t out_before,
                  uint32_t crc_in, uint32_t crc_expect, uint32_t isize, uint64_t cap_mul) {
    FileDesc F{};
    F.gz = win;
    F.gz_len = win_len;
    F.s0_bit = b;
    F.end_bit = last ? (win_len - 8) * 8 : win_len * 8;
    F.crc_expect = crc_expect;
    F.isize_expect = isize;
    F.mode = 3;
    F.out_hi = kNone;
    F.win0 = first ? nullptr : win0;
    F.out_before = out_before;
    F.crc_in = crc_in;
    F.last_seg = last ? 1u : 0u;
    const uint64_t stop = last ? F.end_bit : seg_end;
    const uint64_t csize = (stop - b + 7) / 8;
    uint64_t n;
    if (ctx->cfg.n_chunks > 0) n = (uint64_t)ctx->cfg.n_chunks;
    else n = std::max<uint64_t>(1, (csize + ctx->cfg.chunk_bytes - 1) / ctx->cfg.chunk_bytes);
    n = std::max<uint64_t>(1, std::min<uint64_t>(n, std::max<uint64_t>(1, csize / 64)));
    const uint64_t per = (stop - b + n - 1) / n;     // bits
    // symbols per part: 2x the compressed size bounds text; an overflow doubles the part's capacity
    const uint64_t cap = std::min<uint64_t>(round_up(cap_mul * (4 * csize / n + 65536), 8), kMaxPartSymbols);
    F.chunk0 = (int32_t)P.chunks.size();
    const uint64_t np = n + (last ? 0 : 1);
    F.nchunks = (int32_t)np;
    uint64_t cap_sum = 0;
    for (uint64_t i = 0; i < np; ++i) {
        ChunkDesc C{};
        if (i < n) {
            C.lo = b + i * per;
            C.hi = std::min<uint64_t>(b + (i + 1) * per, stop);
            C.disabled = (i > 0 && C.lo >= stop) ? 1u : 0u;
        } else {
            C.lo = seg_end;
            C.hi = probe_hi;
            C.probe = 1;
        }
        if (i == 0) {
            C.hi = b + 1;
            C.given = first ? 0u : 1u;
        }
        C.file = (int32_t)P.files.size();
        C.index = (int32_t)(i + (first ? 0 : 1));     // part 0 of the member only in the first segment
        C.cap = cap;
        C.stop_hint = kNone;
        C.sync = kNone;
        cap_sum += cap;
        P.chunks.push_back(C);
    }
    F.out_cap = cap_sum;                              // the caller sizes the output buffer to it
    const uint64_t gsz = std::max<uint64_t>(1, (uint64_t)std::ceil(std::sqrt((double)np)));
    F.group0 = (int32_t)P.g0.size();
    F.ngroups = 0;
    for (uint64_t a = 0; a < np; a += gsz) {
        P.g0.push_back(F.chunk0 + (int32_t)a);
        P.gn.push_back((int32_t)std::min<uint64_t>(gsz, np - a));
        P.gfile.push_back((int32_t)P.files.size());
        F.ngroups++;
    }
    P.files.push_back(F);
}

// BGZF (SAM/BAM specification): a member whose FEXTRA holds the subfield
// SI1 = 'B', SI2 = 'C', SLEN = 2 carries its total size minus one; *size is
// that total.  h holds `avail` bytes from the member start.
bool bgzf_member_size(const uint8_t* h, uint64_t avail, uint64_t* size) {
    if (avail < 18 || h[0] != 0x1f || h[1] != 0x8b || h[2] != 8 || !(h[3] & 4)) return false;
    const uint32_t xlen = h[10] | ((uint32_t)h[11] << 8);
    if (12ull + xlen > avail) return false;
    for (uint32_t q = 12; q + 4 <= 12 + xlen;) {
        const uint32_t slen = h[q + 2] | ((uint32_t)h[q + 3] << 8);
        if (h[q] == 'B' && h[q + 1] == 'C' && slen == 2 && q + 6 <= 12 + xlen) {
            *size = (uint64_t)(h[q + 4] | ((uint32_t)h[q + 5] << 8)) + 1;
            return true;
        }
        q += 4 + slen;
    }
    return false;
}

}  // namespace

namespace {

void begin_plan(Plan& P);

// header of the member starting at byte `off` of gz (device memory): *s0 receives the absolute byte offset
// of its DEFLATE data; PGZ_E_HEADER if no member header starts there
int member_header_at(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint64_t off, uint64_t* s0) {
    if (off >= gz_len || gz_len - off < 18) return PGZ_E_HEADER;
    const uint64_t rest = gz_len - off;
    uint64_t want = std::min<uint64_t>(rest, 4096);
    for (;;) {
        if (cuda_status(ctx->hdr.ensure(want))) return PGZ_E_NOMEM;
        uint8_t* h = ctx->hdr.as<uint8_t>();
        if (cudaMemcpyAsync(h, gz + off, want, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return PGZ_E_CUDA;
        uint64_t s = 0;
        const int r = parse_header(h, want, rest, &s);
        if (r == -1 && want < rest) {
            want = std::min<uint64_t>(rest, want * 4);
            continue;
        }
        if (r != PGZ_OK) return PGZ_E_HEADER;
        *s0 = off + s;
        return PGZ_OK;
    }
}

void add_stats(pgz_stats* acc, const pgz_stats& s) {
    acc->in_bytes += s.in_bytes;
    acc->out_bytes += s.out_bytes;
    acc->chunks += s.chunks;
    acc->empty_chunks += s.empty_chunks;
    acc->false_syncs += s.false_syncs;
    acc->retries += s.retries;
    acc->placeholders += s.placeholders;
    acc->symbols += s.symbols;
    acc->ms_sync += s.ms_sync;
    acc->ms_inflate += s.ms_inflate;
    acc->ms_chain += s.ms_chain;
    acc->ms_translate += s.ms_translate;
    acc->ms_crc += s.ms_crc;
    acc->ms_total += s.ms_total;
    acc->determined += s.determined;
}

// Every member of gz (device memory, 4-byte aligned), outputs concatenated in out (RFC 1952 2.2: a gzip
// file is a series of members).  When every member is a BGZF member (its size in its header), the members
// are found by walking the headers and decoded in one run; otherwise member after member, each decoded
// as an open member whose end is where its final block ends.
int decompress_members(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint8_t* out, uint64_t out_cap,
                       uint64_t* out_len, pgz_stats* st) {
    *out_len = 0;
    if (st) memset(st, 0, sizeof *st);
    if (gz_len < 18) return PGZ_E_HEADER;
    {   // BGZF: the whole stream is read once on the host to walk the headers
        const uint64_t first = std::min<uint64_t>(gz_len, 4096);
        if (cuda_status(ctx->hdr.ensure(first))) return PGZ_E_NOMEM;
        uint8_t* h = ctx->hdr.as<uint8_t>();
        if (cudaMemcpyAsync(h, gz, first, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return PGZ_E_CUDA;
        uint64_t sz = 0;
        if (bgzf_member_size(h, first, &sz) && sz < gz_len) {
            if (cuda_status(ctx->hdr.ensure(gz_len))) return PGZ_E_NOMEM;
            h = ctx->hdr.as<uint8_t>();
            if (cudaMemcpyAsync(h, gz, gz_len, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                return PGZ_E_CUDA;
            std::vector<std::pair<uint64_t, uint64_t>> mem;
            bool ok = true;
            for (uint64_t off = 0; off < gz_len && ok;) {
                ok = bgzf_member_size(h + off, gz_len - off, &sz) && sz >= 18 && sz <= gz_len - off;
                if (ok) mem.emplace_back(off, sz);
                off += ok ? sz : 0;
            }
            if (ok) {
                Plan& P = ctx->plan;
                begin_plan(P);
                uint64_t o = 0;
                for (const auto& m : mem) {
                    const uint8_t* mh = h + m.first;
                    uint64_t hl = 0;
                    if (parse_header(mh, m.second, m.second, &hl) != PGZ_OK) return PGZ_E_HEADER;
                    const uint8_t* tr = mh + m.second - 8;
                    MemberInfo mi;
                    mi.s0 = m.first + hl;
                    mi.crc = tr[0] | ((uint32_t)tr[1] << 8) | ((uint32_t)tr[2] << 16) | ((uint32_t)tr[3] << 24);
                    mi.isize = tr[4] | ((uint32_t)tr[5] << 8) | ((uint32_t)tr[6] << 16) | ((uint32_t)tr[7] << 24);
                    if (o + mi.isize > out_cap) {                 // size needed: the sum of the ISIZE fields
                        uint64_t need = o;
                        for (size_t k = P.files.size(); k < mem.size(); ++k) {
                            const uint8_t* t2 = h + mem[k].first + mem[k].second - 4;
                            need += t2[0] | ((uint32_t)t2[1] << 8) | ((uint32_t)t2[2] << 16) | ((uint32_t)t2[3] << 24);
                        }
                        *out_len = need;
                        return PGZ_E_CAPACITY;
                    }
                    plan_member(ctx, P, gz, m.first + m.second, out + o, mi.isize, mi, 0);
                    o += mi.isize;
                }
                const int e = execute(ctx, P, st);
                uint64_t total = 0;
                for (const auto& F : P.files) total += F.total;
                *out_len = total;
                return e;
            }
        }
    }
    uint64_t off = 0, total = 0;
    for (;;) {
        uint64_t s0 = 0;
        int e = member_header_at(ctx, gz, gz_len, off, &s0);
        if (e) return off == 0 ? e : PGZ_E_UNSUPPORTED;        // data after a member that is no member
        MemberInfo mi;
        mi.s0 = s0;
        mi.crc = mi.isize = 0;                                  // read by the device at the member's end
        Plan& P = ctx->plan;
        begin_plan(P);
        plan_member(ctx, P, gz, gz_len, total < out_cap ? out + total : out + out_cap,
                    total < out_cap ? out_cap - total : 0, mi, 0);
        P.files[0].open_end = 1;
        pgz_stats s1;
        e = execute(ctx, P, st ? &s1 : nullptr);
        if (st) add_stats(st, s1);
        total += P.files[0].total;
        *out_len = total;
        if (e) return e;
        off = P.files[0].member_end;
        if (off >= gz_len) return PGZ_OK;
    }
}

}  // namespace

namespace {

void begin_plan(Plan& P) {
    P.files.clear();
    P.chunks.clear();
    P.g0.clear();
    P.gn.clear();
    P.gfile.clear();
    P.seg0.clear();
    P.chain = P.translate = P.crc = true;
    P.results_valid = false;
    P.fill = nullptr;
    if (P.graph) cudaGraphExecDestroy(P.graph);
    P.graph = nullptr;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

}  // namespace

// ---------------------------------------------------------------------------
// serving state
// ---------------------------------------------------------------------------
namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvFile {
    const uint8_t* gz = nullptr;
    uint64_t gz_len = 0;
    MemberInfo mi{};
    uint64_t d_est = 0;          // decompressed size bound used for charging (ISIZE is exact below 4 GiB)
    pgz_index* idx = nullptr;    // part starts and resolved windows, built by the first range request
};

struct SrvSlot {
    pgz_ctx* ctx = nullptr;      // own stream, plan and scratch
    cudaEvent_t done = nullptr;  // recorded after the run's last operation
    bool busy = false;
    uint64_t charged = 0;
    std::vector<pgz_request*> reqs;
};

constexpr int kServerMaxBatch = 256;   // requests in one run

}  // namespace

struct pgz_server {
    pgz_config cfg{};
    uint64_t budget = 0, in_use = 0;
    std::vector<SrvFile> files;
    std::vector<SrvSlot> slots;
    std::deque<pgz_request*> queue;
};

namespace {

uint64_t request_cost(const pgz_server* S, const pgz_request* r) {
    const SrvFile& f = S->files[(size_t)r->file];
    if (r->whole) return f.gz_len + 3 * f.d_est;
    // the parts covering the range: about the range plus two parts of output
    const uint64_t csize = std::max<uint64_t>(1, f.gz_len - 8 - f.mi.s0);
    const uint64_t part_out = f.d_est / std::max<uint64_t>(1, (csize + S->cfg.chunk_bytes - 1) / std::max<uint64_t>(1, S->cfg.chunk_bytes));
    return 3 * (r->length + 2 * part_out) + 2 * S->cfg.chunk_bytes;
}

void complete(pgz_request* r, int status, uint64_t n, int* n_done) {
    r->status = status;
    r->out_len = n;
    r->t_done = now_s();
    if (n_done) ++*n_done;
}

// one run of the pass kernels over the requests of `batch` on slot s (asynchronous)
int launch_slot(pgz_server* S, SrvSlot& sl, std::vector<pgz_request*>& batch, int* n_done) {
    pgz_ctx* ctx = sl.ctx;
    // range requests need their member's index (a full decode, once per member)
    std::vector<pgz_request*> ok;
    for (pgz_request* r : batch) {
        SrvFile& f = S->files[(size_t)r->file];
        if (!r->whole && !f.idx) {
            const int e = pgz_index_build(ctx, f.gz, f.gz_len, &f.idx);
            if (e) {
                complete(r, e, 0, n_done);
                continue;
            }
        }
        if (!r->whole && (r->offset > f.idx->total || r->length > f.idx->total - r->offset)) {
            complete(r, PGZ_E_ARG, 0, n_done);
            continue;
        }
        if (!r->whole && r->length == 0) {
            complete(r, PGZ_OK, 0, n_done);
            continue;
        }
        ok.push_back(r);
    }
    batch.swap(ok);
    if (batch.empty()) return PGZ_OK;
    Plan& P = ctx->plan;
    begin_plan(P);
    std::vector<std::vector<std::pair<size_t, size_t>>> wins(batch.size());
    bool any_whole = false;
    for (size_t k = 0; k < batch.size(); ++k) {
        pgz_request* r = batch[k];
        const SrvFile& f = S->files[(size_t)r->file];
        if (r->whole) {
            plan_member(ctx, P, f.gz, f.gz_len, r->out, r->out_cap, f.mi, 0);
            any_whole = true;
        } else {
            plan_range(P, f.idx, r->offset, r->length, r->out, wins[k]);
        }
    }
    P.chain = any_whole;
    P.wpb = ctx->kp.wpb;
    reset_results(P);
    int e = layout(P);
    if (!e && cuda_status(P.d_windows.ensure(P.chunks.size() * (size_t)kWin))) e = PGZ_E_NOMEM;
    if (!e) {
        upload_static(P, ctx->stream);
        for (size_t k = 0; k < batch.size(); ++k)
            if (!batch[k]->whole) copy_range_windows(P, S->files[(size_t)batch[k]->file].idx, wins[k], ctx->stream);
        e = enqueue(ctx, P, ctx->stream, false);
    }
    if (!e && cudaEventRecord(sl.done, ctx->stream) != cudaSuccess) e = PGZ_E_CUDA;
    if (e) {
        for (pgz_request* r : batch) complete(r, e, 0, n_done);
        return e;
    }
    const double t = now_s();
    for (pgz_request* r : batch) r->t_start = t;
    sl.reqs = batch;
    sl.busy = true;
    return PGZ_OK;
}

// results of a finished run; a run that needs recovery (false start, capacity) is re-run to completion here
void finish_slot(pgz_server* S, SrvSlot& sl, int* n_done) {
    pgz_ctx* ctx = sl.ctx;
    Plan& P = ctx->plan;
    const FileDesc* hf = P.h_files.as<FileDesc>();
    bool again = false;
    for (size_t f = 0; f < P.files.size(); ++f)
        if (hf[f].bad_chunk != 0xffffffffu) again = true;
    if (again) execute(ctx, P, nullptr);
    for (size_t k = 0; k < sl.reqs.size(); ++k) {
        pgz_request* r = sl.reqs[k];
        const int st = (int)hf[k].status;
        complete(r, st, st == PGZ_OK ? (r->whole ? hf[k].total : r->length) : (r->whole ? hf[k].total : 0), n_done);
    }
    S->in_use -= sl.charged;
    sl.charged = 0;
    sl.reqs.clear();
    sl.busy = false;
}

}  // namespace


namespace {

// parts of members of the given compressed sizes (gzip header of 10 bytes) as plan_member cuts them
uint64_t parts_for(const std::vector<uint64_t>& gz_len, uint64_t c) {
    uint64_t total = 0;
    for (const uint64_t L : gz_len) {
        const uint64_t cs = L > 18 ? L - 18 : 1;
        const uint64_t n = std::max<uint64_t>(1, (cs + c - 1) / c);
        total += std::max<uint64_t>(1, std::min<uint64_t>(n, std::max<uint64_t>(1, cs / 64)));
    }
    return total;
}

// the smallest part size (>= 4096) whose part count over the members is at most `target`
uint64_t size_for_parts(const std::vector<uint64_t>& gz_len, uint64_t target) {
    uint64_t lo = 4096, hi = 4096;
    for (const uint64_t L : gz_len) hi = std::max<uint64_t>(hi, L);
    if (parts_for(gz_len, lo) <= target) return lo;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (parts_for(gz_len, mid) <= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void pgz_config_init(pgz_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->device = 0;
    cfg->cuda_stream = nullptr;
    cfg->chunk_bytes = 64 << 10;
    cfg->n_chunks = 0;
    cfg->threads_per_chunk = 32;
    for (int b = 0; b < 256; ++b)
        if (b == 9 || b == 10 || b == 13 || (b >= 32 && b <= 126)) cfg->allowed[b >> 3] |= (uint8_t)(1u << (b & 7));
    cfg->confirm_blocks = 5;
    cfg->min_block = 1024;
    cfg->max_block = 4u << 20;
    cfg->dev_mem_budget = 0;
    cfg->spin_cap = 0;
    cfg->warps_per_block = 4;
    cfg->exec_pipelined = 0;
}

int pgz_create(pgz_ctx** out, const pgz_config* cfg) {
    if (!out || !cfg) return PGZ_E_ARG;
    *out = nullptr;
    if (cfg->threads_per_chunk != 32 || cfg->confirm_blocks < 0 || (cfg->n_chunks <= 0 && cfg->chunk_bytes == 0))
        return PGZ_E_ARG;
    if (cfg->warps_per_block != 0 && cfg->warps_per_block != 2 && cfg->warps_per_block != 4 &&
        cfg->warps_per_block != 8)
        return PGZ_E_ARG;
    if (cfg->exec_pipelined != 0 && cfg->exec_pipelined != 1) return PGZ_E_ARG;
    if (cfg->determined_tail != 0 && cfg->determined_tail != 1) return PGZ_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return PGZ_E_CUDA;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return PGZ_E_CUDA;
    pgz_ctx* ctx = new (std::nothrow) pgz_ctx();
    if (!ctx) return PGZ_E_NOMEM;
    ctx->cfg = *cfg;
    ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    for (int k = 0; k < 8; ++k) ctx->kp.allowed[k] = 0;
    for (int b = 0; b < 256; ++b)
        if ((cfg->allowed[b >> 3] >> (b & 7)) & 1) ctx->kp.allowed[b >> 5] |= 1u << (b & 31);
    ctx->kp.min_block = cfg->min_block;
    ctx->kp.max_block = cfg->max_block;
    ctx->kp.confirm_blocks = cfg->confirm_blocks;
    ctx->kp.wpb = cfg->warps_per_block ? cfg->warps_per_block : 4;
    ctx->kp.pipe = cfg->exec_pipelined;
    ctx->kp.tail = cfg->determined_tail;
    upload_crc_tables();
    for (int k = 0; k < 8; ++k) cudaEventCreate(&ctx->ev[k]);
    if (cudaGetLastError() != cudaSuccess) {
        delete ctx;
        return PGZ_E_CUDA;
    }
    *out = ctx;
    return PGZ_OK;
}

void pgz_destroy(pgz_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->cfg.device);
    cudaStreamSynchronize(ctx->stream);
    ctx->plan.release();
    ctx->carry_win.release();
    for (int k = 0; k < 2; ++k) {
        ctx->sin[k].release();
        ctx->sout[k].release();
        ctx->stage[k].release();
    }
    ctx->hdr.release();
    ctx->in_buf.release();
    ctx->out_buf.release();
    ctx->fill_buf.release();
    for (int k = 0; k < 8; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    if (ctx->hb_up) cudaStreamSynchronize(ctx->hb_up);
    if (ctx->hb_down) cudaStreamSynchronize(ctx->hb_down);
    for (int g = 0; g < pgz_ctx::kHostGroups; ++g) {
        ctx->hb_plan[g].release();
        if (ctx->hb_ev_up[g]) cudaEventDestroy(ctx->hb_ev_up[g]);
        if (ctx->hb_ev_run[g]) cudaEventDestroy(ctx->hb_ev_run[g]);
    }
    ctx->hb_in.release();
    ctx->hb_out.release();
    if (ctx->hb_up) cudaStreamDestroy(ctx->hb_up);
    if (ctx->hb_down) cudaStreamDestroy(ctx->hb_down);
    delete ctx;
}

int pgz_decompress(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint8_t* out, uint64_t out_cap,
                   uint64_t* out_len, pgz_stats* st) {
    if (!ctx || !gz || !out_len || (!out && out_cap) || !aligned4(gz)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    return decompress_members(ctx, gz, gz_len, out, out_cap, out_len, st);
}

int pgz_decompress_host(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint8_t* out, uint64_t out_cap,
                        uint64_t* out_len, pgz_stats* st) {
    if (!ctx || !gz || !out_len || (!out && out_cap)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    *out_len = 0;
    if (gz_len < 18) return PGZ_E_HEADER;
    if (cuda_status(ctx->in_buf.ensure(gz_len)) || cuda_status(ctx->out_buf.ensure(out_cap))) return PGZ_E_NOMEM;
    if (cudaMemcpyAsync(ctx->in_buf.p, gz, gz_len, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return PGZ_E_CUDA;
    const int e = decompress_members(ctx, ctx->in_buf.as<uint8_t>(), gz_len, ctx->out_buf.as<uint8_t>(), out_cap,
                                     out_len, st);
    if (e == PGZ_OK && *out_len) {
        if (cudaMemcpyAsync(out, ctx->out_buf.p, *out_len, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return PGZ_E_CUDA;
    }
    return e;
}

int pgz_decompress_at(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint64_t start_bit, uint16_t* sym_out,
                      uint8_t* byte_out, uint8_t fill, uint64_t out_cap, uint64_t* out_len, uint64_t* block_bit,
                      uint64_t* first_determined) {
    if (!ctx || !gz || !out_len || !aligned4(gz)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    *out_len = 0;
    MemberInfo mi;
    int e = read_member(ctx, gz, gz_len, &mi);
    if (e) return e;
    Plan& P = ctx->plan;
    begin_plan(P);
    const uint64_t s0_bit = mi.s0 * 8, end_bit = (gz_len - 8) * 8;
    FileDesc F{};
    if (!byte_out) {                                   // the translation still counts the placeholders
        if (cuda_status(ctx->out_buf.ensure(out_cap))) return PGZ_E_NOMEM;
        byte_out = ctx->out_buf.as<uint8_t>();
    }
    F.gz = gz;
    F.gz_len = gz_len;
    F.out = byte_out;
    F.out_cap = out_cap;
    F.s0_bit = s0_bit;
    F.end_bit = end_bit;
    F.mode = 1;
    F.out_hi = kNone;
    F.chunk0 = 0;
    F.nchunks = 1;
    F.group0 = 0;
    F.ngroups = 0;
    P.files.push_back(F);
    ChunkDesc C{};
    const bool at_start = start_bit <= s0_bit;
    C.lo = at_start ? s0_bit : start_bit;
    C.hi = end_bit;
    C.index = at_start ? 0 : 1;
    C.stop_hint = kNone;
    C.sync = kNone;
    C.cap = std::min<uint64_t>(round_up(std::max<uint64_t>(out_cap, 65536), 8), kMaxPartSymbols);
    P.chunks.push_back(C);
    P.chain = false;
    P.crc = false;
    P.translate = true;
    if (cuda_status(ctx->fill_buf.ensure(kWin))) return PGZ_E_NOMEM;
    cudaMemsetAsync(ctx->fill_buf.p, fill, kWin, ctx->stream);
    P.fill = ctx->fill_buf.as<uint8_t>();
    e = execute(ctx, P, nullptr);
    if (e == PGZ_OK || e == PGZ_E_CAPACITY) {
        if (count_and_read_chunks(ctx, P)) return PGZ_E_CUDA;
    }
    const ChunkDesc* res = P.h_chunks.as<ChunkDesc>();
    if (e == PGZ_OK && res[0].state != CS_DONE) e = PGZ_E_NOSYNC;
    if (e == PGZ_E_DATA) {
        if (read_chunks(ctx, P)) return PGZ_E_CUDA;
        if (res[0].state == CS_EMPTY) e = PGZ_E_NOSYNC;
    }
    if (e == PGZ_OK) {
        *out_len = res[0].n;
        if (block_bit) *block_bit = res[0].sync;
        if (first_determined) *first_determined = res[0].last_ph;
        if (sym_out && res[0].n) {
            if (cudaMemcpyAsync(sym_out, P.d_sym.as<uint16_t>() + res[0].sym_base, res[0].n * sizeof(uint16_t),
                                cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                return PGZ_E_CUDA;
        }
    } else if (e == PGZ_E_CAPACITY) {
        *out_len = res[0].n;
    }
    return e;
}

int pgz_decompress_batch(pgz_ctx* ctx, int n, pgz_job* jobs, pgz_stats* st) {
    if (!ctx || n < 0 || (n && !jobs)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    Plan& P = ctx->plan;
    begin_plan(P);
    std::vector<int> idx;
    int first_bad = PGZ_OK;
    for (int k = 0; k < n; ++k) {
        jobs[k].out_len = 0;
        if (!jobs[k].gz || !aligned4(jobs[k].gz) || (!jobs[k].out && jobs[k].out_cap)) {
            jobs[k].status = PGZ_E_ARG;
            continue;
        }
        MemberInfo mi;
        const int e = read_member(ctx, jobs[k].gz, jobs[k].gz_len, &mi);
        if (e) {
            jobs[k].status = e;
            continue;
        }
        plan_member(ctx, P, jobs[k].gz, jobs[k].gz_len, jobs[k].out, jobs[k].out_cap, mi, 0);
        idx.push_back(k);
    }
    int e = idx.empty() ? PGZ_OK : execute(ctx, P, st);
    if (e == PGZ_E_CUDA || e == PGZ_E_NOMEM) return e;
    for (size_t f = 0; f < idx.size(); ++f) {
        jobs[idx[f]].status = (int)P.files[f].status;
        jobs[idx[f]].out_len = P.files[f].total;
    }
    for (int k = 0; k < n; ++k)
        if (jobs[k].status != PGZ_OK && first_bad == PGZ_OK) first_bad = jobs[k].status;
    return first_bad;
}

// Jobs in host memory.  The jobs are cut into up to kHostGroups groups of consecutive jobs with about equal
// compressed bytes.  All uploads are issued at once on an upload stream; each group's run of the pass
// kernels waits only for its own upload, and the runs follow each other on the context's stream with no
// host wait between them; each group's output goes down on a download stream as soon as its run ends.
// The host then collects the results group by group; a group that needs recovery (a false block start, a
// capacity) is re-run with recovery and its output copied again.
int pgz_decompress_batch_host(pgz_ctx* ctx, int n, pgz_job* jobs, pgz_stats* st) {
    if (!ctx || n < 0 || (n && !jobs)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    if (st) memset(st, 0, sizeof *st);
    if (n == 0) return PGZ_OK;
    constexpr int G = pgz_ctx::kHostGroups;
    if (!ctx->hb_up) {
        if (cudaStreamCreateWithFlags(&ctx->hb_up, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ctx->hb_down, cudaStreamNonBlocking) != cudaSuccess)
            return PGZ_E_CUDA;
        for (int g = 0; g < G; ++g)
            if (cudaEventCreateWithFlags(&ctx->hb_ev_up[g], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->hb_ev_run[g], cudaEventDisableTiming) != cudaSuccess)
                return PGZ_E_CUDA;
    }
    // headers and trailers from the host copies; device offsets (16-byte aligned) of every job
    std::vector<MemberInfo> mi((size_t)n);
    std::vector<uint64_t> in_off((size_t)n), out_off((size_t)n), down((size_t)n, 0);
    std::vector<char> valid((size_t)n, 0);
    uint64_t in_total = 0, out_total = 0;
    for (int k = 0; k < n; ++k) {
        pgz_job& J = jobs[k];
        J.out_len = 0;
        J.status = PGZ_OK;
        if (!J.gz || (!J.out && J.out_cap)) {
            J.status = PGZ_E_ARG;
            continue;
        }
        uint64_t s0 = 0;
        if (J.gz_len < 18 || parse_header(J.gz, J.gz_len, J.gz_len, &s0) != PGZ_OK) {
            J.status = PGZ_E_HEADER;
            continue;
        }
        const uint8_t* t = J.gz + J.gz_len - 8;
        mi[k].s0 = s0;
        mi[k].crc = t[0] | ((uint32_t)t[1] << 8) | ((uint32_t)t[2] << 16) | ((uint32_t)t[3] << 24);
        mi[k].isize = t[4] | ((uint32_t)t[5] << 8) | ((uint32_t)t[6] << 16) | ((uint32_t)t[7] << 24);
        in_off[k] = in_total;
        out_off[k] = out_total;
        in_total += round_up(J.gz_len, 16);
        out_total += round_up(J.out_cap, 16);
        valid[k] = 1;
    }
    if (cuda_status(ctx->hb_in.ensure(in_total)) || cuda_status(ctx->hb_out.ensure(out_total))) return PGZ_E_NOMEM;
    uint8_t* din = ctx->hb_in.as<uint8_t>();
    uint8_t* dout = ctx->hb_out.as<uint8_t>();
    // groups of consecutive jobs.  Only the first group's upload and the last group's download are not
    // overlapped with decoding, so with enough bytes there are three: a short first and last group (about
    // 15 % of the compressed bytes each) around a long middle one, whose run keeps most parts in whole waves
    // of one launch; with fewer bytes two halves, or one group.  (Measured on the 512-member batch: 102 ms a
    // call against 106 ms for three or four equal groups.)
    static_assert(G >= 3, "three host-batch groups");
    const int ng = (int)std::min<uint64_t>((uint64_t)n, in_total >= (288ull << 20) ? 3 : in_total >= (192ull << 20) ? 2 : 1);
    const double edge[3] = {ng == 3 ? 0.15 : 0.5, ng == 3 ? 0.85 : 1.0, 1.0};   // cumulative share at each group's end
    std::vector<int> gfirst((size_t)ng + 1, n);
    {
        uint64_t acc = 0;
        int g = 0;
        gfirst[0] = 0;
        for (int k = 0; k < n && g + 1 < ng; ++k) {
            acc += valid[k] ? round_up(jobs[k].gz_len, 16) : 0;
            if ((double)acc >= edge[g] * (double)in_total) gfirst[++g] = k + 1;
        }
        for (int h = g + 1; h <= ng; ++h) gfirst[h] = n;
    }
    // the groups' runs back to back.  Each group's bytes and then its run's own small uploads of the plan go
    // on the upload stream, in that order, so that a run waits for its own group's bytes only: a copy engine
    // busy with a later group's bytes would not take a plan copy waiting on another stream before that whole
    // copy ends.  Each group's output goes down as its run ends (ISIZE bytes: the length of a good member
    // below 4 GiB, corrected below when the run says otherwise).
    int status = PGZ_OK;
    std::vector<char> started((size_t)ng, 0);
    const pgz_config saved = ctx->cfg;
    const uint64_t W = ctx->cfg.n_chunks > 0 ? 0 : (uint64_t)pass1_warps(1 << 30, ctx->kp.wpb);
    for (int g = 0; g < ng; ++g) {
        Plan& P = ctx->hb_plan[g];
        begin_plan(P);
        if (W) {   // the group's parts in a whole number of waves of pass-1 warps, near the context's part size
            std::vector<uint64_t> lens;
            for (int k = gfirst[g]; k < gfirst[g + 1]; ++k)
                if (valid[k]) lens.push_back(jobs[k].gz_len);
            if (!lens.empty()) {
                const uint64_t waves = std::max<uint64_t>(1, (parts_for(lens, saved.chunk_bytes) + W / 2) / W);
                ctx->cfg.chunk_bytes = size_for_parts(lens, waves * W);
            }
        }
        for (int k = gfirst[g]; k < gfirst[g + 1]; ++k)
            if (valid[k])
                plan_member(ctx, P, din + in_off[k], jobs[k].gz_len, dout + out_off[k], jobs[k].out_cap, mi[k], 0);
        ctx->cfg = saved;
        if (P.files.empty()) continue;
        for (int k = gfirst[g]; k < gfirst[g + 1]; ++k)
            if (valid[k] && cudaMemcpyAsync(din + in_off[k], jobs[k].gz, jobs[k].gz_len, cudaMemcpyHostToDevice,
                                            ctx->hb_up) != cudaSuccess)
                return PGZ_E_CUDA;
        const int e = start_run(ctx, P, false, ctx->hb_up, ctx->hb_ev_up[g]);
        if (e) {
            status = e;
            break;
        }
        started[g] = 1;
        if (cudaEventRecord(ctx->hb_ev_run[g], ctx->stream) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->hb_down, ctx->hb_ev_run[g], 0) != cudaSuccess)
            return PGZ_E_CUDA;
        for (int k = gfirst[g]; k < gfirst[g + 1]; ++k) {
            if (!valid[k]) continue;
            down[k] = std::min<uint64_t>(jobs[k].out_cap, mi[k].isize);
            if (down[k] && cudaMemcpyAsync(jobs[k].out, dout + out_off[k], down[k], cudaMemcpyDeviceToHost,
                                           ctx->hb_down) != cudaSuccess)
                return PGZ_E_CUDA;
        }
    }
    // results, group by group (recovery re-runs a group and copies its output again)
    for (int g = 0; g < ng; ++g) {
        if (!started[g]) continue;
        Plan& P = ctx->hb_plan[g];
        uint64_t again = 0;
        {
            if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
            const FileDesc* hf = P.h_files.as<FileDesc>();
            for (size_t f = 0; f < P.files.size(); ++f) again |= hf[f].bad_chunk != 0xffffffffu;
        }
        const int e = finish_run(ctx, P, nullptr);
        if (e == PGZ_E_CUDA || e == PGZ_E_NOMEM) return e;
        const FileDesc* hf = P.h_files.as<FileDesc>();
        size_t f = 0;
        for (int k = gfirst[g]; k < gfirst[g + 1]; ++k) {
            if (!valid[k]) continue;
            jobs[k].status = (int)hf[f].status;
            jobs[k].out_len = hf[f].total;
            if (st) {
                st->in_bytes += jobs[k].gz_len;
                st->out_bytes += hf[f].total;
            }
            const uint64_t want = jobs[k].status == PGZ_OK ? hf[f].total : 0;
            if (jobs[k].status == PGZ_OK && (again || want != down[k])) {
                if (cudaMemcpyAsync(jobs[k].out, dout + out_off[k], want, cudaMemcpyDeviceToHost, ctx->hb_down) !=
                    cudaSuccess)
                    return PGZ_E_CUDA;
            }
            ++f;
        }
        if (st) st->chunks += P.chunks.size();
    }
    if (cudaStreamSynchronize(ctx->hb_down) != cudaSuccess) return PGZ_E_CUDA;
    if (status != PGZ_OK) return status;
    for (int k = 0; k < n; ++k)
        if (jobs[k].status != PGZ_OK) return jobs[k].status;
    return PGZ_OK;
}

int pgz_batch_prepare(pgz_ctx* ctx, int n, const pgz_job* jobs, pgz_batch** out) {
    if (!ctx || !out || n <= 0 || !jobs) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    *out = nullptr;
    pgz_batch* b = new (std::nothrow) pgz_batch();
    if (!b) return PGZ_E_NOMEM;
    b->ctx = ctx;
    b->jobs.assign(jobs, jobs + n);
    Plan& P = b->plan;
    begin_plan(P);
    for (int k = 0; k < n; ++k) {
        if (!jobs[k].gz || !aligned4(jobs[k].gz) || (!jobs[k].out && jobs[k].out_cap)) {
            delete b;
            return PGZ_E_ARG;
        }
        MemberInfo mi;
        const int e = read_member(ctx, jobs[k].gz, jobs[k].gz_len, &mi);
        if (e) {
            delete b;
            return e;
        }
        plan_member(ctx, P, jobs[k].gz, jobs[k].gz_len, jobs[k].out, jobs[k].out_cap, mi, 0);
    }
    // one untimed run settles the plan (capacities, false starts), then the
    // settled plan is captured
    int e = execute(ctx, P, nullptr);
    if (e == PGZ_E_CUDA || e == PGZ_E_NOMEM) {
        P.release();
        delete b;
        return e;
    }
    reset_results(P);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        P.release();
        delete b;
        return PGZ_E_CUDA;
    }
    cudaGraph_t g = nullptr;
    cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    const uint64_t before = ctx->launches;
    enqueue(ctx, P, cs, false);
    ctx->launches = before;
    cudaError_t ce = cudaStreamEndCapture(cs, &g);
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&P.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) {
        P.release();
        delete b;
        return PGZ_E_CUDA;
    }
    *out = b;
    return PGZ_OK;
}

int pgz_batch_run(pgz_batch* b, pgz_job* jobs, pgz_stats* st) {
    if (!b || !jobs) return PGZ_E_ARG;
    pgz_ctx* ctx = b->ctx;
    cudaSetDevice(ctx->cfg.device);
    Plan& P = b->plan;
    if (st) {
        memset(st, 0, sizeof *st);
        cudaEventRecord(ctx->ev[6], ctx->stream);
    }
    if (cudaGraphLaunch(P.graph, ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
    ctx->launches += (uint64_t)kernels_per_run();
    if (st) cudaEventRecord(ctx->ev[7], ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
    const FileDesc* hf = P.h_files.as<FileDesc>();
    int first_bad = PGZ_OK;
    for (size_t f = 0; f < b->jobs.size(); ++f) {
        jobs[f].status = (int)hf[f].status;
        jobs[f].out_len = hf[f].total;
        if (hf[f].status != PGZ_OK && first_bad == PGZ_OK) first_bad = (int)hf[f].status;
    }
    if (st) {
        for (size_t f = 0; f < b->jobs.size(); ++f) {
            st->in_bytes += P.files[f].gz_len;
            st->out_bytes += hf[f].total;
        }
        st->chunks = P.chunks.size();
        cudaEventElapsedTime(&st->ms_total, ctx->ev[6], ctx->ev[7]);
    }
    return first_bad;
}

void pgz_batch_free(pgz_batch* b) {
    if (!b) return;
    cudaSetDevice(b->ctx->cfg.device);
    cudaStreamSynchronize(b->ctx->stream);
    b->plan.release();
    delete b;
}

static const ChunkDesc* inspect_results(pgz_ctx* ctx) {
    Plan& P = ctx->plan;
    if (!P.results_valid || P.chunks.empty()) return nullptr;
    cudaSetDevice(ctx->cfg.device);
    if (count_and_read_chunks(ctx, P)) return nullptr;
    return P.h_chunks.as<ChunkDesc>();
}

int pgz_inspect_parts(pgz_ctx* ctx, int n, uint64_t* start_bit, uint64_t* nsym, uint64_t* nph, int* nparts) {
    if (!ctx) return PGZ_E_ARG;
    const ChunkDesc* R = inspect_results(ctx);
    if (!R) return PGZ_E_ARG;
    const Plan& P = ctx->plan;
    if (nparts) *nparts = (int)P.chunks.size();
    for (int i = 0; i < n && i < (int)P.chunks.size(); ++i) {
        const bool used = R[i].state == CS_DONE;
        if (start_bit) start_bit[i] = used ? R[i].sync : kNone;
        if (nsym) nsym[i] = used ? R[i].n : 0;
        if (nph) nph[i] = used ? R[i].nph : 0;
    }
    return PGZ_OK;
}

int pgz_inspect_symbols(pgz_ctx* ctx, int part, uint16_t* host_dst, uint64_t cap, uint64_t* nsym) {
    if (!ctx || part < 0 || part >= (int)ctx->plan.chunks.size()) return PGZ_E_ARG;
    const ChunkDesc* R = inspect_results(ctx);
    if (!R) return PGZ_E_ARG;
    const ChunkDesc& C = R[part];
    const uint64_t n = C.state == CS_DONE ? C.n : 0;
    if (nsym) *nsym = n;
    if (!host_dst || n == 0) return PGZ_OK;
    if (cap < n) return PGZ_E_CAPACITY;
    // u16 symbols before the determined tail; the tail's bytes (symbol k at byte det + k) widened
    const uint64_t nw = C.det < n ? C.det : n;
    const uint16_t* d = ctx->plan.d_sym.as<uint16_t>() + C.sym_base;
    if (nw && cudaMemcpy(host_dst, d, nw * sizeof(uint16_t), cudaMemcpyDeviceToHost) != cudaSuccess) return PGZ_E_CUDA;
    if (nw < n) {
        std::vector<uint8_t> t((size_t)(n - nw));
        if (cudaMemcpy(t.data(), reinterpret_cast<const uint8_t*>(d) + C.det + nw, n - nw, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return PGZ_E_CUDA;
        for (uint64_t k = nw; k < n; ++k) host_dst[k] = t[(size_t)(k - nw)];
    }
    return PGZ_OK;
}

int pgz_inspect_window(pgz_ctx* ctx, int part, uint8_t* host_dst) {
    if (!ctx || !host_dst || part < 0 || part >= (int)ctx->plan.chunks.size() || !ctx->plan.chain ||
        !ctx->plan.d_windows.p)
        return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    if (cudaMemcpy(host_dst, ctx->plan.d_windows.as<uint8_t>() + (uint64_t)part * kWin, kWin,
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return PGZ_E_CUDA;
    return PGZ_OK;
}

uint64_t pgz_kernel_launches(const pgz_ctx* ctx) { return ctx ? ctx->launches : 0; }

// the header's part states, error codes and actions are the library's own
static_assert((int)PGZ_PART_FOUND == (int)CS_FOUND && (int)PGZ_PART_EMPTY == (int)CS_EMPTY &&
                  (int)PGZ_PART_DONE == (int)CS_DONE && (int)PGZ_PART_ERROR == (int)CS_ERROR,
              "part states");
static_assert((int)PGZ_PART_OK == (int)CE_OK && (int)PGZ_PART_DATA == (int)CE_DATA &&
                  (int)PGZ_PART_TRUNC == (int)CE_TRUNC && (int)PGZ_PART_DIST == (int)CE_DIST &&
                  (int)PGZ_PART_OVERFLOW == (int)CE_OVERFLOW && (int)PGZ_PART_CHAIN == (int)CE_CHAIN &&
                  (int)PGZ_PART_CONFIRM == (int)CE_CONFIRM && (int)PGZ_PART_TRAIL == (int)CE_TRAIL,
              "part errors");
static_assert((int)PGZ_RECOVER_STOP == kRecoverStop && (int)PGZ_RECOVER_RERUN == kRecoverRerun &&
                  (int)PGZ_RECOVER_GROW == kRecoverGrow,
              "recovery actions");

int pgz_recover_step(int n, pgz_part_state* parts, uint64_t s0_bit, int mode, int last_seg, int confirm_blocks,
                     uint64_t* false_syncs, int* grow) {
    if (n <= 0 || !parts || !false_syncs || !grow || confirm_blocks < 0 || mode < 0 || mode > 3) return -1;
    FileDesc F{};
    F.chunk0 = 0;
    F.nchunks = n;
    F.s0_bit = s0_bit;
    F.mode = (uint32_t)mode;
    F.last_seg = last_seg ? 1u : 0u;
    std::vector<ChunkDesc> plan((size_t)n), res((size_t)n);
    for (int k = 0; k < n; ++k) {
        const pgz_part_state& q = parts[k];
        ChunkDesc& C = plan[(size_t)k];
        C = ChunkDesc{};
        C.lo = q.lo;
        C.index = k;
        C.given = q.given ? 1u : 0u;
        C.probe = q.probe ? 1u : 0u;
        C.disabled = q.disabled ? 1u : 0u;
        C.confirm_ext = q.confirm_ext ? 1u : 0u;
        ChunkDesc& R = res[(size_t)k];
        R = C;
        R.state = (uint32_t)q.state;
        R.err = (uint32_t)q.err;
        R.sync = q.sync;
        R.end = q.end;
        R.blocks = q.blocks;
        R.confirmed = q.confirmed;
    }
    int g = -1;
    const int a = recover_member(F, plan.data(), res.data(), confirm_blocks, false_syncs, &g);
    for (int k = 0; k < n; ++k) {
        parts[k].lo = plan[(size_t)k].lo;
        parts[k].disabled = (int32_t)plan[(size_t)k].disabled;
        parts[k].confirm_ext = (int32_t)plan[(size_t)k].confirm_ext;
    }
    *grow = g;
    return a;
}

int pgz_wave_chunk_bytes(pgz_ctx* ctx, const pgz_job* jobs, int n_jobs, int warps_per_block, double waves,
                         uint64_t* chunk_bytes, int* resident_warps) {
    if (!ctx || !jobs || n_jobs <= 0 || !chunk_bytes || !(waves > 0.0) ||
        (warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8))
        return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    const uint64_t W = (uint64_t)pass1_warps(1 << 30, warps_per_block);
    if (resident_warps) *resident_warps = (int)W;
    const uint64_t target = std::max<uint64_t>(1, (uint64_t)std::llround(waves * (double)W));
    std::vector<uint64_t> lens((size_t)n_jobs);
    for (int k = 0; k < n_jobs; ++k) lens[(size_t)k] = jobs[k].gz_len;
    *chunk_bytes = size_for_parts(lens, target);
    return PGZ_OK;
}

int pgz_set_tuning(pgz_ctx* ctx, uint64_t chunk_bytes, int warps_per_block, int exec_pipelined) {
    if (!ctx || chunk_bytes < 4096 || (warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8) ||
        (exec_pipelined != 0 && exec_pipelined != 1))
        return PGZ_E_ARG;
    ctx->cfg.n_chunks = 0;
    ctx->cfg.chunk_bytes = chunk_bytes;
    ctx->cfg.warps_per_block = warps_per_block;
    ctx->cfg.exec_pipelined = exec_pipelined;
    ctx->kp.wpb = warps_per_block;
    ctx->kp.pipe = exec_pipelined;
    return PGZ_OK;
}

// --------------------------------------------------------------------------- streaming
namespace {

// a streamed segment's place in the member: its first block (bit), its bytes on the device, its nominal end
struct SegGeom {
    uint64_t b, win_lo, win_hi, seg_end;
    bool last;
};

SegGeom seg_geom(uint64_t b, uint64_t segment_bytes, uint64_t look, uint64_t gz_len) {
    SegGeom g;
    const uint64_t data_end = gz_len - 8;
    const uint64_t bb = b >> 3;
    g.b = b;
    g.win_lo = bb & ~4095ull;            // the block-start scan reads from 128-byte boundaries
    g.seg_end = bb + segment_bytes;
    g.last = g.seg_end + look + 65536 >= data_end;
    g.win_hi = g.last ? gz_len : g.seg_end + look;
    return g;
}

// host -> device copies of member bytes into a streaming input buffer, on the upload stream
struct Upload {
    uint64_t lo = 0, hi = 0;             // member bytes [lo, hi) held
    cudaEvent_t done = nullptr;
};

int upload_bytes(DBuf& buf, Upload& u, const uint8_t* gz, uint64_t lo, uint64_t hi, cudaStream_t up) {
    if (cuda_status(buf.ensure(hi - lo))) return PGZ_E_NOMEM;
    if (cudaMemcpyAsync(buf.p, gz + lo, hi - lo, cudaMemcpyHostToDevice, up) != cudaSuccess) return PGZ_E_CUDA;
    if (cudaEventRecord(u.done, up) != cudaSuccess) return PGZ_E_CUDA;
    u.lo = lo;
    u.hi = hi;
    return PGZ_OK;
}

struct StreamRes {                       // per-call streams and events, released on every return
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_dn[2] = {};
    Upload upl[2];
    int init() {
        if (cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) != cudaSuccess) return PGZ_E_CUDA;
        if (cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess) return PGZ_E_CUDA;
        for (int k = 0; k < 2; ++k) {
            if (cudaEventCreateWithFlags(&ev_dn[k], cudaEventDisableTiming) != cudaSuccess) return PGZ_E_CUDA;
            if (cudaEventCreateWithFlags(&upl[k].done, cudaEventDisableTiming) != cudaSuccess) return PGZ_E_CUDA;
        }
        return PGZ_OK;
    }
    ~StreamRes() {
        if (up) cudaStreamSynchronize(up);
        if (down) cudaStreamSynchronize(down);
        for (int k = 0; k < 2; ++k) {
            if (ev_dn[k]) cudaEventDestroy(ev_dn[k]);
            if (upl[k].done) cudaEventDestroy(upl[k].done);
        }
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
    }
};

}  // namespace

// Segments alternate between two input and two output buffers.  While segment k runs on the context's
// stream, the bytes segment k + 1 can need (its first block lies in segment k's probe range) go up on an
// upload stream, and segment k - 1's output comes down on a download stream and is handed to the sink.
int pgz_decompress_stream(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint64_t segment_bytes,
                          pgz_sink sink, void* user, uint64_t* out_len, pgz_stats* st) {
    if (!ctx || !gz || !sink || !out_len) return PGZ_E_ARG;
    if (segment_bytes == 0) segment_bytes = 256ull << 20;
    if (segment_bytes < (1ull << 20)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    *out_len = 0;
    if (st) memset(st, 0, sizeof *st);
    if (gz_len < 18) return PGZ_E_HEADER;
    uint64_t s0 = 0;
    if (parse_header(gz, gz_len, gz_len, &s0) != PGZ_OK) return PGZ_E_HEADER;
    const uint8_t* t = gz + gz_len - 8;
    const uint32_t crc_expect = t[0] | ((uint32_t)t[1] << 8) | ((uint32_t)t[2] << 16) | ((uint32_t)t[3] << 24);
    const uint32_t isize = t[4] | ((uint32_t)t[5] << 8) | ((uint32_t)t[6] << 16) | ((uint32_t)t[7] << 24);
    if (s0 >= gz_len - 8) return PGZ_E_DATA;
    StreamRes R;
    if (R.init() != PGZ_OK) return PGZ_E_CUDA;
    if (cuda_status(ctx->carry_win.ensure(kWin))) return PGZ_E_NOMEM;
    Plan& P = ctx->plan;
    uint32_t reg = 0xffffffffu;          // CRC-32 register after the output so far
    uint64_t produced = 0;               // output bytes of the segments decoded so far
    uint64_t look = std::max<uint64_t>(segment_bytes / 8, 1ull << 20);
    uint64_t cap_mul = 1;
    bool first = true;
    int i = 0;                           // buffers of the current segment
    int pend = -1;                       // buffers of the output still to deliver, and its size
    uint64_t pend_n = 0;
    // hands the pending output to the sink; false if the sink stopped the decode
    auto deliver = [&]() -> int {
        if (pend < 0) return PGZ_OK;
        const int k = pend;
        pend = -1;
        if (cudaEventSynchronize(R.ev_dn[k]) != cudaSuccess) return PGZ_E_CUDA;
        if (pend_n && sink(user, ctx->stage[k].as<uint8_t>(), pend_n) != 0) return PGZ_E_ABORTED;
        *out_len += pend_n;
        return PGZ_OK;
    };
    // the caller's sink may stop the decode while a run is in flight: wait for it before returning
    auto quit = [&](int status) -> int {
        cudaStreamSynchronize(ctx->stream);
        return status;
    };
    SegGeom g = seg_geom(s0 * 8, segment_bytes, look, gz_len);
    for (;;) {
        // the segment's bytes: from the upload made while the previous segment ran, else now
        Upload& u = R.upl[i];
        if (!(u.lo <= g.win_lo && g.win_hi <= u.hi)) {
            const int e = upload_bytes(ctx->sin[i], u, gz, g.win_lo, g.win_hi, R.up);
            if (e) return quit(e);
        }
        if (cudaStreamWaitEvent(ctx->stream, u.done, 0) != cudaSuccess) return quit(PGZ_E_CUDA);
        begin_plan(P);
        plan_segment(ctx, P, ctx->sin[i].as<uint8_t>() + (g.win_lo - u.lo), g.win_hi - g.win_lo, g.b - g.win_lo * 8,
                     (g.seg_end - g.win_lo) * 8, (g.seg_end + look / 2 - g.win_lo) * 8, first, g.last,
                     ctx->carry_win.as<uint8_t>(), produced, reg, crc_expect, isize, cap_mul);
        FileDesc& F = P.files[0];
        if (cuda_status(ctx->sout[i].ensure(F.out_cap))) return quit(PGZ_E_NOMEM);
        F.out = ctx->sout[i].as<uint8_t>();
        int e = start_run(ctx, P, st != nullptr);
        if (e) return quit(e);
        // while it runs: the bytes the next segment can need, and the previous segment's output
        if (!g.last) {
            Upload& v = R.upl[i ^ 1];
            const uint64_t lo = g.seg_end & ~4095ull;
            const uint64_t hi = std::min<uint64_t>(gz_len, g.seg_end + look / 2 + segment_bytes + look + 65544);
            if (!(v.lo <= lo && hi <= v.hi)) {
                e = upload_bytes(ctx->sin[i ^ 1], v, gz, lo, hi, R.up);
                if (e) return quit(e);
            }
        }
        e = deliver();
        if (e) return quit(e);
        pgz_stats s1;
        e = finish_run(ctx, P, st ? &s1 : nullptr);
        if (st) add_stats(st, s1);
        if (e == PGZ_E_CAPACITY && cap_mul < 64) {        // more output than the capacities allowed
            cap_mul *= 2;
            continue;
        }
        if (e != PGZ_OK) {
            // a segment whose end found no block start in its look-ahead: retry with a longer one
            ChunkDesc pc{};
            if (!g.last && cudaMemcpy(&pc, P.d_chunks.as<ChunkDesc>() + F.chunk0 + F.nchunks - 1, sizeof pc,
                                      cudaMemcpyDeviceToHost) == cudaSuccess &&
                pc.state == CS_EMPTY && look < 4 * segment_bytes) {
                look *= 2;
                g = seg_geom(g.b, segment_bytes, look, gz_len);
                continue;
            }
            return e;
        }
        const FileDesc& H = P.h_files.as<FileDesc>()[0];
        const uint64_t n = H.total;
        if (n) {
            if (cuda_status(ctx->stage[i].ensure(n))) return PGZ_E_NOMEM;
            if (cudaMemcpyAsync(ctx->stage[i].p, ctx->sout[i].p, n, cudaMemcpyDeviceToHost, R.down) != cudaSuccess)
                return PGZ_E_CUDA;
        }
        if (cudaEventRecord(R.ev_dn[i], R.down) != cudaSuccess) return PGZ_E_CUDA;
        pend = i;
        pend_n = n;
        produced += n;
        reg = H.crc;
        if (g.last) return deliver();
        // the block start where the next segment begins, and the window this segment leaves before it
        ChunkDesc pc{};
        const int pr = F.chunk0 + F.nchunks - 1;
        cudaMemcpyAsync(&pc, P.d_chunks.as<ChunkDesc>() + pr, sizeof pc, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(ctx->carry_win.p, P.d_windows.as<uint8_t>() + (uint64_t)pr * kWin, kWin,
                        cudaMemcpyDeviceToDevice, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PGZ_E_CUDA;
        if (pc.state != CS_DONE || pc.sync == kNone) return PGZ_E_DATA;
        g = seg_geom(g.win_lo * 8 + pc.sync, segment_bytes, look, gz_len);
        first = false;
        cap_mul = 1;
        i ^= 1;
    }
}

// --------------------------------------------------------------------------- index / range
int pgz_index_build(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, pgz_index** idx) {
    if (!ctx || !gz || !idx || !aligned4(gz)) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    *idx = nullptr;
    MemberInfo mi;
    int e = read_member(ctx, gz, gz_len, &mi);
    if (e) return e;
    // decompress once into scratch (verifies CRC-32/ISIZE), keep the windows
    const uint64_t csize = gz_len - 8 - mi.s0;
    uint64_t cap = std::max<uint64_t>(mi.isize, 2 * csize) + 65536;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (cuda_status(ctx->out_buf.ensure(cap))) return PGZ_E_NOMEM;
        Plan& P = ctx->plan;
        begin_plan(P);
        plan_member(ctx, P, gz, gz_len, ctx->out_buf.as<uint8_t>(), cap, mi, 0);
        pgz_stats st;
        e = execute(ctx, P, &st);
        if (e == PGZ_E_CAPACITY) {
            cap = P.files[0].total + 65536;
            continue;
        }
        if (e) return e;
        pgz_index* I = new (std::nothrow) pgz_index();
        if (!I) return PGZ_E_NOMEM;
        I->gz = gz;
        I->gz_len = gz_len;
        I->total = P.files[0].total;
        I->info.push_back(mi);
        std::vector<int> parts;
        for (size_t c = 0; c < P.chunks.size(); ++c)
            if (P.chunks[c].state == CS_DONE) parts.push_back((int)c);
        for (size_t k = 0; k < parts.size(); ++k) {
            const ChunkDesc& C = P.chunks[parts[k]];
            I->sync.push_back(C.sync);
            I->off.push_back(C.out_off);
            I->n.push_back(C.n);
            I->stop.push_back(k + 1 < parts.size() ? P.chunks[parts[k + 1]].sync : kNone);
        }
        if (cuda_status(I->windows.ensure(parts.size() * (size_t)kWin))) {
            delete I;
            return PGZ_E_NOMEM;
        }
        for (size_t k = 0; k < parts.size(); ++k)
            cudaMemcpyAsync(I->windows.as<uint8_t>() + k * kWin, P.d_windows.as<uint8_t>() + (uint64_t)parts[k] * kWin,
                            kWin, cudaMemcpyDeviceToDevice, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            I->windows.release();
            delete I;
            return PGZ_E_CUDA;
        }
        *idx = I;
        return PGZ_OK;
    }
    return PGZ_E_CAPACITY;
}

int pgz_index_info(const pgz_index* idx, uint64_t* total_out, uint64_t* nparts) {
    if (!idx) return PGZ_E_ARG;
    if (total_out) *total_out = idx->total;
    if (nparts) *nparts = idx->sync.size();
    return PGZ_OK;
}

int pgz_decompress_range(pgz_ctx* ctx, const pgz_index* idx, uint64_t d_off, uint64_t len, uint8_t* out) {
    if (!ctx || !idx || (!out && len)) return PGZ_E_ARG;
    if (d_off > idx->total || len > idx->total - d_off) return PGZ_E_ARG;
    if (len == 0) return PGZ_OK;
    cudaSetDevice(ctx->cfg.device);
    Plan& P = ctx->plan;
    begin_plan(P);
    std::vector<std::pair<size_t, size_t>> wins;
    plan_range(P, idx, d_off, len, out, wins);
    P.chain = false;
    P.crc = false;
    P.wpb = ctx->kp.wpb;
    int e = layout(P);
    if (e) return e;
    if (cuda_status(P.d_windows.ensure(P.chunks.size() * (size_t)kWin))) return PGZ_E_NOMEM;
    copy_range_windows(P, idx, wins, ctx->stream);
    e = execute(ctx, P, nullptr);
    return e;
}

void pgz_index_free(pgz_index* idx) {
    if (!idx) return;
    idx->windows.release();
    delete idx;
}

int pgz_extract_sequences(pgz_ctx* ctx, const uint16_t* sym, uint64_t n, uint32_t min_len, uint64_t* spans,
                          uint64_t max_spans, uint64_t* n_spans, uint64_t* n_undetermined) {
    if (!ctx || (!sym && n) || (!spans && max_spans) || !n_spans || !n_undetermined) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    *n_spans = *n_undetermined = 0;
    if (cuda_status(ctx->fill_buf.ensure(std::max<size_t>(kWin, 2 * sizeof(unsigned long long))))) return PGZ_E_NOMEM;
    unsigned long long* counts = ctx->fill_buf.as<unsigned long long>();
    launch_sequences(sym, n, min_len, spans, max_spans, counts, ctx->stream);
    if (cudaPeekAtLastError() != cudaSuccess) return PGZ_E_CUDA;
    if (cuda_status(ctx->hdr.ensure(2 * sizeof(unsigned long long)))) return PGZ_E_NOMEM;
    unsigned long long* h = ctx->hdr.as<unsigned long long>();
    if (cudaMemcpyAsync(h, counts, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return PGZ_E_CUDA;
    *n_spans = h[0];
    *n_undetermined = h[1];
    ctx->launches += 1;
    return PGZ_OK;
}

int pgz_autotune(pgz_ctx* ctx, pgz_job* jobs, int n_jobs, const uint64_t* chunk_bytes, int n_chunk_bytes,
                 const int* warps_per_block, int n_wpb, int sweep_exec, int reps, pgz_tune_entry* entries,
                 pgz_tune_entry* best) {
    if (!ctx || !jobs || n_jobs <= 0 || !chunk_bytes || !warps_per_block || n_chunk_bytes <= 0 || n_wpb <= 0 ||
        reps < 1)
        return PGZ_E_ARG;
    for (int a = 0; a < n_chunk_bytes; ++a)
        if (chunk_bytes[a] < 4096) return PGZ_E_ARG;
    for (int b = 0; b < n_wpb; ++b)
        if (warps_per_block[b] != 2 && warps_per_block[b] != 4 && warps_per_block[b] != 8) return PGZ_E_ARG;
    cudaSetDevice(ctx->cfg.device);
    const pgz_config saved = ctx->cfg;
    const KParams saved_kp = ctx->kp;
    const int nx = sweep_exec ? 2 : 1;
    pgz_tune_entry pick{};
    pick.status = PGZ_E_ARG;
    int first_bad = PGZ_OK;
    std::vector<float> t((size_t)reps);
    for (int a = 0; a < n_chunk_bytes; ++a) {
        for (int b = 0; b < n_wpb; ++b) {
            for (int x = 0; x < nx; ++x) {
                pgz_tune_entry e{};
                e.chunk_bytes = chunk_bytes[a];
                e.warps_per_block = warps_per_block[b];
                e.exec_pipelined = sweep_exec ? x : saved.exec_pipelined;
                ctx->cfg.n_chunks = 0;
                ctx->cfg.chunk_bytes = e.chunk_bytes;
                ctx->cfg.warps_per_block = e.warps_per_block;
                ctx->cfg.exec_pipelined = e.exec_pipelined;
                ctx->kp.wpb = e.warps_per_block;
                ctx->kp.pipe = e.exec_pipelined;
                e.status = pgz_decompress_batch(ctx, n_jobs, jobs, nullptr);   // settles buffers and plan
                for (int r = 0; r < reps && e.status == PGZ_OK; ++r) {
                    cudaEventRecord(ctx->ev[6], ctx->stream);
                    e.status = pgz_decompress_batch(ctx, n_jobs, jobs, nullptr);
                    cudaEventRecord(ctx->ev[7], ctx->stream);
                    if (cudaEventSynchronize(ctx->ev[7]) != cudaSuccess) e.status = PGZ_E_CUDA;
                    else cudaEventElapsedTime(&t[(size_t)r], ctx->ev[6], ctx->ev[7]);
                }
                if (e.status == PGZ_OK) {
                    std::sort(t.begin(), t.end());
                    e.ms = t[(size_t)reps / 2];
                    if (pick.status != PGZ_OK || e.ms < pick.ms) pick = e;
                } else if (first_bad == PGZ_OK) {
                    first_bad = e.status;
                }
                if (entries) entries[((size_t)a * n_wpb + b) * nx + x] = e;
            }
        }
    }
    ctx->cfg = saved;
    ctx->kp = saved_kp;
    if (pick.status != PGZ_OK) return first_bad;
    ctx->cfg.n_chunks = 0;
    ctx->cfg.chunk_bytes = pick.chunk_bytes;
    ctx->cfg.warps_per_block = pick.warps_per_block;
    ctx->cfg.exec_pipelined = pick.exec_pipelined;
    ctx->kp.wpb = pick.warps_per_block;
    ctx->kp.pipe = pick.exec_pipelined;
    if (best) *best = pick;
    return PGZ_OK;
}

int pgz_server_create(pgz_server** out, const pgz_config* cfg, int slots, uint64_t mem_budget) {
    if (!out || !cfg || slots < 1 || slots > 64) return PGZ_E_ARG;
    *out = nullptr;
    pgz_server* S = new (std::nothrow) pgz_server();
    if (!S) return PGZ_E_NOMEM;
    S->cfg = *cfg;
    S->budget = mem_budget;
    S->slots.resize((size_t)slots);
    for (SrvSlot& sl : S->slots) {
        pgz_config c = *cfg;
        c.cuda_stream = nullptr;
        int e = pgz_create(&sl.ctx, &c);
        cudaStream_t st = nullptr;
        if (!e && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) e = PGZ_E_CUDA;
        if (!e) sl.ctx->stream = st;
        if (!e && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) e = PGZ_E_CUDA;
        if (e) {
            pgz_server_destroy(S);
            return e;
        }
    }
    *out = S;
    return PGZ_OK;
}

int pgz_server_add_file(pgz_server* S, const uint8_t* gz, uint64_t gz_len, int* file) {
    if (!S || !gz || !file || !aligned4(gz)) return PGZ_E_ARG;
    pgz_ctx* ctx = S->slots[0].ctx;
    cudaSetDevice(ctx->cfg.device);
    SrvFile f;
    f.gz = gz;
    f.gz_len = gz_len;
    const int e = read_member(ctx, gz, gz_len, &f.mi);
    if (e) return e;
    f.d_est = std::max<uint64_t>(f.mi.isize, gz_len < (1ull << 31) ? 0 : 2 * gz_len);
    *file = (int)S->files.size();
    S->files.push_back(f);
    return PGZ_OK;
}

int pgz_server_submit(pgz_server* S, pgz_request* r) {
    if (!S || !r || r->file < 0 || r->file >= (int)S->files.size() || (!r->out && (r->whole || r->length)))
        return PGZ_E_ARG;
    if (!r->whole && r->out_cap < r->length) return PGZ_E_ARG;
    r->status = -1;
    r->out_len = 0;
    r->t_submit = now_s();
    r->t_start = r->t_done = 0;
    S->queue.push_back(r);
    return PGZ_OK;
}

int pgz_server_poll(pgz_server* S, int* n_done) {
    if (!S) return PGZ_E_ARG;
    if (n_done) *n_done = 0;
    cudaSetDevice(S->cfg.device);
    for (SrvSlot& sl : S->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return PGZ_E_CUDA;
        finish_slot(S, sl, n_done);
    }
    // the queue is spread over the free slots (each run takes its share of the queued requests and at most
    // budget / slots of scratch), so the runs of several slots are on the GPU at once
    int free_slots = 0;
    for (const SrvSlot& sl : S->slots) free_slots += sl.busy ? 0 : 1;
    const uint64_t run_cap = S->budget ? std::max<uint64_t>(1, S->budget / S->slots.size()) : 0;
    for (SrvSlot& sl : S->slots) {
        if (sl.busy) continue;
        if (S->queue.empty()) break;
        const int share = std::max(1, (int)((S->queue.size() + free_slots - 1) / std::max(1, free_slots)));
        --free_slots;
        std::vector<pgz_request*> batch;
        uint64_t charge = 0;
        while (!S->queue.empty() && (int)batch.size() < std::min(kServerMaxBatch, share)) {
            pgz_request* r = S->queue.front();
            const uint64_t c = request_cost(S, r);
            if (S->budget && c > S->budget) {                // can never be admitted
                S->queue.pop_front();
                complete(r, PGZ_E_NOMEM, 0, n_done);
                continue;
            }
            if (S->budget && S->in_use + charge + c > S->budget) break;
            if (run_cap && !batch.empty() && charge + c > run_cap) break;
            S->queue.pop_front();
            batch.push_back(r);
            charge += c;
        }
        if (batch.empty()) break;                            // the budget is taken by running requests
        sl.charged = charge;
        S->in_use += charge;
        if (launch_slot(S, sl, batch, n_done) != PGZ_OK || !sl.busy) {
            S->in_use -= charge;
            sl.charged = 0;
        }
    }
    return PGZ_OK;
}

int pgz_server_pending(const pgz_server* S) {
    if (!S) return 0;
    int n = (int)S->queue.size();
    for (const SrvSlot& sl : S->slots) n += (int)sl.reqs.size();
    return n;
}

int pgz_server_drain(pgz_server* S) {
    if (!S) return PGZ_E_ARG;
    for (;;) {
        const int e = pgz_server_poll(S, nullptr);
        if (e) return e;
        if (pgz_server_pending(S) == 0) return PGZ_OK;
        for (SrvSlot& sl : S->slots)                         // wait for one run instead of spinning
            if (sl.busy) {
                cudaEventSynchronize(sl.done);
                break;
            }
    }
}

void pgz_server_destroy(pgz_server* S) {
    if (!S) return;
    for (SrvSlot& sl : S->slots) {
        if (sl.ctx) {
            cudaSetDevice(sl.ctx->cfg.device);
            cudaStream_t st = sl.ctx->stream;
            pgz_destroy(sl.ctx);
            if (st) cudaStreamDestroy(st);
        }
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (SrvFile& f : S->files)
        if (f.idx) pgz_index_free(f.idx);
    delete S;
}

const char* pgz_strerror(int status) {
    switch (status) {
        case PGZ_OK: return "ok";
        case PGZ_E_ARG: return "invalid argument";
        case PGZ_E_HEADER: return "not a gzip member header";
        case PGZ_E_DATA: return "invalid or truncated DEFLATE data";
        case PGZ_E_CRC: return "CRC-32 mismatch";
        case PGZ_E_ISIZE: return "ISIZE mismatch";
        case PGZ_E_CAPACITY: return "output buffer too small";
        case PGZ_E_NOSYNC: return "no block start after the offset";
        case PGZ_E_UNSUPPORTED: return "data after a gzip member that is not a gzip member";
        case PGZ_E_TIMEOUT: return "device wait timed out";
        case PGZ_E_CUDA: return "CUDA error";
        case PGZ_E_NOMEM: return "out of device memory";
        case PGZ_E_ABORTED: return "stopped by the caller's sink";
        default: return "unknown status";
    }
}

}  // extern "C"
