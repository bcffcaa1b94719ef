/*
 * pgz.h -- C ABI of libpgz: two-pass parallel gzip decompression on one GB300
 * (sm_103a), after Kerbiriou & Chikhi, "Parallel decompression of
 * gzip-compressed files and random access to DNA sequences" (arXiv 1905.07224).
 *
 * The method (Section "Full file decompression in two passes (pugz)"):
 *   (a) the compressed stream of a gzip member is cut into parts of equal
 *       compressed size; every part after the first finds the first DEFLATE
 *       block start at or after its nominal offset by trial decoding at every
 *       bit (Section "Detection of DEFLATE block start positions", Appendix
 *       "DEFLATE block decompression checks");
 *   (b) pass 1 decodes every part against a symbolic context
 *       [U_0 .. U_32767]: back-references into the unknown 32 KiB before the
 *       part stay as placeholders U_j;
 *   (c) pass 2 resolves the windows w_i (the last 32 KiB before part i) from
 *       part to part and replaces every U_j by w_i[j]; the output is then
 *       checked against the gzip trailer's CRC-32 and ISIZE (RFC 1952; the
 *       paper's own implementation does not compute the CRC, Section
 *       "Discussion").
 *
 * Conventions for every call:
 *  - Pointers named "device" must point to memory of the context's device
 *    (cudaMalloc / torch tensors); "host" pointers to host memory.  Compressed
 *    input in device memory must be 4-byte aligned; otherwise PGZ_E_ARG.
 *  - The caller owns every input and output buffer.  The context owns its
 *    scratch memory, which grows on demand and is kept between calls.
 *  - Work is issued on the context's CUDA stream (pgz_config.cuda_stream);
 *    calls return after their final status has been read back, i.e. they
 *    synchronise that stream once or twice.  pgz_decompress_stream also
 *    copies on two streams of its own, and each server slot has its own
 *    context and stream.
 *  - Return values are pgz_status codes; pgz_strerror() names them.  No call
 *    aborts the process or faults the GPU on malformed input: every device
 *    read is bounds-checked against the buffer sizes given here.
 *  - The output of a successful call is byte-exact: identical to sequential
 *    gunzip (Algorithm "DEFLATE decompression" applied from the stream start).
 */
#ifndef PGZ_H
#define PGZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pgz_status {
    PGZ_OK = 0,
    PGZ_E_ARG = 1,          /* bad argument (NULL, size, alignment, config) */
    PGZ_E_HEADER = 2,       /* not an RFC 1952 member header */
    PGZ_E_DATA = 3,         /* invalid or truncated DEFLATE data */
    PGZ_E_CRC = 4,          /* CRC-32 of the output differs from the trailer */
    PGZ_E_ISIZE = 5,        /* output length mod 2^32 differs from the trailer */
    PGZ_E_CAPACITY = 6,     /* out_cap too small; *out_len holds the size needed */
    PGZ_E_NOSYNC = 7,       /* no block start after the requested offset */
    PGZ_E_UNSUPPORTED = 8,  /* data after a member that is not a gzip member; a batch job with several members */
    PGZ_E_TIMEOUT = 9,      /* a bounded device wait gave up */
    PGZ_E_CUDA = 10,        /* a CUDA runtime call failed */
    PGZ_E_NOMEM = 11,       /* scratch allocation failed or exceeds the budget */
    PGZ_E_ABORTED = 12      /* the caller's sink stopped a streamed decode */
} pgz_status;

typedef struct pgz_ctx pgz_ctx;

typedef struct pgz_config {
    int device;                 /* CUDA device ordinal */
    void* cuda_stream;          /* cudaStream_t to issue work on; NULL = default stream */
    uint64_t chunk_bytes;       /* compressed bytes per part (used when n_chunks is 0) */
    int n_chunks;               /* > 0: exactly this many parts per file (overrides chunk_bytes) */
    int threads_per_chunk;      /* threads decoding one part: 32 (one warp) is the only value */
    uint8_t allowed[32];        /* literal bytes accepted at a block start, bit b of byte b/8 */
    int confirm_blocks;         /* blocks after a block start that must also decode (5) */
    uint32_t min_block;         /* a block start's block yields >= min_block bytes (1024) */
    uint32_t max_block;         /* ... and < max_block bytes (4 MiB) */
    uint64_t dev_mem_budget;    /* upper bound on scratch bytes; 0 = none */
    uint64_t spin_cap;          /* reserved for bounded device waits; 0 = default */
    int warps_per_block;        /* CTA shape of the pass-1 kernels: 2, 4 or 8 warps (one part each); 0 = 4 */
    int exec_pipelined;         /* 1: pass 1 executes tokens in pipelined passes, 0: one pass at a time
                                   (default); which is faster depends on the data and the part size, and
                                   pgz_autotune can choose */
    int determined_tail;        /* 1: once a part's last 32 KiB of output hold no placeholder (none can
                                   follow), pass 1 stores the rest of the part as bytes and the translation
                                   copies them; 0: u16 symbols throughout (default).  The output is the same
                                   either way; which is faster depends on how soon placeholders die out */
} pgz_config;

/* per-call statistics; the ms_* fields are CUDA-event times of the stages */
typedef struct pgz_stats {
    uint64_t in_bytes, out_bytes;
    uint64_t chunks;            /* parts planned */
    uint64_t empty_chunks;      /* parts that held no accepted block start */
    uint64_t false_syncs;       /* accepted block starts rejected by the chain check */
    uint64_t retries;           /* re-runs (false start, confirmation, capacity) */
    uint64_t placeholders;      /* placeholder symbols produced by pass 1 */
    uint64_t symbols;           /* symbols produced by pass 1 (= out_bytes) */
    float ms_sync, ms_inflate, ms_chain, ms_translate, ms_crc, ms_total;
    uint64_t determined;        /* symbols pass 1 stored as bytes: those after a point where the part's last
                                   32 KiB of output held no placeholder (none can follow; Section
                                   "Undetermined context propagation technique"), translated by a copy */
} pgz_stats;

/* One entry of a batch: device pointers; results are written back. */
typedef struct pgz_job {
    const uint8_t* gz;          /* device: one gzip member */
    uint64_t gz_len;
    uint8_t* out;               /* device: output buffer */
    uint64_t out_cap;
    uint64_t out_len;           /* result: bytes written (or needed, with PGZ_E_CAPACITY) */
    int status;                 /* result: pgz_status of this job */
} pgz_job;

typedef struct pgz_index pgz_index;
typedef struct pgz_batch pgz_batch;

/* Defaults: device 0, default stream, parts of 64 KiB of compressed data
   (about two DEFLATE blocks of zlib output; the part count of the paper's
   setting is a free parameter, Section "Full file decompression in two
   passes"), ASCII bytes 9, 10, 13, 32..126
   (reading of the Appendix's "valid ASCII characters"), confirm_blocks 5
   (Section "Detection of DEFLATE block start positions"), block bounds
   1 KiB .. 4 MiB (Appendix "DEFLATE block decompression checks"). */
void pgz_config_init(pgz_config* cfg);

/* Creates a context on cfg->device.  *out receives it; PGZ_E_ARG for a bad
   config, PGZ_E_CUDA if the device cannot be used. */
int pgz_create(pgz_ctx** out, const pgz_config* cfg);
void pgz_destroy(pgz_ctx* ctx);

/* Exact decompression of a whole gzip file (Section "Full file
   decompression in two passes (pugz)"; the result is that of Algorithm
   "DEFLATE decompression" from the stream start).  A file of several members
   (RFC 1952 2.2) gives the concatenation of their outputs, each member
   checked against its own trailer: BGZF members (their size in the header's
   'BC' subfield) are all decoded in one run; other members one after
   another, each ending where its final block ends.
   gz [device, gz_len bytes]: the gzip file; out [device, out_cap bytes].
   *out_len: bytes written; with PGZ_E_CAPACITY the bytes needed (for members
   decoded one after another: up to the member that did not fit).
   st (nullable): statistics of this call (summed over the runs). */
int pgz_decompress(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len,
                   uint8_t* out, uint64_t out_cap, uint64_t* out_len, pgz_stats* st);

/* The same with HOST buffers: the input is copied to the device and the
   output back to `out`, both inside the call. */
int pgz_decompress_host(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len,
                        uint8_t* out, uint64_t out_cap, uint64_t* out_len, pgz_stats* st);

/* Receives the output of a streamed decode in order: n bytes at `bytes`
   (pinned host memory, valid only during the call).  A non-zero return
   stops the decode with PGZ_E_ABORTED. */
typedef int (*pgz_sink)(void* user, const uint8_t* bytes, uint64_t n);

/* Memory-bounded streaming of one gzip member held in HOST memory (Section
   "Full file decompression in two passes", run over consecutive segments of
   the compressed data).  Each segment of about segment_bytes compressed
   bytes is one run of the pass kernels:
   - its first part starts at a known block start, with the resolved 32 KiB
     window the previous segment left (the member's start and an empty
     window for the first segment);
   - its other parts search their block starts as in pgz_decompress;
   - a probe part past its nominal end finds the block start where the next
     segment begins (within a look-ahead of max(segment_bytes / 8, 1 MiB),
     doubled when nothing is found there), and the segment's last part must
     end exactly on it.
   The CRC-32 register and the output length are carried from segment to
   segment on the device, and the last segment checks them against the
   trailer.  Output reaches sink(user, bytes, n) segment by segment, in
   order; when a later segment fails, the bytes already delivered stay
   delivered and the status says why the rest could not be decoded.
   Device memory in use is bounded by the segment, not by the member: about
   17 bytes per compressed byte of a segment at 64 KiB parts for data that
   expands at most 2x (input, symbol scratch, output, windows); more where a
   segment expands further, its capacities doubling on demand.
   gz [host, gz_len bytes]: one gzip member.  segment_bytes: 0 for 256 MiB,
   else at least 1 MiB (PGZ_E_ARG otherwise).  *out_len: bytes delivered to
   the sink.
   st (nullable): statistics summed over the segments' runs.
   Errors: PGZ_E_HEADER, PGZ_E_DATA, PGZ_E_CRC, PGZ_E_ISIZE and
   PGZ_E_UNSUPPORTED (data after the member) as for pgz_decompress;
   PGZ_E_ABORTED when the sink returns non-zero. */
int pgz_decompress_stream(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint64_t segment_bytes,
                          pgz_sink sink, void* user, uint64_t* out_len, pgz_stats* st);

/* Problem "Random access in DEFLATE stream" (Section "Feasibility of random
   access"): from compressed BIT offset start_bit of a gzip member, find the
   first accepted block start b >= start_bit (Section "Detection of DEFLATE
   block start positions"; if start_bit is at or before the first block, b is
   the first block and the context is known to be empty), then decode from b
   to the end of the member against the symbolic context.
   sym_out [device, nullable, out_cap u16]: symbols, 0x00..0xFF a byte,
     0x8000|j the placeholder U_j of the 32 KiB before b;
   byte_out [device, nullable, out_cap bytes]: the same with every U_j
     replaced by `fill` (the undetermined '?' context of Section
     "Undetermined context propagation technique");
   *out_len: symbols decoded; *block_bit: b; *first_determined: one past the
   last placeholder (0 if none).  PGZ_E_NOSYNC if no block start follows. */
int pgz_decompress_at(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, uint64_t start_bit,
                      uint16_t* sym_out, uint8_t* byte_out, uint8_t fill, uint64_t out_cap,
                      uint64_t* out_len, uint64_t* block_bit, uint64_t* first_determined);

/* Many independent gzip members decoded together: every stage is one launch
   over the parts of all jobs.  jobs [host array of n]; their gz/out are device
   pointers.  Returns PGZ_OK if every job succeeded, else the first failing
   job's status; each job's own status and out_len are filled in. */
int pgz_decompress_batch(pgz_ctx* ctx, int n, pgz_job* jobs, pgz_stats* st);

/* The same method over many members held in HOST memory (Section "Full
   file decompression in two passes", over a batch): jobs [host array of n],
   each job's gz and out are HOST pointers (page-locked memory lets the copies
   overlap the decoding; pageable memory works but copies synchronously).  The
   jobs are cut into groups of consecutive jobs: from 288 MiB of compressed
   bytes three (about 15 %, 70 % and 15 % of the bytes: only the first
   group's upload and the last group's download are not overlapped), from
   192 MiB two halves, else one.  Each group's part size is the one nearest
   the context's that gives a whole number of waves of pass-1 warps
   (pgz_wave_chunk_bytes; the context's size as is with n_chunks set).  Every
   group is copied to device memory owned by the context, then its run's
   plan, on one upload stream in that order, so that a run waits for its own
   group only; it is decoded by one run of the pass kernels as soon as its
   own copy has arrived, and its output copied back to the jobs' `out` while
   the next group decodes.  Statuses, out_len and the return
   value as for pgz_decompress_batch; st (nullable) receives in_bytes,
   out_bytes and chunks (the ms_* fields are not timed here).  The call returns
   when every output is in host memory. */
int pgz_decompress_batch_host(pgz_ctx* ctx, int n, pgz_job* jobs, pgz_stats* st);

/* A batch planned once and replayed as one CUDA graph: pgz_batch_prepare
   reads the jobs' headers, sizes the scratch and captures the stage
   launches; pgz_batch_run replays them on the context's stream and reads the
   results back into `jobs` (same inputs as at prepare time, which the caller
   must keep alive); pgz_batch_free releases the plan's scratch. */
int pgz_batch_prepare(pgz_ctx* ctx, int n, const pgz_job* jobs, pgz_batch** out);
int pgz_batch_run(pgz_batch* b, pgz_job* jobs, pgz_stats* st);
void pgz_batch_free(pgz_batch* b);

/* A resident random-access index of one member (the per-part block start,
   decompressed offset and resolved 32 KiB window w_i of pass 2): built by a
   full decompression, then pgz_decompress_range decodes only the parts that
   cover [d_off, d_off + len) of the decompressed stream into out [device].
   gz must stay valid and unchanged while the index is used. */
int pgz_index_build(pgz_ctx* ctx, const uint8_t* gz, uint64_t gz_len, pgz_index** idx);
int pgz_index_info(const pgz_index* idx, uint64_t* total_out, uint64_t* nparts);
int pgz_decompress_range(pgz_ctx* ctx, const pgz_index* idx, uint64_t d_off, uint64_t len, uint8_t* out);
void pgz_index_free(pgz_index* idx);

/* Inspection of the last pgz_decompress / pgz_decompress_at call on ctx, for
   tests: per part i < n the start bit (UINT64_MAX if empty), the symbol count
   of pass 1, the placeholder count, and the pass-1 symbols / the window w_i
   (copied to HOST buffers).  PGZ_E_ARG if i is out of range. */
int pgz_inspect_parts(pgz_ctx* ctx, int n, uint64_t* start_bit, uint64_t* nsym,
                      uint64_t* nph, int* nparts);
int pgz_inspect_symbols(pgz_ctx* ctx, int part, uint16_t* host_dst, uint64_t cap, uint64_t* nsym);
int pgz_inspect_window(pgz_ctx* ctx, int part, uint8_t* host_dst /* 32768 bytes */);

/* Whole-member decompression that allocates nothing (the paper has no
   counterpart; this is a deployment convenience).  For callers that cannot let
   a library allocate device memory -- applications that give all GPU memory
   to their own allocator at start-up, services with a fixed device-memory
   budget, loops that cannot afford cudaFree's device-wide synchronisation --
   it runs the same kernels as pgz_decompress with every scratch buffer inside
   one fixed file-scope __device__ array of about 23 MiB, held on each GPU that
   loads the library until the process exits.  No cudaMalloc, cudaFree or other
   allocating routine is called.
   gz [device, 4-byte aligned, gz_len bytes], out [device, out_cap bytes] on
   the current device; cuda_stream: the cudaStream_t to use (NULL = default).
   Limits: output (ISIZE) <= 4 MiB, gz_len <= 4 MiB + 64 KiB + 4 KiB, gzip
   header <= 4 KiB; larger inputs return PGZ_E_ARG.  The first call on a device
   sets up the array's address there; make it before any stream capture.
   Calls share the array: calls that overlap on the GPU (other streams or
   threads) race and must be serialised by the caller.
   One gzip member per call: data after the member's trailer returns
   PGZ_E_UNSUPPORTED (pgz_decompress accepts several members).  The
   configuration is pgz_config_init's (allowed bytes, confirmation, block
   bounds, 4 warps per pass-1 block, one execution pass at a time), except the
   part size: 32 KiB of compressed data, at most 64 parts; when a part needs
   more symbols than its share of the array, the call is re-planned with half
   as many parts.  Recovery from false block starts is that of
   pgz_decompress.  *out_len: bytes written. */
int pgz_decompress_noalloc(const uint8_t* gz, uint64_t gz_len, uint8_t* out, uint64_t out_cap,
                           uint64_t* out_len, void* cuda_stream);

/* DNA sequences in decoded symbols that may hold undetermined characters
   (Appendix "Heuristic extraction of DNA sequences in DEFLATE block"; with
   pgz_decompress_at this is random access to FASTQ reads, Section
   "Heuristic determination of sequence-resolved blocks"): the maximal
   non-overlapping substrings matching T D+ (U+ D+)* T, with T a newline or an
   undetermined character, D one of A C G T N and U an undetermined character,
   without the delimiting T's and at least min_len long.  A match needs both
   delimiters inside the n symbols.
   sym [device, n u16 symbols as pgz_decompress_at writes them: bit 15 set =
   undetermined]; spans [device, 2 * max_spans u64]: spans[2k] = start,
   spans[2k+1] = length | bit 63 if an undetermined symbol lies inside, in no
   particular order.  *n_spans: spans found (the first max_spans are written);
   *n_undetermined: those holding an undetermined symbol.  The block is
   sequence-resolved (the paper's term) when *n_spans reaches the caller's
   threshold and *n_undetermined is 0.  Stream-ordered; waits for the counts. */
int pgz_extract_sequences(pgz_ctx* ctx, const uint16_t* sym, uint64_t n, uint32_t min_len, uint64_t* spans,
                          uint64_t max_spans, uint64_t* n_spans, uint64_t* n_undetermined);

/* One timed configuration of the autotuner. */
typedef struct pgz_tune_entry {
    uint64_t chunk_bytes;       /* compressed bytes per part */
    int warps_per_block;        /* CTA shape of the pass-1 kernels */
    int exec_pipelined;         /* pass-1 token execution (pgz_config.exec_pipelined) */
    int status;                 /* pgz_status of the calls with this configuration */
    float ms;                   /* median CUDA-event time of one pgz_decompress_batch call */
} pgz_tune_entry;

/* Autotuner.  The number of parts n is a free parameter of the method
   (Section "Full file decompression in two passes": n roughly equal parts);
   this picks the part size and the pass-1 CTA shape for the caller's data.
   For every pair chunk_bytes[a] x warps_per_block[b] -- and, with
   sweep_exec, both forms of pass-1 token execution -- it runs
   pgz_decompress_batch on the n_jobs jobs (device buffers, the batch rules;
   one job is one member) once untimed and reps times timed (CUDA events on the
   context's stream), and then sets the context's chunk_bytes, warps_per_block
   and exec_pipelined (n_chunks = 0) to the configuration with the smallest
   median time among those whose calls returned PGZ_OK for every job.
   entries: n_chunk_bytes * n_wpb * (sweep_exec ? 2 : 1) results, ordered by
   chunk size, then CTA shape, then execution form (NULL: not returned);
   best: the chosen configuration (NULL: not returned).  The jobs' outputs and
   statuses are those of the last call.  Returns PGZ_E_ARG for empty lists,
   chunk sizes below 4 KiB, CTA shapes other than 2, 4 or 8 warps, or reps < 1;
   if no pair succeeded, the first failing status (the context is left
   unchanged). */
int pgz_autotune(pgz_ctx* ctx, pgz_job* jobs, int n_jobs, const uint64_t* chunk_bytes, int n_chunk_bytes,
                 const int* warps_per_block, int n_wpb, int sweep_exec, int reps, pgz_tune_entry* entries,
                 pgz_tune_entry* best);

/* The part size that cuts the jobs' members (gz_len of each; one member per
   job, 10-byte gzip headers assumed) into about waves x R parts, where R is
   the number of pass-1 warps the device holds at once with the given CTA
   shape (*resident_warps, nullable): the pass-1 kernels are persistent grids
   of R warps, one part per warp at a time, so a part count of whole waves
   leaves no warp idle at the end of a launch.  *chunk_bytes: the smallest
   size (>= 4096) whose part count does not exceed the target.  For the
   autotuner's list of sizes; no device work.  PGZ_E_ARG for bad arguments
   (warps_per_block not 2, 4 or 8; waves <= 0). */
int pgz_wave_chunk_bytes(pgz_ctx* ctx, const pgz_job* jobs, int n_jobs, int warps_per_block, double waves,
                         uint64_t* chunk_bytes, int* resident_warps);

/* Sets the context's part size (n_chunks = 0), pass-1 CTA shape and pass-1
   execution form, as pgz_autotune does with its choice: for a configuration
   chosen earlier (a tuning cache) without timing anything.  No device call.
   PGZ_E_ARG for a NULL context, chunk_bytes < 4096, warps_per_block not 2, 4
   or 8, or exec_pipelined not 0 or 1 (the context is then unchanged). */
int pgz_set_tuning(pgz_ctx* ctx, uint64_t chunk_bytes, int warps_per_block, int exec_pipelined);

/* ---------------------------------------------------------------------------
   Serving: a request loop with continuous batching.  Registered members stay
   resident (compressed input; for byte ranges also the index of part starts
   and resolved windows, built by the first range request of a member).  The
   server owns `slots` contexts, each with its own CUDA stream.  A request is a
   whole member or a byte range [offset, offset + length) of its decompressed
   output (Problem 1 with known starts: decoding begins at the indexed block
   start before the range, with the indexed window as context).  pgz_server_poll
   finishes the runs whose work has completed and admits queued requests, in
   arrival order, into free slots: all requests admitted to one slot form one
   run of the pass kernels, and the runs of different slots overlap on the
   GPU.  The queue is spread over the free slots, and one run takes at most
   mem_budget / slots of scratch (but at least one request).  A request is
   admitted while the scratch charged to running requests (compressed size +
   3 x decompressed size each) stays within mem_budget; one that alone exceeds
   it fails with PGZ_E_NOMEM.  One host thread drives a server.  Every result is exactly the
   member's decompressed bytes, whatever else runs beside it.
   --------------------------------------------------------------------------- */
typedef struct pgz_server pgz_server;

typedef struct pgz_request {
    int file;                   /* id from pgz_server_add_file */
    int whole;                  /* 1: the whole member (offset, length ignored); 0: a byte range */
    uint64_t offset, length;    /* range in decompressed bytes */
    uint8_t* out;               /* device: output buffer */
    uint64_t out_cap;
    int status;                 /* result: -1 while queued or running, then a pgz_status */
    uint64_t out_len;           /* result: bytes written */
    double t_submit, t_start, t_done;   /* host steady-clock seconds: submitted, admitted, completed */
} pgz_request;

/* mem_budget: bytes of scratch for running requests (0 = no limit); slots >= 1.
   cfg as for pgz_create (cfg->cuda_stream is ignored: each slot has a stream). */
int pgz_server_create(pgz_server** out, const pgz_config* cfg, int slots, uint64_t mem_budget);
/* Registers a member held by the caller in device memory (4-byte aligned) for
   the server's lifetime; reads its header and trailer.  *file receives the id. */
int pgz_server_add_file(pgz_server* srv, const uint8_t* gz, uint64_t gz_len, int* file);
/* Queues a request; the server keeps the pointer until the request is done.
   PGZ_E_ARG for an unknown member, a range outside the member, or out too small. */
int pgz_server_submit(pgz_server* srv, pgz_request* req);
/* Completes finished runs and admits queued requests; never waits for the GPU.
   *n_done (nullable): requests completed by this call. */
int pgz_server_poll(pgz_server* srv, int* n_done);
/* Polls until every submitted request is done. */
int pgz_server_drain(pgz_server* srv);
/* Requests queued or running. */
int pgz_server_pending(const pgz_server* srv);
void pgz_server_destroy(pgz_server* srv);

/* Number of kernels this library launched on ctx since it was created. */
uint64_t pgz_kernel_launches(const pgz_ctx* ctx);

/* For tests of the host logic (no device work; works without a GPU): one
   step of the recovery the library runs after a pass-1 run of one member,
   on a description of its parts.  The rules are those of Section "Detection
   of DEFLATE block start positions" and Section "Full file decompression in
   two passes": a searched start whose block, or one of the confirm_blocks
   blocks after it, fails the checks is dropped and the search goes on from
   the bit after it (a part that ends exactly on the next part's start
   before its window is complete continues its window with that part's
   checked blocks); a part that does not end exactly on the next part's start
   shows that start to be false: the next part is merged into it when its
   own confirmation passed, decoded past its stop when the run left the
   confirmation open, searched on from the bit after it when it ends a
   streamed segment; a part whose symbols overflowed needs more capacity.
   parts [host array of n, part i of the member in order]: the plan fields
   and the run's results on input; on return the plan fields (lo, disabled,
   confirm_ext) hold the next run's plan.  s0_bit: the member's first DEFLATE
   bit (part 0 with lo <= s0_bit is the member start); mode and last_seg as
   for the member's description (0: a whole member; 3 with last_seg 0: a
   streamed segment that does not reach the member's end).  Returns
   PGZ_RECOVER_STOP (the parts' errors are final), PGZ_RECOVER_RERUN or
   PGZ_RECOVER_GROW (*grow: the part that needs more symbol capacity), or -1
   for bad arguments; *false_syncs is increased by one for every start the
   step drops as false without searching on from it. */
typedef enum pgz_part_status {
    PGZ_PART_FOUND = 1, PGZ_PART_EMPTY = 2, PGZ_PART_DONE = 3, PGZ_PART_ERROR = 4
} pgz_part_status;
typedef enum pgz_part_error {
    PGZ_PART_OK = 0, PGZ_PART_DATA = 1, PGZ_PART_TRUNC = 2, PGZ_PART_DIST = 3, PGZ_PART_OVERFLOW = 4,
    PGZ_PART_CHAIN = 5,    /* did not end exactly on the next part's block start */
    PGZ_PART_CONFIRM = 6,  /* a block of the start's confirmation window failed its checks */
    PGZ_PART_TRAIL = 7     /* data after the member's final block */
} pgz_part_error;
typedef enum pgz_recover_action {
    PGZ_RECOVER_STOP = 0, PGZ_RECOVER_RERUN = 1, PGZ_RECOVER_GROW = 2
} pgz_recover_action;
typedef struct pgz_part_state {
    /* plan */
    uint64_t lo;           /* first bit of the block-start search */
    int32_t given;         /* lo is a known block start (no search) */
    int32_t probe;         /* only the block start is searched (the end of a streamed segment) */
    int32_t disabled;      /* merged into the previous part */
    int32_t confirm_ext;   /* decodes past its stop until its confirmation is settled */
    /* results of the run */
    int32_t state;         /* pgz_part_status */
    int32_t err;           /* pgz_part_error when state is PGZ_PART_ERROR */
    uint64_t sync;         /* block start taken (UINT64_MAX: none) */
    uint64_t end;          /* bit where the part's decoding stopped */
    uint32_t blocks;       /* blocks the part decoded (its own start's block first) */
    uint32_t confirmed;    /* its start's confirmation window passed */
} pgz_part_state;
int pgz_recover_step(int n, pgz_part_state* parts, uint64_t s0_bit, int mode, int last_seg, int confirm_blocks,
                     uint64_t* false_syncs, int* grow);

const char* pgz_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* PGZ_H */
