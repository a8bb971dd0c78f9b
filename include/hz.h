/*
 * hz.h -- C ABI of libhz, a GB300 (sm_103a) implementation of the
 * block-decomposed Huffman coder of Cloud, Curry, Ward, Skjellum and
 * Bangalore, "Accelerating Lossless Data Compression with GPUs"
 * (arXiv 1107.1525).
 *
 * Stream format (Sec. 2.1 and Figs. 3-4 of the paper, plus a container the
 * paper leaves unspecified).  All integers little-endian:
 *   offset 0    "HZB1"
 *   offset 4    u32 flags      bit 0: block-offset index present
 *                              bit 1: sub-block offsets present (needs bit 0)
 *   offset 8    u64 n          uncompressed bytes
 *   offset 16   u32 B          symbols (bytes) per block
 *   offset 20   u32 nb         ceil(n / B)
 *   offset 24   u8  len[256]   Huffman code length of each byte value (0 = absent)
 *   offset 280  u32 word_offset[nb]   only if flags bit 0; record k's position
 *               in 32-bit words from the first byte after the index sections
 *   then, only if flags bit 1: u32 S (a multiple of 32 that divides B), and
 *               for every block k the B/S - 1 words u32 sub_offset[k][j],
 *               j = 1 .. B/S - 1: the payload bit at which the code of the
 *               block's symbol j*S starts (bits_k when the block has fewer
 *               than j*S + 1 symbols).  The same kind of table as the index,
 *               one level down: it lets the S-symbol parts of one block be
 *               decoded independently (an addition to the paper's format,
 *               which Sec. 2.1 leaves at block granularity; the records are
 *               unchanged).
 *   then nb block records back to back.  Record k = u32 bits_k (the payload
 *   length in bits: the "unencoded four byte integer" of Sec. 2.1), then
 *   ceil(bits_k / 32) payload words holding the canonical codes of block k's
 *   symbols in input order, most significant bit first within each word,
 *   zero-padded to the word boundary (32-63 bits of overhead per block).
 * Code values are canonical (in (length, byte) order; the first code is 0 and
 * each next one is (previous + 1) << (growth in length)); lengths are Huffman
 * leaf depths with ties broken by (weight, id), leaf id = byte value and the
 * t-th merged node id = 256 + t.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers (global memory of the context's
 *     device) owned by the caller; they must stay valid until the work queued
 *     on `stream` has finished.  Pointers named h_* are host pointers.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that take a stream only enqueue work on it and return at once, unless
 *     stated otherwise.
 *   - Argument errors are returned immediately (HZ_ERR_ARG) and enqueue
 *     nothing.  Errors found on the device (a corrupt stream, an output buffer
 *     that is too small, a bounded wait that ran out) are recorded in the
 *     context's device status word and returned by the next hz_sync() on that
 *     context; kernels never trap.
 *   - A context is not thread-safe, and its scratch memory is reused by every
 *     call: calls on one context must be issued from one host thread and run
 *     in stream order (one stream, or streams ordered by events).
 *   - Limits: n < 2^32, 1 <= B <= 2^24, code lengths <= 64.
 */
#ifndef HZ_H
#define HZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hz_status;
#define HZ_OK 0
#define HZ_PENDING 1
#define HZ_ERR_ARG (-1)
#define HZ_ERR_CAPACITY (-2)
#define HZ_ERR_CORRUPT (-3)
#define HZ_ERR_NOMEM (-4)
#define HZ_ERR_BUSY (-5)
#define HZ_ERR_TIMEOUT (-6)
#define HZ_ERR_CUDA (-7)

#define HZ_HEADER_BYTES 280u
#define HZ_MAX_BLOCK (1u << 24)
#define HZ_MAX_CODE_LEN 64

typedef struct hz_ctx hz_ctx;

/* Code table in host memory: len[s] is the code length of byte value s
 * (0 = not coded), code[s] its canonical code value in the low len[s] bits. */
typedef struct {
  uint8_t len[256];
  uint64_t code[256];
} hz_codes;

/*
 * Create a context on CUDA device `device`.  The context owns its device
 * scratch (status word, histogram, code table, scan state, decode tables),
 * grown on demand.  mem_budget_bytes bounds the device memory that
 * hz_submit() may have admitted at once (0 = no limit).
 * Returns HZ_ERR_ARG for a bad device, HZ_ERR_NOMEM / HZ_ERR_CUDA on failure.
 */
hz_status hz_create(hz_ctx** ctx, int device, uint64_t mem_budget_bytes);

/* Wait for the context's work and free everything it owns.  NULL is a no-op. */
void hz_destroy(hz_ctx* ctx);

/*
 * Worst-case stream size in bytes for n input bytes in blocks of block_size
 * symbols, when the code is built from the same data (Sec. 2: a Huffman code
 * never averages more than 8 bits per byte, and Sec. 2.1: each block adds
 * 32-63 bits): 280 + 4*nb (index) + 8*nb + 4*ceil(n/4) + 4*nb.
 * block_size 0 means the context's automatic choice is not known yet; the
 * bound then assumes 1-byte blocks.  Returns 0 for n >= 2^32.
 */
uint64_t hz_compress_bound(uint64_t n, uint32_t block_size);

/*
 * The same bound for the streams hz_compress writes on `ctx` with its current
 * options: block_size 0 resolves to the context's choice, and with
 * HZ_OPT_SUB_BLOCK = S (when S divides the block size) the bound includes the
 * 4 + 4 * nb * (B/S - 1) bytes of sub-block offsets.  0 for a NULL ctx or
 * n >= 2^32.
 */
uint64_t hz_compress_bound_ctx(hz_ctx* ctx, uint64_t n, uint32_t block_size);

/*
 * Sec. 2 ("counting the appearance of every distinct symbol", then the
 * Huffman code of Fig. 2): histogram d_in[0..n) on the GPU and build its code.
 * Writes the lengths and canonical codes to *codes_out (host memory).
 * Synchronous: returns after the table has reached the host.
 */
hz_status hz_build_codes(hz_ctx* ctx, const uint8_t* d_in, uint64_t n, hz_codes* codes_out,
                         void* stream);

/*
 * Sec. 2.1: compress d_in[0..n) into the stream format above, in blocks of
 * block_size symbols (0 = the context's autotuned choice for this size).
 * codes == NULL builds the code from d_in's histogram (Sec. 2); otherwise
 * codes->len is used (it must satisfy Kraft's inequality and give every byte
 * present in d_in a nonzero length; codes->code must be the canonical values
 * for those lengths, else HZ_ERR_ARG).  d_out receives the stream (capacity
 * out_cap bytes); *d_out_len (a device u64) receives its size, or the size
 * that would be needed when out_cap is too small (then hz_sync() reports
 * HZ_ERR_CAPACITY and d_out holds no valid stream).
 * Asynchronous on `stream`; device errors surface through hz_sync().
 */
hz_status hz_compress(hz_ctx* ctx, const uint8_t* d_in, uint64_t n, uint32_t block_size,
                      const hz_codes* codes, uint8_t* d_out, uint64_t out_cap,
                      uint64_t* d_out_len, void* stream);

/*
 * Sec. 2.1, last paragraph: decode a stream d_in[0..in_len) whose blocks are
 * located through the offset table (read from the index when flags bit 0 is
 * set, rebuilt from the length delimiters otherwise) and decoded
 * independently.  The stream must end exactly at its last record.  d_out
 * receives n bytes (capacity out_cap); *d_out_len (device u64) receives n.
 * A stream that fails any check (magic, header fields, Kraft inequality,
 * index vs. delimiters, a code that does not decode, a block that does not
 * use exactly bits_k bits, nonzero padding) is reported as HZ_ERR_CORRUPT by
 * hz_sync(); out_cap < n as HZ_ERR_CAPACITY.  The host reads nothing of the
 * stream: the header is parsed on the device, so the call never blocks.
 * Asynchronous on `stream`.
 */
hz_status hz_decompress(hz_ctx* ctx, const uint8_t* d_in, uint64_t in_len, uint8_t* d_out,
                        uint64_t out_cap, uint64_t* d_out_len, void* stream);

/*
 * Wait for `stream`, then return and clear the context's device status:
 * HZ_OK, or the first error a kernel recorded since the last hz_sync().
 */
hz_status hz_sync(hz_ctx* ctx, void* stream);

/*
 * Host-buffer round trips (the end-to-end path of Sec. 4, "sans memory
 * transfer" vs. total throughput): copy h_in to the device, run
 * hz_compress / hz_decompress there on `stream`, copy the result back to
 * h_out and synchronise.  *out_len receives the result size (or the size
 * needed, with HZ_ERR_CAPACITY).  h_in / h_out should be pinned
 * (cudaHostAlloc / cudaHostRegister) for full copy bandwidth.
 */
hz_status hz_compress_host(hz_ctx* ctx, const uint8_t* h_in, uint64_t n, uint32_t block_size,
                           uint8_t* h_out, uint64_t out_cap, uint64_t* out_len, void* stream);
hz_status hz_decompress_host(hz_ctx* ctx, const uint8_t* h_in, uint64_t in_len, uint8_t* h_out,
                             uint64_t out_cap, uint64_t* out_len, void* stream);

/*
 * hz_compress_noalloc: hz_compress (code built from d_in, block-offset index
 * written) for callers that must not allocate device memory -- for example
 * code that runs under a framework's caching allocator or a fixed memory
 * reservation that a cudaMalloc would bypass, or a latency-critical path that
 * cannot afford cudaMalloc's implicit synchronisation.  The paper has no
 * counterpart; it is an interface addition.
 *
 * It takes no context and allocates nothing: its scratch is one file-scope
 * device array of about 1 MiB, which every GPU that loads the library holds
 * until the process exits.  That array bounds the input: n <= 2^28 bytes
 * (256 MiB); larger n returns HZ_ERR_ARG at once.  The caller passes inputs
 * and outputs as for hz_compress, plus d_status, a device int32 that receives
 * the call's device-side status (0 or a negative hz_status, e.g.
 * HZ_ERR_CAPACITY with *d_out_len = the size needed) once the work has run.
 * The first call on a device looks up the array's device address and clears
 * it, synchronously, with that device current; make that first call before
 * any stream capture.  Every call shares the one array and clears what must
 * start at zero, so calls that overlap on the GPU (different streams or host
 * threads without ordering) race; order them.  Asynchronous on `stream`
 * otherwise.  HZ_ERR_CUDA if a launch or the set-up fails.  block_size 0
 * takes the built-in size table (<= 64 KiB: 4 KiB, <= 32 MiB: 16 KiB, larger:
 * 64 KiB), never a context's autotuned choice, so for the same input it can
 * pick another block size than hz_compress with block_size 0.
 */
hz_status hz_compress_noalloc(const uint8_t* d_in, uint64_t n, uint32_t block_size,
                              uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len,
                              int32_t* d_status, void* stream);

/* ------------------------------------------------------------- options */
#define HZ_OPT_INDEX 1        /* 1 (default): write the block-offset index */
#define HZ_OPT_PROFILE 2      /* 1: time every kernel launch with CUDA events */
#define HZ_OPT_DECODE_LUT_BITS 3  /* decode table width W, 8..12 (default 12) */
#define HZ_OPT_DECODE_THREADS 4   /* threads per decode CTA (one warp decodes a block of
                                     up to 64 KiB; a CTA decodes a larger block):
                                     128 or 256 (default 256) */
#define HZ_OPT_AUTOTUNE 5     /* 1 (default): block_size 0 picks the tuned size */
#define HZ_OPT_BATCH_PLAIN 6  /* 1: hz_submit runs each request through hz_compress /
                                 hz_decompress in turn (the one-launch-per-buffer baseline) */
#define HZ_OPT_BATCH_MAX_REQS 7  /* most requests in one device batch when queued
                                    submissions merge (default 4096; a larger
                                    single submission still goes alone) */
#define HZ_OPT_SUB_BLOCK 8    /* S > 0: hz_compress (and hz_compress_host) write the
                                 sub-block offsets of every S symbols (flags bit 1)
                                 when S divides the block size and the index is on;
                                 S a multiple of 32.  0 (default): the paper's layout
                                 with the block index only.  HZ_SUB_BLOCK_AUTO: S is
                                 picked per call from n, the block size and the
                                 device: the largest of 4096 .. 512 that divides the
                                 block size and gives at least four sub-blocks per
                                 decoder lane the device keeps resident (SMs x 768),
                                 else 512 if that gives at least one per lane, else
                                 none (the paper's layout).  Decoders accept any
                                 layout. */
#define HZ_SUB_BLOCK_AUTO 1
#define HZ_OPT_SPIN_LIMIT 9   /* polls the encoder's look-back scan makes while waiting
                                 for a predecessor before it records HZ_ERR_TIMEOUT and
                                 returns (1 .. 2^24, default 2^20; each poll sleeps
                                 about 64 ns) */
#define HZ_OPT_TUNE_BATCHED 11  /* 1: hz_autotune times its block-size candidates on
                                   batches of slices through hz_submit (the choice for
                                   batched and served requests) instead of one call
                                   per slice (default 0) */
#define HZ_OPT_INJECT_SCAN_STALL 10  /* host-side fault injection for tests: 1 = the
                                 next hz_compress hands its scan CTAs tickets from 1
                                 instead of 0, so the first one waits for a
                                 predecessor that never publishes and its bounded wait
                                 runs out; hz_sync then returns HZ_ERR_TIMEOUT.  One
                                 shot: cleared when used.  Nothing on the device is
                                 changed; the context stays usable. */

/* Set an option; HZ_ERR_ARG for an unknown key or value. */
hz_status hz_set_option(hz_ctx* ctx, int key, int64_t value);
int64_t hz_get_option(hz_ctx* ctx, int key);

/*
 * Autotuner: choose, per input-size class (<= 64 KiB, <= 1 MiB, <= 16 MiB,
 * larger), the block size used when hz_compress / hz_submit get
 * block_size 0, then the decode table width W and the threads per decode
 * CTA, by timing compress + decompress round trips of slices of
 * d_sample[0..n) (device memory, the caller's representative data) for B in
 * {4, 8, 16, 32, 64} KiB -- one call per slice, or with HZ_OPT_TUNE_BATCHED
 * batches of up to 64 slices through hz_submit -- and decompressions of the
 * largest slice for W in {10, 11, 12} and 128 or 256 threads.  A candidate
 * replaces the default (the built-in block size, W = 12, 256 threads) only
 * when it is more than 3 % faster.  Candidates whose format overhead
 * (Sec. 2.1: 32-63 bits per block) exceeds 1 % of the stream are skipped.  The choice is kept in the
 * context and, when the environment variable HZ_TUNE_CACHE names a file,
 * written there as JSON; hz_create loads that file when it exists.
 * Synchronous; allocates scratch for the trial streams.
 */
hz_status hz_autotune(hz_ctx* ctx, const uint8_t* d_sample, uint64_t n, void* stream);

/* The tuned block size for n input bytes (the default when nothing is tuned). */
uint32_t hz_tuned_block_size(hz_ctx* ctx, uint64_t n);

/* ------------------------------------------------------ instrumentation */
/* Number of kernels this context has launched since creation. */
uint64_t hz_launch_count(hz_ctx* ctx);

/*
 * With HZ_OPT_PROFILE on, every kernel launch is bracketed by CUDA events on
 * its stream.  hz_profile_read() waits for them, writes up to `max` records
 * (kernel name id, milliseconds) and clears the log; it returns the number of
 * records written.  hz_kernel_name() maps an id to a static string.
 */
int hz_profile_read(hz_ctx* ctx, int32_t* ids, float* ms, int max);
const char* hz_kernel_name(int32_t id);

/* ------------------------------------------- batching and serving (a10, a11) */
/*
 * One request of a batch: op 0 = compress d_src[0..src_len) in blocks of
 * block_size (0 = tuned) with a code built from that buffer, op 1 =
 * decompress the stream d_src[0..src_len).  d_dst (capacity dst_cap) receives
 * the result.
 */
typedef struct {
  int32_t op;
  uint32_t block_size;
  const uint8_t* d_src;
  uint64_t src_len;
  uint8_t* d_dst;
  uint64_t dst_cap;
} hz_request;

#define HZ_OP_COMPRESS 0
#define HZ_OP_DECOMPRESS 1

/*
 * Queue `count` requests as one submission and return at once with a ticket.
 * Submissions are admitted in order against the context's device-memory
 * budget (each request's src_len + dst_cap, plus per-request scratch).  The
 * context runs up to three device batches at once, each on its own stream as
 * one CUDA graph with one persistent kernel per phase over all its requests;
 * when a batch slot frees up, it takes every queued submission that fits the
 * budget and HZ_OPT_BATCH_MAX_REQS (continuous batching).  HZ_ERR_BUSY if the
 * submission alone exceeds the budget; HZ_ERR_ARG for a malformed request
 * (unknown op, NULL pointer, src_len >= 2^32, block_size > 2^24, d_dst not
 * 4-byte aligned, or a decompress d_src not 4-byte aligned).  The batch that
 * carries the submission runs on the context's own streams, after the work
 * enqueued on `stream` (NULL = the legacy default stream) before this call:
 * the caller may write the sources there and submit without waiting.  The
 * caller keeps every buffer alive and untouched until the ticket completes.
 * HZ_ERR_CUDA if the ordering event cannot be recorded on `stream`.
 */
hz_status hz_submit(hz_ctx* ctx, const hz_request* reqs, uint32_t count, uint64_t* ticket_out,
                    void* stream);

/*
 * Wait up to timeout_ns (0 = just look, < 0 = forever) for batch `ticket`.
 * HZ_PENDING if it has not finished; otherwise HZ_OK and, per request,
 * per_req[i] (its status) and out_lens[i] (result bytes), both host arrays
 * of the batch's length (either may be NULL).  A ticket can be polled to
 * completion once.
 */
hz_status hz_poll(hz_ctx* ctx, uint64_t ticket, int64_t timeout_ns, hz_status* per_req,
                  uint64_t* out_lens);

/*
 * Request replay (the serving loop): an open-loop client over the batcher.
 * Item i is submitted alone at items[i].arrival_s seconds after the call
 * starts (items sorted by arrival_s); the batcher merges whatever is queued
 * when a slot frees up (see hz_submit).  An item whose req.d_dst is NULL
 * takes req.dst_cap bytes of the device ring d_ring[0..ring_bytes) (256-byte
 * aligned, owned by the caller) from submission to completion, and waits for
 * room when the ring is full.  The call first waits for all work on the
 * device (so the sources are ready whichever stream wrote them), then starts
 * its clock.  Blocks until every item has completed; then
 * records[i] (host array of `count`) holds its times (seconds from the
 * start: handed to the batcher, completion seen on the host), status, result
 * length, the device batch that carried it and its ring offset (~0 for items
 * with their own d_dst; ring results are overwritten by later items).
 * *wall_s (may be NULL) = start to the last completion.  HZ_ERR_ARG for
 * unsorted items, a NULL d_dst without a usable ring, or a dst_cap larger
 * than the ring.  Per-item errors go to records[i].status.
 */
typedef struct {
  double arrival_s;
  hz_request req;
} hz_serve_item;

typedef struct {
  double submit_s;
  double done_s;
  uint64_t out_len;
  uint64_t launch;
  uint64_t dst_offset;
  int32_t status;
  uint32_t pad;
} hz_serve_record;

hz_status hz_serve_replay(hz_ctx* ctx, const hz_serve_item* items, uint64_t count,
                          uint8_t* d_ring, uint64_t ring_bytes, hz_serve_record* records,
                          double* wall_s);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
