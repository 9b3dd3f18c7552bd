/*
 * libvbyte -- GPU decoding of VByte-compressed uint32 streams on GB300
 * (sm_103a).
 *
 * The operation follows Plaisance, Kurz, Lemire, "Vectorized VByte Decoding"
 * (arXiv 1503.07387):
 *   - format (Sec. 1, Table 1): each integer is written seven bits at a time,
 *     least significant group first; the high bit of every byte is 1 except
 *     on the integer's last byte.  Integers in [0,2^7) take one byte,
 *     [2^7,2^14) two, ... up to five bytes for uint32;
 *   - decoding (Sec. 2, Algorithm 1): the result is exactly what the
 *     conventional byte-at-a-time decoder appends, with uint32 arithmetic
 *     (a fifth byte contributes b * 2^28 modulo 2^32);
 *   - differential coding (Sec. 1 "Differential coding", Sec. 2 and Sec. 4
 *     "Differential Coding"): the stream holds gaps x_i - x_{i-1} with
 *     x_0 = prev, and decoding returns the prefix sums x_i modulo 2^32.
 *
 * Conventions for every entry point below:
 *   - "d_" pointers are device memory owned by the caller; "h_" pointers are
 *     host memory owned by the caller (page-locked memory gives the fastest
 *     copies).  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device work is queued on it and the call returns without
 *     synchronising, except where an entry point says otherwise.
 *   - The library keeps one small workspace per (device, stream): a status
 *     word, tile and chunk counters, and the per-tile descriptors through
 *     which the CTAs pass counts and running sums to one another (16 bytes
 *     per 4 KiB of input).  It grows on demand with
 *     cudaMallocAsync on that stream; a call made while the stream is being
 *     captured into a CUDA graph never allocates and returns VBYTE_ENOMEM if
 *     the workspace is too small (run the same call once before capture).
 *   - A stream is driven by one host thread at a time: a call that grows a
 *     stream's workspace frees the old one in stream order, so two threads
 *     queueing work on the same stream at once can race on it.  Calls on
 *     different streams may come from any threads.
 *   - Return codes are synchronous argument/launch checks (VBYTE_OK ...).
 *     Errors that depend on the data are recorded asynchronously in the
 *     per-stream status word (VBYTE_ERR_* bits) and read with
 *     vbyte_get_status(); the decode path never synchronises to look.
 *   - Output writes are always clamped to [0, n).  When a data error is
 *     recorded, output slots the stream does not define are unspecified.
 */
#ifndef VBYTE_H
#define VBYTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- synchronous return codes ------------------------------------------ */
#define VBYTE_OK 0
#define VBYTE_EINVAL 1 /* null pointer with a nonzero size, misaligned output */
#define VBYTE_ECUDA 2  /* a CUDA runtime call or kernel launch failed */
#define VBYTE_ENOMEM 3 /* workspace could not be grown */
#define VBYTE_ETOOBIG 4 /* input above VBYTE_NOALLOC_MAX_BYTES (vbyte_decode_noalloc) */

/* ---- data-error bits of the per-stream status word --------------------- */
/* A run of five or more consecutive bytes with the high bit set: Algorithm 1
 * would consume a fifth byte whose high bit it never tests (Sec. 2). */
#define VBYTE_ERR_MALFORMED_LONG 1u
/* The last byte of a stream (or list) has the high bit set: the input ends
 * inside an integer. */
#define VBYTE_ERR_TRUNCATED 2u
/* The number of terminator bytes (high bit clear) differs from the expected
 * count n (or from val_off[j+1]-val_off[j] for list j). */
#define VBYTE_ERR_COUNT_MISMATCH 4u
/* A wait on another tile's count or running sum gave up after its time
 * limit (about two seconds); the outputs of that call are unspecified. */
#define VBYTE_ERR_TIMEOUT 8u
/* Batched calls: the offset arrays break their contract (not non-decreasing,
 * or not running from 0 to nbytes and from 0 to n). */
#define VBYTE_ERR_BAD_OFFSETS 16u

/* ---- host-side encoding (input generation) ----------------------------- */

/* Upper bound on the encoded size of n uint32 values: 5*n bytes (Sec. 1). */
size_t vbyte_max_encoded_size(size_t n);

/* Encode n values (Sec. 1, Table 1) into h_out, which must hold
 * vbyte_max_encoded_size(n) bytes.  Returns the number of bytes written.
 * Host memory only; no CUDA call. */
size_t vbyte_encode(const uint32_t *h_in, size_t n, uint8_t *h_out);

/* Differential coding (Sec. 1): encode the gaps h_in[i] - h_in[i-1] modulo
 * 2^32 with h_in[-1] = prev.  Returns the number of bytes written. */
size_t vbyte_encode_delta(const uint32_t *h_in, size_t n, uint32_t prev,
                          uint8_t *h_out);

/* The differential variant Sec. 1 names for lists without repeated values:
 * encode h_in[0] - prev, then h_in[i] - h_in[i-1] - 1 (modulo 2^32).
 * Returns the number of bytes written. */
size_t vbyte_encode_delta_m1(const uint32_t *h_in, size_t n, uint32_t prev,
                             uint8_t *h_out);

/* Blocked differences (Sec. 1): encode h_in[i] - h_in[i-4] modulo 2^32 with
 * h_in[-4..-1] = h_prev4[0..3] (NULL for zeros: the paper's x_1, x_2, x_3,
 * x_4, x_5 - x_1, ...).  Returns the number of bytes written. */
size_t vbyte_encode_delta4(const uint32_t *h_in, size_t n, const uint32_t *h_prev4,
                           uint8_t *h_out);

/* Encode num_lists lists laid end to end: list j is
 * h_in[h_val_off[j] .. h_val_off[j+1]).  With delta != 0 each list is
 * differentially coded on its own, starting from h_prev[j] (0 when h_prev is
 * NULL).  Writes h_byte_off[0..num_lists] (h_byte_off[0] = 0) and returns the
 * total number of bytes.  h_out must hold vbyte_max_encoded_size(total). */
size_t vbyte_encode_batched(const uint32_t *h_in, const uint64_t *h_val_off,
                            size_t num_lists, int delta, const uint32_t *h_prev,
                            uint8_t *h_out, uint64_t *h_byte_off);

/* ---- GPU encoding -------------------------------------------------------- */

/* Encode the n uint32 at d_in (4-byte aligned) into d_out, exactly as
 * vbyte_encode would (Sec. 1, Table 1: 7-bit groups, least significant
 * first, the high bit set on every byte but the last; the shortest form).
 * d_out must hold vbyte_max_encoded_size(n) bytes.  The number of bytes
 * written goes to *d_nbytes (device memory) when the stream reaches it; no
 * host synchronisation.  All pointers are caller-owned device memory; the
 * call uses the stream's workspace and allocates only when it grows.
 * Returns VBYTE_OK; VBYTE_EINVAL for a null pointer with n > 0, a null
 * d_nbytes or a misaligned d_in; VBYTE_ENOMEM / VBYTE_ECUDA for allocation
 * or launch failures.  Every value is encodable, so the only data-dependent
 * status bit is VBYTE_ERR_TIMEOUT (vbyte_get_status). */
int vbyte_encode_device(const uint32_t *d_in, size_t n, uint8_t *d_out,
                        uint64_t *d_nbytes, void *stream);

/* Differential coding (Sec. 1) on the device: encode the gaps
 * d_in[i] - d_in[i-1] modulo 2^32 with d_in[-1] = prev, as
 * vbyte_encode_delta would.  Arguments and errors as vbyte_encode_device. */
int vbyte_encode_delta_device(const uint32_t *d_in, size_t n, uint32_t prev,
                              uint8_t *d_out, uint64_t *d_nbytes,
                              void *stream);

/* The gaps-minus-one variant (vbyte_encode_delta_m1) on the device.
 * Arguments and errors as vbyte_encode_device. */
int vbyte_encode_delta_m1_device(const uint32_t *d_in, size_t n, uint32_t prev,
                                 uint8_t *d_out, uint64_t *d_nbytes,
                                 void *stream);

/* ---- single-stream GPU decoding ----------------------------------------- */

/* Decode the nbytes-byte stream at d_in (any alignment) into the n uint32 at
 * d_out (4-byte aligned), exactly as Algorithm 1 (Sec. 2) would.  n is the
 * number of values the caller expects (e.g. the posting-list length); a
 * different terminator count sets VBYTE_ERR_COUNT_MISMATCH.  n = 0 with
 * nbytes = 0 is a no-op.  Returns VBYTE_EINVAL for a null pointer with a
 * nonzero size or a d_out that is not 4-byte aligned.  The library picks the
 * kernel from the input size and mean code length (nbytes / n): a single
 * launch with a decoupled look-back under 16 MiB, count then decode in one
 * launch for one-byte codes, else separate count, scan and decode launches;
 * all give the same values and status bits (vbyte_debug_force_passes). */
int vbyte_decode(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n,
                 void *stream);

/* As vbyte_decode, then undo differential coding: d_out[i] = prev + g_0 +
 * ... + g_i modulo 2^32 where g_i are the decoded gaps (Sec. 1, Sec. 2,
 * Sec. 4 "Differential Coding").  Passing the last value of one piece as prev
 * for the next decodes a stream piece by piece. */
int vbyte_decode_delta(const uint8_t *d_in, size_t nbytes, uint32_t *d_out,
                       size_t n, uint32_t prev, void *stream);

/* The gaps-minus-one variant (Sec. 1, "Differential coding": for lists
 * without repeated values the stored gaps are x_1 - x_0, x_2 - x_1 - 1, ...):
 * d_out[i] = prev + g_0 + ... + g_i + i modulo 2^32.  Arguments and errors as
 * vbyte_decode_delta; the bytes are those vbyte_encode_delta_m1 writes.  For
 * a piece after the first, pass as prev the last value before it plus one. */
int vbyte_decode_delta_m1(const uint8_t *d_in, size_t nbytes, uint32_t *d_out,
                          size_t n, uint32_t prev, void *stream);

/* Blocked differences (Sec. 1, "Differential coding": storing x_1, x_2, x_3,
 * x_4, x_5 - x_1, x_6 - x_2, ... so that four running sums proceed side by
 * side): d_out[i] = g_i + d_out[i-4] modulo 2^32 over the decoded integers
 * g, with d_out[-4..-1] = h_prev4[0..3] (four values in HOST memory, read
 * during the call; NULL for zeros, which gives the paper's list).  Each of
 * the four classes of ranks modulo 4 is its own running sum.  Arguments and
 * errors as vbyte_decode; the bytes are those vbyte_encode_delta4 writes.
 * For a piece after the first, pass the last four values before it (the one
 * at rank i - 4 ... i - 1 for the piece's rank i) as h_prev4, ordered by
 * rank modulo 4 relative to the piece: h_prev4[k] is the value four ranks
 * before the piece's k-th value. */
int vbyte_decode_delta4(const uint8_t *d_in, size_t nbytes, uint32_t *d_out,
                        size_t n, const uint32_t *h_prev4, void *stream);

/* ---- batched GPU decoding ------------------------------------------------ */

/* Decode num_lists lists laid end to end in one launch (Sec. 5 decodes
 * posting lists one after another; here they are decoded together).  List j
 * is the bytes d_in[d_byte_off[j] .. d_byte_off[j+1]) and decodes to
 * d_out[d_val_off[j] .. d_val_off[j+1]).  The offset arrays hold
 * num_lists + 1 uint64 each, in device memory (8-byte aligned), and must be
 * non-decreasing with d_byte_off[0] = 0, d_byte_off[num_lists] = nbytes,
 * d_val_off[0] = 0, d_val_off[num_lists] = n (nbytes and n are passed from
 * the host so the call needs no device-to-host read); a violation sets
 * VBYTE_ERR_BAD_OFFSETS.  Each list must hold exactly its value count
 * (VBYTE_ERR_COUNT_MISMATCH otherwise) and end on a terminator byte
 * (VBYTE_ERR_TRUNCATED otherwise).  Empty lists are allowed.  Since a
 * well-formed list ends on a terminator, the values equal those of
 * vbyte_decode on the concatenation.  num_lists = 0 requires nbytes = n = 0.
 * Returns VBYTE_EINVAL for null or misaligned pointers. */
int vbyte_decode_batched(const uint8_t *d_in, size_t nbytes,
                         const uint64_t *d_byte_off, uint32_t *d_out, size_t n,
                         const uint64_t *d_val_off, size_t num_lists,
                         void *stream);

/* As vbyte_decode_batched, each list differentially coded on its own (Sec. 1
 * "Differential coding"): d_out[d_val_off[j] + i] = d_prev[j] + g_0 + ... +
 * g_i modulo 2^32 over list j's gaps g.  d_prev (num_lists uint32, device)
 * may be NULL for x_0 = 0 in every list. */
int vbyte_decode_delta_batched(const uint8_t *d_in, size_t nbytes,
                               const uint64_t *d_byte_off, uint32_t *d_out,
                               size_t n, const uint64_t *d_val_off,
                               size_t num_lists, const uint32_t *d_prev,
                               void *stream);

/* ---- batched plans: tuned once, replayed from a CUDA graph -------------- */

/* An opaque, reusable batched decode of one fixed batch (the arguments of
 * vbyte_decode_batched / vbyte_decode_delta_batched; d_prev is ignored when
 * delta = 0).  Creation synchronises `stream` (the inputs must be ready),
 * copies the offsets to the host, allocates the plan's own device memory
 * (cudaMalloc), chooses how to decode, and captures the launch sequence into
 * a CUDA graph.  The lists are grouped in length classes (class k: lists of
 * 2^k .. 2^(k+1) - 1 bytes, as Sec. 5 groups posting lists by length).  Two
 * kernels are candidates:
 *   - list items: one warp decodes one item -- a whole list of at most C
 *     bytes in a single pass, or a C-byte chunk of a longer list after a
 *     count launch over the chunks and a scan of each list's chunk counts and
 *     sums (count then decode) -- so the chunk size C decides, per length
 *     class, between the single pass and count-then-decode; the decode
 *     launch runs 128 or 256 threads per block;
 *   - the segmented stream kernel of vbyte_decode_batched (the lists laid end
 *     to end decoded as one stream), with CTAs per SM and how far counting
 *     runs ahead of decoding.
 * With autotune != 0 every candidate (C in 8, 16, 32, 64 KiB x 128 or 256
 * threads per block; with 256 threads also the table-driven steps of Sec. 4
 * in place of per-terminator assembly; and the segmented kernel) is timed on
 * this batch, or the
 * choice made earlier for the same batch class (device, delta, log2 of mean
 * bytes per list, log2 of total bytes) is reused; otherwise list items with
 * C = 32 KiB and 256 threads per block (the segmented kernel if the offsets
 * break their contract).  Creation overwrites d_out (with the decoded
 * values) while tuning.  A plan may be launched any
 * number of times; launches of one plan must not overlap on the GPU (they
 * share its workspace).  Data errors go to the plan's own status word.
 * Returns VBYTE_EINVAL as vbyte_decode_batched does (and for num_lists = 0),
 * VBYTE_ENOMEM if the workspace cannot be allocated. */
typedef struct vbyte_plan vbyte_plan;
int vbyte_plan_create(vbyte_plan **plan, const uint8_t *d_in, size_t nbytes,
                      const uint64_t *d_byte_off, uint32_t *d_out, size_t n,
                      const uint64_t *d_val_off, size_t num_lists,
                      const uint32_t *d_prev, int delta, int autotune,
                      void *stream);
/* Queue the plan's graph on `stream` (cudaGraphLaunch); does not wait. */
int vbyte_plan_launch(vbyte_plan *plan, void *stream);
/* Synchronise `stream`, return and clear the plan's VBYTE_ERR_* bits. */
int vbyte_plan_get_status(vbyte_plan *plan, void *stream, uint32_t *status_out);
/* The chosen launch parameters (ctas_per_sm 0 = occupancy limit), the tuned
 * time in ms, and tuned = 0 (defaults), 1 (timed now), 2 (from the cache). */
int vbyte_plan_describe(const vbyte_plan *plan, int *ctas_per_sm,
                        uint64_t *lead_slack, float *tuned_ms, int *tuned);
/* The chosen kernel: 0 = the segmented stream kernel, 1 = list items, 2 =
 * list items decoded by the table-driven steps of Sec. 4 (vbyte_table); for
 * list items the chunk size C in bytes and the decode launch's threads per
 * block (0 and 256 for the segmented kernel). */
int vbyte_plan_choice(const vbyte_plan *plan, int *kernel, uint64_t *chunk_bytes,
                      int *threads_per_block);
/* Length class k (0..63; lists of 2^k .. 2^(k+1) - 1 bytes, class 0 also the
 * empty lists): its lists, its values, and how the plan decodes them:
 * 0 = no lists, 1 = single pass (each list one item), 2 = count then decode
 * (lists cut into chunks), 3 = the segmented stream kernel.  VBYTE_EINVAL for
 * k outside 0..63. */
int vbyte_plan_class(const vbyte_plan *plan, int k, uint64_t *lists,
                     uint64_t *values, int *mode);
/* Free the plan's graph and workspace (synchronises the device). */
void vbyte_plan_destroy(vbyte_plan *plan);

/* The form batched decoding replaces, kept for comparison: one
 * vbyte_decode / vbyte_decode_delta call per list, queued back to back on
 * `stream` with no synchronisation in between.  The offsets (and h_prev,
 * nullable) are in HOST memory here.  Data errors go to the stream's status
 * word. */
int vbyte_decode_each(const uint8_t *d_in, const uint64_t *h_byte_off,
                      uint32_t *d_out, const uint64_t *h_val_off,
                      size_t num_lists, int delta, const uint32_t *h_prev,
                      void *stream);

/* ---- serving: a resident pool and a continuous-batching request loop ---- */

/* A server keeps a pool of compressed lists (laid end to end in d_pool, list
 * j = bytes [h_byte_off[j], h_byte_off[j+1]) holding h_val_off[j+1] -
 * h_val_off[j] values; offsets in host memory, copied) resident on the
 * current device and decodes queries, each naming up to max_batch_lists of
 * its lists, as they arrive.  A scheduler thread admits waiting queries in
 * arrival order into a batch as long as the batch's decoded output fits in
 * the free part of a device arena (arena_bytes), its compressed lists take
 * at most staging_bytes and the batch limits hold; up to max_inflight
 * batches run at once, each on its own stream, so queries that arrive while
 * others are on the GPU start as soon as a slot and arena space free up.
 * While batches are in flight the scheduler thread polls their completion
 * (yielding between polls, so it keeps one host core busy); with nothing in
 * flight it sleeps until a query arrives or arena space is released.
 * per_list = 0: a batch is decoded in place with one set of launches -- its
 * lists become work items (a whole list, or a 32 KiB chunk of a long one)
 * that warps decode straight from the pool into the arena; per_list = 1 (a
 * comparison form): each list with its own vbyte_decode / vbyte_decode_delta
 * call; per_list = 2 (another): the lists gathered end to end into a staging
 * buffer of staging_bytes, then one segmented batched launch.  A query's values (the concatenation of its lists'
 * values, in the order named) stay in the arena until it is released.  All
 * device memory is allocated at creation.  The pool and its offsets must
 * not change while the server lives. */
typedef struct vbyte_server vbyte_server;
typedef struct vbyte_server_config {
    size_t arena_bytes;      /* device memory for decoded outputs */
    size_t staging_bytes;    /* per in-flight batch: gathered compressed bytes */
    int max_inflight;        /* batches on the GPU at once */
    int max_batch_queries;   /* queries per batch */
    int max_batch_lists;     /* lists per batch (and per query) */
    int per_list;            /* 0 in place, 1 one call per list, 2 gather then batched */
} vbyte_server_config;
int vbyte_server_create(vbyte_server **srv, const uint8_t *d_pool,
                        size_t pool_bytes, const uint64_t *h_byte_off,
                        const uint64_t *h_val_off, size_t num_lists, int delta,
                        const uint32_t *h_prev, const vbyte_server_config *cfg);
/* Queue a query (k list indices, host memory); returns at once with its id.
 * VBYTE_EINVAL if a list index is out of range or the query can never fit
 * (more lists than max_batch_lists, more bytes than staging_bytes, more
 * output than arena_bytes). */
int vbyte_server_submit(vbyte_server *srv, const uint32_t *h_lists, size_t k,
                        uint64_t *query_id);
/* Block until the query is decoded; its latency (arrival to completion seen
 * by the scheduler, seconds) and data-error bits. */
int vbyte_server_wait(vbyte_server *srv, uint64_t query_id, double *latency_s,
                      uint32_t *status);
/* Device pointer to a decoded, unreleased query's n values, and how many
 * queries shared its batch. */
int vbyte_server_result(vbyte_server *srv, uint64_t query_id,
                        uint32_t **d_values, size_t *n,
                        uint32_t *batch_queries);
/* Return a decoded query's arena space. */
int vbyte_server_release(vbyte_server *srv, uint64_t query_id);
/* Open-loop replay: query i (lists h_query_lists[h_query_off[i] ..
 * h_query_off[i+1])) arrives h_arrival_s[i] seconds after the call starts;
 * blocks until all are decoded, writes each latency (from its scheduled
 * arrival) and status; queries are released as they complete. */
int vbyte_server_replay(vbyte_server *srv, const uint64_t *h_query_off,
                        const uint32_t *h_query_lists, size_t num_queries,
                        const double *h_arrival_s, double *h_latency_s,
                        uint32_t *h_status);
/* Batches launched, queries admitted, values and lists decoded so far. */
int vbyte_server_stats(vbyte_server *srv, uint64_t *batches, uint64_t *queries,
                       uint64_t *values, uint64_t *lists);
/* Stop the scheduler, wait for the GPU, free everything. */
void vbyte_server_destroy(vbyte_server *srv);

/* End-to-end form of vbyte_decode / vbyte_decode_delta for data in host memory: copies
 * h_in to the device, decodes (differentially when delta != 0) and copies the
 * n values back to h_out, through library-owned device buffers kept per
 * stream.  Inputs of 128 MiB or more go in pieces of 64 MiB: while later
 * pieces are still being copied in, earlier ones are counted and decoded
 * (the split count, scan and decode launches, the scan carrying the count
 * and running sum from piece to piece) and their values copied back, on
 * library-owned streams ordered after `stream`; page-locked h_in and h_out
 * let the copies in both directions overlap.  Synchronises the stream before
 * returning.  The data-error status is still read with vbyte_get_status(). */
int vbyte_decode_host(const uint8_t *h_in, size_t nbytes, uint32_t *h_out,
                      size_t n, int delta, uint32_t prev, void *stream);

/* ---- decoding without allocation ---------------------------------------- */

/* Largest input vbyte_decode_noalloc accepts: 128 MiB (about 2^27 one-byte
 * integers).  Its scratch is a fixed device array of about 576 KiB. */
#define VBYTE_NOALLOC_MAX_BYTES ((size_t)128 << 20)

/* The paper has no counterpart to this entry point: it is a deployment form
 * of vbyte_decode / vbyte_decode_delta for callers that cannot allocate
 * device memory -- a process whose device memory is all owned by another
 * allocator (a framework's caching allocator, an arena set aside at
 * start-up), or a latency-bound serving loop that cannot take the implicit
 * device synchronisation of cudaMalloc/cudaFree or an out-of-memory failure
 * in the middle of a request.  It decodes exactly as vbyte_decode (delta = 0)
 * or vbyte_decode_delta (delta != 0, from prev) and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Scratch: the per-tile descriptors live in one file-scope __device__ array
 * in the library, shared by every call on a device.  The first call on each
 * device (with that device current) looks up that array's address with
 * cudaGetSymbolAddress and the device's SM count; make that first call
 * before any stream capture.  Each call clears the part of the array that
 * must start at zero (cudaMemsetAsync on `stream`) before its kernel.
 * Calls whose work overlaps on the GPU -- on two streams, or from two host
 * threads without ordering -- race on the shared array and give unspecified
 * output: order them (one stream, or events).
 *
 * d_status: a caller-owned, 4-byte-aligned device word into which data
 * errors are OR-ed (VBYTE_ERR_* bits; never cleared by the library), or NULL
 * to discard them.  vbyte_get_status() does not see these errors.
 *
 * Returns VBYTE_ETOOBIG if nbytes > VBYTE_NOALLOC_MAX_BYTES (nothing is
 * queued), VBYTE_EINVAL as vbyte_decode does (and for a misaligned
 * d_status), VBYTE_ECUDA if the set-up or a launch fails. */
int vbyte_decode_noalloc(const uint8_t *d_in, size_t nbytes, uint32_t *d_out,
                         size_t n, int delta, uint32_t prev, uint32_t *d_status,
                         void *stream);

/* ---- the table-driven step (Sec. 4) ------------------------------------ */

/* The decoding table of Masked VByte (Sec. 4) as this library builds it, on
 * the host and in each CTA's shared memory: h_entries[m] (4096 entries) for
 * the 12-bit mask m of the high bits of the next 12 bytes (bit b: byte b) is
 * the number of bytes consumed (bits 0..3; 0: an integer of more than five
 * bytes, malformed) and the case (bits 4..11): 0..63, the next six integers
 * take one or two bytes each; 64..144, else the next four take at most three
 * bytes; 145..169, else the next two take at most five bytes; 255 for mask 0
 * (twelve one-byte integers).  h_cases[i] (170 entries) describes case i:
 * bits 0..2 the number of integers, bits 3+3t..5+3t the t-th length, bits
 * 24..27 the bytes consumed.  Host memory only; returns VBYTE_EINVAL for a
 * null pointer. */
int vbyte_table(uint16_t *h_entries, uint32_t *h_cases);

/* Decode a byte stream on the host by the table-driven steps (a table step
 * per whole 12-byte window, then one integer at a time, as Sec. 4 falls back
 * to the conventional decoder near the end); stores the first cap values in
 * h_out and returns how many the stream holds.  It gives Algorithm 1's
 * values; it exists to pin the table to them. */
size_t vbyte_table_decode(const uint8_t *h_in, size_t nbytes, uint32_t *h_out,
                          size_t cap);

/* ---- status ---------------------------------------------------------- */

/* Synchronise `stream`, return the OR of the VBYTE_ERR_* bits recorded by
 * every call on it since the last vbyte_get_status(), and clear them. */
int vbyte_get_status(void *stream, uint32_t *status_out);

/* A static English description of a return code. */
const char *vbyte_strerror(int code);

/* Bytes of workspace a call on an nbytes-byte input needs (for planning
 * graph capture); the library allocates it itself on first use. */
size_t vbyte_workspace_size(size_t nbytes);

/* Give `stream` (on the current device) a caller-owned workspace in place of
 * the one the library would allocate.  d_ws: device memory, 256-byte
 * aligned, `bytes` long, bytes >= vbyte_workspace_size(0).  From then on the
 * calls on that stream use it and never allocate a workspace: a call that
 * needs more than `bytes` (vbyte_workspace_size of its input) returns
 * VBYTE_ENOMEM and queues nothing.  The first 4 bytes become the stream's
 * status word; the bits recorded so far carry over (a 4-byte copy queued on
 * `stream`), and a workspace the library had allocated for the stream is
 * freed, queued on `stream`.  The buffer serves the stream until it is
 * replaced, handed back (d_ws = NULL: the library allocates again, the
 * status bits carry over) or dropped by vbyte_release_stream; the library
 * never frees it.  The staging buffers of vbyte_decode_host stay the
 * library's.  Returns VBYTE_EINVAL for a misaligned or too small buffer or
 * while `stream` is being captured, VBYTE_ENOMEM if handing back cannot
 * allocate, VBYTE_ECUDA if a queued copy fails. */
int vbyte_set_workspace(void *stream, void *d_ws, size_t bytes);

/* Forget `stream` (current device): free the workspace and the host-call
 * staging buffers the library allocated for it (queued on `stream`) and
 * drop a caller-owned workspace without freeing it.  Call it before
 * destroying the stream; status bits not yet read are lost.  Returns
 * VBYTE_OK, also for a stream the library has not seen. */
int vbyte_release_stream(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VBYTE_H */
