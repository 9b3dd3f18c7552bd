// Single-stream decoder (vbyte_decode, vbyte_decode_delta).
//
// Operation (arXiv 1503.07387): Algorithm 1 (Sec. 2) on a VByte byte stream
// (Sec. 1, Table 1), optionally followed by the prefix sum that undoes
// differential coding (Sec. 1 "Differential coding", Sec. 4).
//
// Design: count, then decode, with the input read from HBM once; two CTA
// barriers per 4 KiB tile.
//   * The stream is cut into 4 KiB tiles aligned to 16 bytes in absolute
//     address space; a tile owns the integers whose terminator byte lies in
//     it; the 16 bytes before it are staged too, so an integer that starts
//     up to four bytes earlier is assembled by the tile holding its
//     terminator.
//   * Persistent CTAs take tickets; ticket k counts tile k and, from ticket
//     `lead` (one 8 MiB chunk plus slack) on, decodes tile k - lead.  The
//     next ticket's tiles travel with cp.async while the current one is
//     processed.
//   * Count (a): per warp, terminator counts and (delta) value sums of its
//     slices; after the iteration's middle barrier one warp publishes the
//     tile's descriptor word and increments the chunk's counter.  The
//     data-error contract is checked here.
//   * Chunk scan: the CTA whose count completes a chunk (its increment of the
//     chunk's counter returns the last value) scans the chunk's 2048 tile
//     descriptors at the start of its next iteration: one prefix word per
//     tile, relative to the chunk's start, then the chunk's totals chained
//     to the chunk before it -- before the chunk's first decode ticket, and
//     before any decode of its own that could wait on it.
//   * Every word passed between CTAs (tile descriptors, tile prefixes, chunk
//     totals) carries a validity bit and is written and read with one 64-bit
//     relaxed access, so no step takes a memory fence.
//   * Decode (b, c): the tile prefix (its word and the totals of the chunk
//     before it) is staged an iteration ahead.  Each warp
//     stages its 512 bytes' values in its own buffer -- one-byte integers
//     straight from the bytes, codes of at most two bytes by a SWAR byte-pair
//     merge, longer codes by per-terminator assembly, each value assembled
//     once, then (delta) running sums relative to the warp's first value.
//     One barrier exchanges the per-warp totals (and the count partials and
//     the prefix); then each warp adds its base and writes its rank range
//     with coalesced 16-byte stores.
// Every wait is on work of a CTA holding an earlier ticket; each is bounded
// by the global timer (VBYTE_ERR_TIMEOUT on expiry).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "vbyte.h"
#include "vbyte_device.cuh"
#include "vbyte_emit.cuh"
#include "vbyte_internal.h"

namespace vbk {
namespace sd {

constexpr int kLanes = 32;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * kLanes;
constexpr int kTile = kThreads * kBPT;          // 4 KiB per tile
constexpr int kWarpBytes = kLanes * kBPT;       // 512 bytes per warp
constexpr uint64_t kChunk = 2048;               // tiles per chunk (8 MiB)
constexpr uint64_t kSlack = 4608;               // tickets between a chunk's last count ticket and its first decode
constexpr int kByteBuf = kHalo + kTile + 16;
constexpr int kWarpValBuf = kWarpBytes + 16;    // staged values of one warp (528)
constexpr int kStages = 2;                      // tickets in flight per CTA (processed + staged ahead)
static_assert(kChunk % kThreads == 0, "chunk scan: whole tiles per thread");
static_assert(kTile == 1 << 12, "tile addresses are t << 12");
static_assert(kChunk * kTile < (1ull << 24), "relative tile prefixes fit 23 bits");

// Published words (bit 0 = written):
//   tile descriptor  sum << 32 | f << 14 | count << 1 | 1   (count <= 4096)
//   tile prefix      s << 32 | f << 24 | rel << 1 | 1       (rel < 2^23: values
//                    in the chunk before the tile; (f, s) the segmented sum
//                    of the chunk's earlier tiles, f = 0 without list heads)
//   chunk totals     count << 1 | 1, x << 32 | 1            (values and running
//                    x after the chunk)
__device__ __forceinline__ uint64_t desc_word(uint32_t cnt, uint32_t f, uint32_t sum)
{
    return (static_cast<uint64_t>(sum) << 32) | (static_cast<uint64_t>(f) << 14) |
           (static_cast<uint64_t>(cnt) << 1) | 1u;
}
__device__ __forceinline__ uint32_t desc_count(uint64_t w) { return static_cast<uint32_t>(w >> 1) & 0x1FFFu; }
__device__ __forceinline__ uint32_t desc_flag(uint64_t w) { return static_cast<uint32_t>(w >> 14) & 1u; }
__device__ __forceinline__ uint32_t word_hi(uint64_t w) { return static_cast<uint32_t>(w >> 32); }

struct Params {
    const uint8_t *in;
    uint64_t nbytes;
    uint32_t *out;
    uint64_t n;
    uint64_t ntiles;
    uintptr_t base;            // 16-byte aligned address of tile 0
    uint32_t t_in_lo, t_in_hi; // tiles [t_in_lo, t_in_hi) lie wholly inside the stream
    uint64_t *tdesc;           // per tile: descriptor word
    uint64_t *tpre;            // per tile: prefix word
    uint64_t *cnext;           // per chunk: totals words (values, running x after it)
    unsigned int *cdone;       // per chunk: tiles counted
    unsigned int *ctr;         // tickets
    uint32_t *status;
    uint32_t prev;             // x_0
    uint64_t lead;             // tickets [0, lead) only count
    // batched lists only
    const uint64_t *bo;        // list byte offsets [L + 1]
    const uint64_t *vo;        // list value offsets [L + 1]
    const uint32_t *prevs;     // per-list x_0 (nullptr: 0)
    uint64_t L;
    const uint64_t *hr;        // per tile: [first, end) of the lists whose head may own a terminator in it
    // bounded waits and fault injection (tests of the timeout path)
    uint64_t wait_ns;          // bound of every wait
    uint64_t skip_tile;        // this tile's count is never published (~0: none)
    // single pass only
    uint64_t *lagg;            // per tile: its own count and sum
    uint64_t *linc;            // per tile: inclusive count, running x after it
};

struct Shared {
    alignas(16) uint8_t cbytes[kStages][kByteBuf];   // staged tiles to count
    alignas(16) uint8_t dbytes[kStages][kByteBuf];   // staged tiles to decode
    alignas(16) uint32_t vals[kWarps][kWarpValBuf];  // general warps: values at rank + sh
    uint32_t ccnt[kWarps], csum[kWarps];           // count: per-warp totals
    uint32_t dcnt[kWarps], dsum[kWarps];           // decode: per-warp totals
    unsigned long long R0;                         // decode: values before the tile
    uint32_t S0;                                   // decode: running x before the tile
    alignas(16) ulonglong2 pcn[kStages];           // prefetched: totals of the chunk before the decode tile's
    alignas(16) ulonglong2 ptp[kStages];           // prefetched: the decode tile's prefix word (and its pair's)
    uint32_t tnext;                                // the ticket to stage next
    uint32_t tinit[kStages];                       // the first tickets
    uint32_t csc[kWarps], css[kWarps], csf[kWarps];   // chunk scan partials
    long long scan_c;                              // chunk this CTA completed (scans it), or -1
};
// Batched lists: the list heads of the count and the decode tile, per-warp
// segment flags, and the segmented chunk scan's partials.
struct SharedS : Shared {
    alignas(16) unsigned long long hrc[kStages][2];   // head ranges of the staged count tiles (cp.async targets)
    alignas(16) unsigned long long hrd[kStages][2];   // ... of the staged decode tiles
    HeadTab hc, hd;                             // heads of the count and the decode tile
    uint32_t cflag[kWarps];                     // count: a list head was crossed in this warp
    uint32_t dflag[kWarps];                     // decode: the same
    uint32_t dhf[kWarps];                       // decode: this warp's first rank after a head (values from it on are absolute)
};
static_assert(offsetof(SharedS, hrc) % 16 == 0 && offsetof(SharedS, hrd) % 16 == 0, "head range alignment");

static_assert(offsetof(Shared, cbytes) % 16 == 0 && kByteBuf % 16 == 0, "cbytes alignment");
static_assert(offsetof(Shared, dbytes) % 16 == 0 && offsetof(Shared, vals) % 16 == 0, "dbytes/vals alignment");
static_assert((kWarpValBuf * 4) % 16 == 0, "per-warp value buffers keep 16-byte alignment");
static_assert(offsetof(Shared, pcn) % 16 == 0 && offsetof(Shared, ptp) % 16 == 0, "prefix buffers alignment");

__device__ __forceinline__ bool inside(const Params &p, uint32_t t) { return t >= p.t_in_lo && t < p.t_in_hi; }

// Stage tile t (its 16-byte slices, the 16 bytes before it, zeros outside
// the stream) into `bytes`; the caller commits, waits and syncs.  The 16 bytes
// after the tile are zeroed once, at the kernel's start.
__device__ __forceinline__ void issue_stage(const Params &p, uint32_t t, int tid, uint8_t *bytes)
{
    const uintptr_t tstart = p.base + (static_cast<uintptr_t>(t) << 12);
    const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
    uint8_t *dst = bytes + kHalo + tid * kBPT;
    if (t > 0 && t < p.t_in_hi) {   // interior tile (its 16 bytes before too): no checks
        cp_async16(dst, reinterpret_cast<const void *>(va));
        if (tid == 0) cp_async16(bytes, reinterpret_cast<const void *>(tstart - 16));
        return;
    }
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    if (va >= lo && va + kBPT <= hi) {
        cp_async16(dst, reinterpret_cast<const void *>(va));
    } else {
        uint32_t wb[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const uintptr_t ad = va + j;
            if (ad >= lo && ad < hi)
                wb[j >> 2] |= static_cast<uint32_t>(*reinterpret_cast<const uint8_t *>(ad)) << (8 * (j & 3));
        }
        *reinterpret_cast<uint4 *>(dst) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
    }
    if (tid == 0) {
        if (t > 0)
            cp_async16(bytes, reinterpret_cast<const void *>(tstart - 16));
        else
            *reinterpret_cast<uint4 *>(bytes) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// ---- counting

template <bool kDelta>
__device__ __forceinline__ void count_partials(const Params &p, uint64_t t, Shared &S, const uint8_t *bytes)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = inside(p, static_cast<uint32_t>(t));
    const uint4 w0 = *reinterpret_cast<const uint4 *>(bytes + kHalo + tid * kBPT);
    const uint32_t wp0 = reinterpret_cast<const uint32_t *>(bytes)[(kHalo + tid * kBPT) / 4 - 1];
    uint32_t cnt, vsum = 0;
    if (interior && !((w0.x | w0.y | w0.z | w0.w) & 0x80808080u) && !(wp0 & 0x80000000u)) {
        cnt = kBPT;   // one-byte integers only
        if (kDelta) vsum = byte_sum4(w0);
    } else {
        const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
        const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
        cnt = __popc(m.tc);
        const uint32_t c20 = ~m.t20 & 0xFFFFFu;
        if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
            atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
        if (t == p.ntiles - 1 && hi - 1 >= va && hi - 1 < va + kBPT && !((m.tl >> (hi - 1 - va)) & 1u))
            atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        if (kDelta) {
            if (interior && !(c20 & (c20 << 1) & 0xFFFF8u))
                vsum = sum_le2_fast(m.w, m.wprev);
            else
                assemble_all(reinterpret_cast<const uint32_t *>(bytes), tid, m.tl, m.t20, m.tc,
                             [&](uint32_t v) { vsum += v; });
        }
    }
    const uint32_t wc = __reduce_add_sync(~0u, cnt);
    const uint32_t ws = kDelta ? __reduce_add_sync(~0u, vsum) : 0u;
    if (lane == 0) {
        S.ccnt[warp] = wc;
        S.csum[warp] = ws;
    }
}

// One warp, after the middle barrier: publish tile t's descriptor.  Lane 0
// returns the chunk counter's old value (read at the end of the iteration).
template <bool kDelta>
__device__ __forceinline__ unsigned int count_publish(const Params &p, uint64_t t, const Shared &S, int lane)
{
    const uint32_t tc = __reduce_add_sync(~0u, lane < kWarps ? S.ccnt[lane] : 0u);
    const uint32_t ts = kDelta ? __reduce_add_sync(~0u, lane < kWarps ? S.csum[lane] : 0u) : 0u;
    unsigned int old = 0;
    if (lane == 0) {
        if (t != p.skip_tile) st_relaxed_u64(p.tdesc + t, desc_word(tc, 0u, ts));
        old = atomicAdd(p.cdone + t / kChunk, 1u);
    }
    return old;
}

// ---- chunk scan (whole CTA)

__device__ __forceinline__ uint64_t chunk_tiles(const Params &p, long long c)
{
    const uint64_t c0 = static_cast<uint64_t>(c) * kChunk;
    return ((c0 + kChunk < p.ntiles) ? c0 + kChunk : p.ntiles) - c0;
}

// Prefix words of chunk c's tiles from their descriptors (segmented sums
// when kSeg), then the chunk's totals chained to the chunk before it.  Run by
// the CTA that completed the chunk's count.
template <bool kSeg>
__device__ void chunk_scan(const Params &p, uint64_t c, Shared &S)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kPer = static_cast<int>(kChunk / kThreads);   // 8
    const uint64_t c0 = c * kChunk;
    const uint64_t c1 = (c0 + kChunk < p.ntiles) ? c0 + kChunk : p.ntiles;
    const uint64_t tb = c0 + static_cast<uint64_t>(kPer) * tid;
    // the thread's descriptors in one batch of loads (words past the chunk
    // stay inside the workspace and are ignored), then waits for any not yet
    // published
    uint64_t d[kPer];
#pragma unroll
    for (int i = 0; i < kPer; i += 2) {
        ulonglong2 v = make_ulonglong2(0ull, 0ull);
        if (tb + i < c1) v = __ldcg(reinterpret_cast<const ulonglong2 *>(p.tdesc + tb + i));
        d[i] = v.x;
        d[i + 1] = v.y;
    }
    uint32_t tcn = 0;
    Seg ts;
    ts.f = ts.s = 0u;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        if (tb + i < c1) {
            if (!(d[i] & 1u)) d[i] = wait_word(p.tdesc + tb + i, p.status, p.wait_ns);
            Seg e;
            e.f = kSeg ? desc_flag(d[i]) : 0u;
            e.s = word_hi(d[i]);
            tcn += desc_count(d[i]);
            ts = seg_op(ts, e);
        }
    }
    const uint32_t icn = warp_incl_scan(tcn, lane);
    const Seg is = warp_seg_incl(ts, lane);
    if (lane == 31) {
        S.csc[warp] = icn;
        S.css[warp] = is.s;
        S.csf[warp] = is.f;
    }
    __syncthreads();
    uint32_t wc0 = 0, call = 0;
    Seg w0, wall;
    w0.f = w0.s = wall.f = wall.s = 0u;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
        Seg e;
        e.f = S.csf[q];
        e.s = S.css[q];
        if (q < warp) {
            wc0 += S.csc[q];
            w0 = seg_op(w0, e);
        }
        call += S.csc[q];
        wall = seg_op(wall, e);
    }
    Seg ex;
    ex.f = __shfl_up_sync(~0u, is.f, 1);
    ex.s = __shfl_up_sync(~0u, is.s, 1);
    if (lane == 0) ex.f = ex.s = 0u;
    uint32_t rel = wc0 + icn - tcn;
    Seg x = seg_op(w0, ex);
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        if (tb + i < c1) {
            st_relaxed_u64(p.tpre + tb + i, (static_cast<uint64_t>(x.s) << 32) |
                                                (static_cast<uint64_t>(x.f) << 24) |
                                                (static_cast<uint64_t>(rel) << 1) | 1u);
            Seg e;
            e.f = kSeg ? desc_flag(d[i]) : 0u;
            e.s = word_hi(d[i]);
            rel += desc_count(d[i]);
            x = seg_op(x, e);
        }
    }
    if (tid == 0) {
        uint64_t pc = 0;
        uint32_t ps = p.prev;
        if (c > 0) {
            pc = wait_word(p.cnext + 2 * (c - 1), p.status, p.wait_ns) >> 1;
            ps = word_hi(wait_word(p.cnext + 2 * (c - 1) + 1, p.status, p.wait_ns));
        }
        st_relaxed_u64(p.cnext + 2 * c, ((pc + call) << 1) | 1u);
        st_relaxed_u64(p.cnext + 2 * c + 1, (static_cast<uint64_t>(seg_apply(ps, wall)) << 32) | 1u);
        if (c1 == p.ntiles && pc + call != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
    }
}

// ---- tile prefixes

// One thread: the decode tile's values before it (R0) and running x before
// it (S0), from the words staged an iteration ahead, re-read (bounded) if
// they were not yet published then.  After a timeout R0 = n, so nothing is
// written.
__device__ __forceinline__ void tile_prefix(const Params &p, uint64_t t, Shared &S, int b)
{
    const uint64_t c = t / kChunk;
    uint64_t tp = (t & 1u) ? S.ptp[b].y : S.ptp[b].x;
    uint64_t cn0 = 1u, cn1 = (static_cast<uint64_t>(p.prev) << 32) | 1u;
    if (c > 0) {
        cn0 = S.pcn[b].x;
        cn1 = S.pcn[b].y;
    }
    if (!(tp & cn0 & cn1 & 1u)) {   // not yet published when staged
        if (!(tp & 1u)) tp = wait_word(p.tpre + t, p.status, p.wait_ns);
        if (!(cn0 & 1u)) cn0 = wait_word(p.cnext + 2 * (c - 1), p.status, p.wait_ns);
        if (!(cn1 & 1u)) cn1 = wait_word(p.cnext + 2 * (c - 1) + 1, p.status, p.wait_ns);
    }
    const uint32_t rel = static_cast<uint32_t>(tp >> 1) & 0x7FFFFFu;
    const uint32_t s = word_hi(tp);
    S.R0 = (tp & cn0 & cn1 & 1u) ? (cn0 >> 1) + rel : p.n;
    S.S0 = ((tp >> 24) & 1u) ? s : word_hi(cn1) + s;
}

// ---- decoding
//
// Before the middle barrier each warp stages its values in its own buffer:
// warp rank r at vals[4 + r], running sums (delta) relative to the warp's
// first value.  After it, one coalesced copy-out adds the warp's base and
// realigns to 16-byte output quads.  A warp of one-byte integers only may
// instead keep its values in registers until the copy-out (kKeep).

// A warp of one-byte integers only may skip the buffer (kKeep): it writes
// its values at the copy-out straight from the staged bytes.
struct RegA {
    bool on;   // warp-uniform: nothing is in the value buffer
};

// A decoded tile in shared memory: per warp, its staged values and its value
// count and (delta) sum.
struct TileView {
    uint32_t (*vals)[kWarpValBuf];
    uint32_t *dcnt, *dsum;
};

// kCheck: also check the data-error contract (the single-pass kernel has no
// count pass to do it).  kCopy (with kKeep): a one-byte warp copies its staged
// bytes, with 16 before and after, into its value buffer (bytes 16..527 are
// the warp's), so that the copy-out can run after the byte buffer is reused.
template <bool kDelta, bool kKeep, bool kCheck = false, bool kCopy = false>
__device__ __forceinline__ void decode_stage(const Params &p, uint64_t t, const TileView &V, const uint8_t *bytes,
                                             RegA &ra)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = inside(p, static_cast<uint32_t>(t));
    const uint4 w0 = *reinterpret_cast<const uint4 *>(bytes + kHalo + tid * kBPT);
    const uint32_t wp0 = reinterpret_cast<const uint32_t *>(bytes)[(kHalo + tid * kBPT) / 4 - 1];
    const bool mineA = interior && !((w0.x | w0.y | w0.z | w0.w) & 0x80808080u) && !(wp0 & 0x80000000u);
    uint32_t *vals = V.vals[warp];
    uint32_t wc, ws = 0;
    if (kKeep && __all_sync(~0u, mineA)) {
        // one-byte integers only: written from the bytes at the copy-out
        if (kDelta) ws = __reduce_add_sync(~0u, byte_sum4(w0));
        ra.on = true;
        wc = kWarpBytes;
        if (kCopy) {
            const uint4 *src = reinterpret_cast<const uint4 *>(bytes + kHalo + warp * kWarpBytes - 16);
            uint4 *dst = reinterpret_cast<uint4 *>(vals);
            dst[lane] = src[lane];
            if (lane < 2) dst[32 + lane] = src[32 + lane];
        }
    } else if (__all_sync(~0u, mineA)) {
        // one-byte integers only: lane l holds warp ranks 16l .. 16l+15
        uint4 q[4] = {bytes_as_values(w0.x), bytes_as_values(w0.y), bytes_as_values(w0.z),
                      bytes_as_values(w0.w)};
        if (kDelta) {
            const uint32_t mine = byte_sum4(w0);
            const uint32_t incs = warp_incl_scan(mine, lane);
            ws = __shfl_sync(~0u, incs, 31);
            uint32_t run = incs - mine;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                run += q[j].x; q[j].x = run;
                run += q[j].y; q[j].y = run;
                run += q[j].z; q[j].z = run;
                run += q[j].w; q[j].w = run;
            }
        }
        uint4 *d4 = reinterpret_cast<uint4 *>(vals + 4 + 16 * lane);
#pragma unroll
        for (int j = 0; j < 4; ++j) d4[j] = q[j];
        wc = kWarpBytes;
    } else {
        ra.on = false;
        const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
        const uint32_t *const sw = reinterpret_cast<const uint32_t *>(bytes);
        const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
        const uint32_t cnt = __popc(m.tc);
        const uint32_t c20 = ~m.t20 & 0xFFFFFu;
        const bool notB = (c20 & (c20 << 1) & 0xFFFF8u) != 0;
        if (kCheck) {
            if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
                atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
            if (t == p.ntiles - 1 && hi - 1 >= va && hi - 1 < va + kBPT && !((m.tl >> (hi - 1 - va)) & 1u))
                atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        }
        const uint32_t inc = warp_incl_scan(cnt, lane);
        wc = __shfl_sync(~0u, inc, 31);
        uint32_t *dst = vals + 4 + inc - cnt;
        uint32_t vsum = 0;
        if (!__any_sync(~0u, notB)) {
            // codes of at most two bytes: the lane's sum by the byte-weight
            // formula, then the values (with running sums) in one SWAR pass
            uint32_t run = 0;
            if (kDelta) {
                vsum = interior ? sum_le2_fast(m.w, m.wprev) : sum_le2(m.w, m.wprev, m.tc);
                const uint32_t incs = warp_incl_scan(vsum, lane);
                ws = __shfl_sync(~0u, incs, 31);
                run = incs - vsum;
            }
            const uint32_t c4[4] = {m.w.x, m.w.y, m.w.z, m.w.w};
            uint32_t wp = m.wprev;
            int qi = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const Pairs pr = pairs_le2(wp, c4[j]);
                uint32_t q01 = prmt(pr.lob, pr.hib, 0x5140u);
                uint32_t q23 = prmt(pr.lob, pr.hib, 0x7362u);
                q01 -= (q01 & 0xFF00FF00u) >> 1;
                q23 -= (q23 & 0xFF00FF00u) >> 1;
                const uint32_t v4[4] = {q01 & 0xFFFFu, q01 >> 16, q23 & 0xFFFFu, q23 >> 16};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if ((m.tc >> (4 * j + i)) & 1u) {
                        if (kDelta) {
                            run += v4[i];
                            dst[qi++] = run;
                        } else {
                            dst[qi++] = v4[i];
                        }
                    }
                }
                wp = c4[j];
            }
        } else {
            // longer codes: each value assembled once (pass 1), then running
            // sums from this lane's offset within the warp (pass 2)
            assemble_all(sw, tid, m.tl, m.t20, m.tc, [&](uint32_t v) {
                *dst++ = v;
                vsum += v;
            });
            dst -= cnt;
            if (kDelta) {
                const uint32_t incs = warp_incl_scan(vsum, lane);
                ws = __shfl_sync(~0u, incs, 31);
                uint32_t run = incs - vsum;
                for (uint32_t i = 0; i < cnt; ++i) {
                    run += dst[i];
                    dst[i] = run;
                }
            }
        }
    }
    if (lane == 0) {
        V.dcnt[warp] = wc;
        V.dsum[warp] = ws;
    }
}

// After the middle barrier: this warp's values to the output, coalesced;
// with kRank each value also gets its global rank (gaps minus one).  R0, S0:
// the values before the tile and the running x before it; wb: the warp's
// first staged byte (one-byte warps, ra.on).
template <bool kDelta, bool kRank>
__device__ __forceinline__ void decode_emit(const Params &p, const TileView &V, unsigned long long R0, uint32_t S0,
                                            const RegA &ra, const uint8_t *wb)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
    const long long n = static_cast<long long>(p.n);
    // the warps before this one: their value counts and sums
    const uint32_t wbase = __reduce_add_sync(~0u, lane < warp ? V.dcnt[lane] : 0u);
    const uint32_t wsb = kDelta ? __reduce_add_sync(~0u, lane < warp ? V.dsum[lane] : 0u) : 0u;
    const uint32_t wc = V.dcnt[warp];
    const long long G0 = static_cast<long long>(R0 + wbase);   // global rank of warp rank 0
    const uint32_t add = kDelta ? S0 + wsb : 0u;
    const int sh = static_cast<int>((out_word + static_cast<uint32_t>(G0)) & 3u);
    uint32_t *vals = V.vals[warp];
    uint32_t *const oq = p.out + (G0 - sh);   // 16-byte aligned; quad q at oq + 4q
    if (ra.on) {   // warp-uniform
        if (G0 + kWarpBytes <= n) {
            const uint32_t rb = static_cast<uint32_t>(G0);
            switch (sh) {
            case 0: emit_bytes_a<0, kDelta, kRank>(oq, wb, add, rb, lane); break;
            case 1: emit_bytes_a<1, kDelta, kRank>(oq, wb, add, rb, lane); break;
            case 2: emit_bytes_a<2, kDelta, kRank>(oq, wb, add, rb, lane); break;
            default: emit_bytes_a<3, kDelta, kRank>(oq, wb, add, rb, lane); break;
            }
            return;
        }
        // near the end of the output: through the buffer, with the checks
        // (wb may lie inside the buffer: every lane reads before any writes)
        const uint4 w = *reinterpret_cast<const uint4 *>(wb + lane * kBPT);
        __syncwarp();
        uint4 q[4] = {bytes_as_values(w.x), bytes_as_values(w.y), bytes_as_values(w.z), bytes_as_values(w.w)};
        if (kDelta) {
            const uint32_t mine = byte_sum4(w);
            uint32_t run = warp_incl_scan(mine, lane) - mine;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                run += q[j].x; q[j].x = run;
                run += q[j].y; q[j].y = run;
                run += q[j].z; q[j].z = run;
                run += q[j].w; q[j].w = run;
            }
        }
        uint4 *d4 = reinterpret_cast<uint4 *>(vals + 4 + 16 * lane);
#pragma unroll
        for (int j = 0; j < 4; ++j) d4[j] = q[j];
        __syncwarp();
    }
    emit_staged<kRank>(oq, vals, static_cast<int>(wc), add, static_cast<uint32_t>(G0), n - G0, lane, sh);
}

// After the middle barrier: this warp's values to the output, coalesced.
// The same for batched lists: the warp's base is the segmented running value
// before it, added only to ranks below the warp's first head value.
template <bool kDelta>
__device__ __forceinline__ void decode_emit_seg(const Params &p, const SharedS &S)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
    const long long n = static_cast<long long>(p.n);
    uint32_t wbase = 0;
    Seg wsb;
    wsb.f = wsb.s = 0u;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
        wbase += (q < warp) ? S.dcnt[q] : 0u;
        if (kDelta && q < warp) {
            Seg e;
            e.f = S.dflag[q];
            e.s = S.dsum[q];
            wsb = seg_op(wsb, e);
        }
    }
    const uint32_t wc = S.dcnt[warp];
    const long long G0 = static_cast<long long>(S.R0 + wbase);   // global rank of warp rank 0
    const uint32_t add = kDelta ? seg_apply(S.S0, wsb) : 0u;
    const int hf = kDelta ? static_cast<int>(min(S.dhf[warp], wc)) : static_cast<int>(wc);   // ranks [hf, wc) are absolute
    const int sh = static_cast<int>((out_word + static_cast<uint32_t>(G0)) & 3u);
    const uint32_t *vals = S.vals[warp];
    uint32_t *const oq = p.out + (G0 - sh);   // 16-byte aligned; quad q at oq + 4q
    // the same bounds as emit_staged, with the alignment chosen per quad: one
    // copy of the loop keeps this larger kernel's code small
    const long long room = n - G0;
    const int lim = room < wc ? (room > 0 ? static_cast<int>(room) : 0) : static_cast<int>(wc);
    const int qa = sh ? 1 : 0;
    const int qb = (lim + sh) >> 2;
    for (int q = qa + lane; q < qb; q += kLanes) {
        const uint4 U = *reinterpret_cast<const uint4 *>(vals + 4 * q);
        const uint4 V = *reinterpret_cast<const uint4 *>(vals + 4 * q + 4);
        uint4 e;
        switch (sh) {
        case 0: e = V; break;
        case 1: e = make_uint4(U.w, V.x, V.y, V.z); break;
        case 2: e = make_uint4(U.z, U.w, V.x, V.y); break;
        default: e = make_uint4(U.y, U.z, U.w, V.x); break;
        }
        const int r0 = 4 * q - sh;
        e.x += (r0 < hf) ? add : 0u;
        e.y += (r0 + 1 < hf) ? add : 0u;
        e.z += (r0 + 2 < hf) ? add : 0u;
        e.w += (r0 + 3 < hf) ? add : 0u;
        st_quad(oq + 4 * q, e);
    }
    const bool whole = qb > qa;
    const int hb = whole ? min(4 * qa - sh, lim) : lim;   // ranks [0, hb)
    const int tb = whole ? 4 * qb - sh : lim;             // ranks [tb, lim)
    for (int r = lane; r < hb; r += kLanes) oq[sh + r] = vals[4 + r] + (r < hf ? add : 0u);
    for (int r = tb + lane; r < lim; r += kLanes) oq[sh + r] = vals[4 + r] + (r < hf ? add : 0u);
}

// ---- batched lists (segmented sums restart at every list head)

__device__ __forceinline__ HeadSrc head_src(const Params &p) { return HeadSrc{p.bo, p.vo, p.prevs}; }

// Count partials of a tile with list heads: the lane's sum since its last
// head (from that list's x_0), and the warp's segmented aggregate.
__device__ __forceinline__ void count_partials_seg(const Params &p, uint64_t t, SharedS &S, const uint8_t *bytes,
                                                   uint64_t ha, uint64_t he)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = inside(p, static_cast<uint32_t>(t));
    const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
    const uint32_t *const sw = reinterpret_cast<const uint32_t *>(bytes);
    const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
    const uint32_t cnt = __popc(m.tc);
    const uint32_t c20 = ~m.t20 & 0xFFFFFu;
    if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
        atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
    if (t == p.ntiles - 1 && hi - 1 >= va && hi - 1 < va + kBPT && !((m.tl >> (hi - 1 - va)) & 1u))
        atomicOr(p.status, VBYTE_ERR_TRUNCATED);
    const long long trel = static_cast<long long>(tstart) - static_cast<long long>(lo);
    const HeadWin h = head_window(sw, S.hc.bits, tid, m.tl);
    const uint32_t ht = head_terms(h, m.tc);
    Seg sg;
    sg.f = ht ? 1u : 0u;
    sg.s = 0u;
    if (ht) {
        sg.s = slice_seg_sum(head_src(p), S.hc, sw, tid, m.tl, m.t20, m.tc, h, ht, trel + tid * kBPT, ha, he);
    } else if (interior && !(c20 & (c20 << 1) & 0xFFFF8u)) {
        sg.s = sum_le2_fast(m.w, m.wprev);
    } else {
        assemble_all(sw, tid, m.tl, m.t20, m.tc, [&](uint32_t v) { sg.s += v; });
    }
    sg = warp_seg_incl(sg, lane);
    const uint32_t wc = __reduce_add_sync(~0u, cnt);
    if (lane == 31) {
        S.ccnt[warp] = wc;
        S.csum[warp] = sg.s;
        S.cflag[warp] = sg.f;
    }
}

// One warp, after the middle barrier: the tile's segmented descriptor.
template <bool kDelta>
__device__ __forceinline__ unsigned int count_publish_seg(const Params &p, uint64_t t, const SharedS &S, int lane)
{
    const uint32_t tc = __reduce_add_sync(~0u, lane < kWarps ? S.ccnt[lane] : 0u);
    Seg ws;
    ws.f = (kDelta && lane < kWarps) ? S.cflag[lane] : 0u;
    ws.s = (kDelta && lane < kWarps) ? S.csum[lane] : 0u;
    ws = warp_seg_incl(ws, lane);
    const uint32_t f = __shfl_sync(~0u, ws.f, 31), sm = __shfl_sync(~0u, ws.s, 31);
    unsigned int old = 0;
    if (lane == 0) {
        if (t != p.skip_tile) st_relaxed_u64(p.tdesc + t, desc_word(tc, f, sm));
        old = atomicAdd(p.cdone + t / kChunk, 1u);
    }
    return old;
}

// Decode staging of a tile with list heads (every warp takes the general
// path): values with restarts at heads; values from the warp's first head on
// are absolute, earlier ones relative to the warp's first value.
template <bool kDelta>
__device__ __forceinline__ void decode_stage_seg(const Params &p, uint64_t t, SharedS &S, const uint8_t *bytes,
                                                 uint64_t ha, uint64_t he)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = inside(p, static_cast<uint32_t>(t));
    const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
    const uint32_t *const sw = reinterpret_cast<const uint32_t *>(bytes);
    const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
    const uint32_t cnt = __popc(m.tc);
    const uint32_t inc = warp_incl_scan(cnt, lane);
    const uint32_t wc = __shfl_sync(~0u, inc, 31);
    uint32_t *const dst = S.vals[warp] + 4 + inc - cnt;
    uint32_t hf = 0xFFFFFFFFu, wsum = 0, wflag = 0;
    if (kDelta) {
        const long long srel = static_cast<long long>(tstart) - static_cast<long long>(lo) + tid * kBPT;
        const HeadWin h = head_window(sw, S.hd.bits, tid, m.tl);
        const uint32_t ht = head_terms(h, m.tc);
        Seg sg;
        sg.f = ht ? 1u : 0u;
        sg.s = 0u;
        // pass 1: values assembled once; a head restarts the lane's running sum
        int qi = 0;
        assemble_all_o(sw, tid, m.tl, m.t20, m.tc, [&](int o, uint32_t v) {
            dst[qi++] = v;
            if ((ht >> o) & 1u)
                sg.s = head_prev(head_src(p), S.hd, h, o, tid, srel, ha, he) + v;
            else
                sg.s += v;
        });
        const Seg incl = warp_seg_incl(sg, lane);
        wsum = __shfl_sync(~0u, incl.s, 31);
        wflag = __shfl_sync(~0u, incl.f, 31);
        Seg ex;
        ex.f = __shfl_up_sync(~0u, incl.f, 1);
        ex.s = __shfl_up_sync(~0u, incl.s, 1);
        if (lane == 0) ex.f = ex.s = 0u;
        // pass 2: running values (absolute after a head, else relative)
        uint32_t run = ex.s;
        uint32_t mm = m.tc;
        for (int i = 0; mm; ++i) {
            const int o = __ffs(mm) - 1;
            mm &= mm - 1u;
            if ((ht >> o) & 1u)
                run = head_prev(head_src(p), S.hd, h, o, tid, srel, ha, he) + dst[i];
            else
                run += dst[i];
            dst[i] = run;
        }
        // the warp's first absolute rank: its first head value
        if (ht) hf = inc - cnt + __popc(m.tc & ((1u << (__ffs(ht) - 1)) - 1u));
        hf = __reduce_min_sync(~0u, hf);
    }
    if (lane == 0) {
        S.dcnt[warp] = wc;
        S.dsum[warp] = wsum;
        S.dflag[warp] = wflag;
        S.dhf[warp] = hf;
    }
}

// After the middle barrier, tiles with heads: each list head in my slice must
// start at rank vo[j] and follow a terminator.
__device__ __forceinline__ void check_heads(const Params &p, uint64_t t, SharedS &S, const uint8_t *bytes,
                                            uint64_t ha, uint64_t he, unsigned long long R0)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = inside(p, static_cast<uint32_t>(t));
    const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
    const uint32_t *const sw = reinterpret_cast<const uint32_t *>(bytes);
    const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
    const uint32_t cnt = __popc(m.tc);
    const uint32_t inc = warp_incl_scan(cnt, lane);
    uint32_t wbase = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) wbase += (q < warp) ? S.dcnt[q] : 0u;
    const HeadWin h = head_window(sw, S.hd.bits, tid, m.tl);
    uint32_t hs = (h.h24 >> kHeadBack) & 0xFFFFu;
    const long long srel = static_cast<long long>(tstart) - static_cast<long long>(lo) + tid * kBPT;
    while (hs) {
        const int k = __ffs(hs) - 1;
        hs &= hs - 1u;
        const long long pos = srel + k;
        if (pos < 0 || pos >= static_cast<long long>(p.nbytes)) continue;
        if (pos > 0 && !((h.t24 >> (kHeadBack + k - 1)) & 1u)) atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        const uint64_t rank = R0 + wbase + inc - cnt + __popc(m.tc & ((1u << k) - 1u));
        if (he - ha <= static_cast<uint64_t>(kMaxHeadList)) {
            const int qs = kHalo + tid * kBPT + k;
            for (int i = tab_last_le(S.hd, static_cast<int>(he - ha), qs); i >= 0; --i) {
                if (S.hd.pos[i] != qs) break;
                if (S.hd.vo[i] != rank) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
            }
        } else {
            for (long long j = last_list_at(head_src(p), ha, he, pos); j >= static_cast<long long>(ha); --j) {
                if (static_cast<long long>(p.bo[j]) != pos) break;
                if (p.vo[j] != rank) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
            }
        }
    }
}

// ---- kernel

template <bool kDelta, bool kSeg, bool kRank = false>
__global__ void __launch_bounds__(kThreads, kSeg ? 4 : 5) sdecode_kernel(const Params p)
{
    using Sm = typename std::conditional<kSeg, SharedS, Shared>::type;
    __shared__ Sm S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // tickets and tile indices fit 32 bits (checked by the host)
    const uint32_t ntiles = static_cast<uint32_t>(p.ntiles), lead = static_cast<uint32_t>(p.lead);
    const uint32_t total = ntiles + lead;
    if (tid < 2 * kStages) {   // the zeros after each staging buffer
        uint8_t *buf = (tid < kStages) ? S.cbytes[tid] : S.dbytes[tid - kStages];
        *reinterpret_cast<uint4 *>(buf + kHalo + kTile) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int j = 0; j < kStages - 1; ++j) S.tinit[j] = atomicAdd(p.ctr, 1u);
        S.tnext = atomicAdd(p.ctr, 1u);
        S.scan_c = -1;
    }
    __syncthreads();
    // tickets of the buffers b, b + 1, ... (mod kStages): processed now, staged
    uint32_t q[kStages - 1];
#pragma unroll
    for (int j = 0; j < kStages - 1; ++j) q[j] = S.tinit[j];
    auto stage = [&](uint32_t tk, int b) {
        if (tk < ntiles) issue_stage(p, tk, tid, S.cbytes[b]);
        if (tk >= lead && tk < total) {
            const uint32_t t = tk - lead;
            issue_stage(p, t, tid, S.dbytes[b]);
            // the prefix words, probably published by now (checked on use;
            // 16-byte copies bypass L1, which may hold a stale line)
            if (tid == 96) cp_async16(&S.ptp[b], p.tpre + (t & ~1u));
            if (tid == 128 && t >= kChunk) cp_async16(&S.pcn[b], p.cnext + 2 * (t / kChunk - 1));
        }
        if constexpr (kSeg) {   // the tiles' list-head ranges travel with them
            if (tid == 32 && tk < ntiles) cp_async16(S.hrc[b], p.hr + 2 * static_cast<uint64_t>(tk));
            if (tid == 64 && tk >= lead && tk < total) cp_async16(S.hrd[b], p.hr + 2 * static_cast<uint64_t>(tk - lead));
        }
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < kStages - 1; ++j) stage(q[j], j);
    for (int b = 0; q[0] < total; b = (b == kStages - 1) ? 0 : b + 1) {
        const uint32_t k = q[0];
        cp_async_wait_prior<kStages - 2>();   // ticket k's group is complete
        __syncthreads();                      // ... for every thread; the previous iteration is over
        const uint32_t kn = S.tnext;          // staged now, processed kStages - 1 iterations later
        uint32_t knn = 0;
        if (tid == 0) knn = atomicAdd(p.ctr, 1u);
        stage(kn, (b == 0) ? kStages - 1 : b - 1);
        // the count this CTA published last iteration completed its chunk
        if (S.scan_c >= 0) chunk_scan<kSeg>(p, static_cast<uint64_t>(S.scan_c), S);   // CTA-uniform

        const bool dec = k >= lead;
        RegA ra;
        ra.on = false;
        const uint32_t t = k - lead;
        // batched lists: the heads of the count tile (delta only) and of the decode tile
        bool cheads = false, dheads = false;
        uint64_t cha = 0, che = 0, dha = 0, dhe = 0;
        if constexpr (kSeg) {
            if (kDelta && k < ntiles) {
                cha = S.hrc[b][0];
                che = S.hrc[b][1];
                cheads = cha < che;
            }
            if (dec) {
                dha = S.hrd[b][0];
                dhe = S.hrd[b][1];
                dheads = dha < dhe;
            }
            if (cheads || dheads) {   // CTA-uniform
                for (int i = tid; i < kHeadWords; i += kThreads) {
                    S.hc.bits[i] = 0u;
                    S.hd.bits[i] = 0u;
                }
                __syncthreads();
                if (cheads) fill_heads(head_src(p), static_cast<long long>(p.base + k * kTile) -
                                                         static_cast<long long>(reinterpret_cast<uintptr_t>(p.in)),
                                       cha, che, S.hc, true, false, kThreads);
                if (dheads) fill_heads(head_src(p), static_cast<long long>(p.base + t * kTile) -
                                                         static_cast<long long>(reinterpret_cast<uintptr_t>(p.in)),
                                       dha, dhe, S.hd, kDelta, true, kThreads);
                __syncthreads();
            }
        }
        if (k < ntiles) {
            if constexpr (kSeg) {
                if (cheads)
                    count_partials_seg(p, k, S, S.cbytes[b], cha, che);
                else {
                    count_partials<kDelta>(p, k, S, S.cbytes[b]);
                    if (lane == 0) S.cflag[warp] = 0u;
                }
            } else {
                count_partials<kDelta>(p, k, S, S.cbytes[b]);
            }
        }
        if (dec) {
            if (tid == 0) tile_prefix(p, t, S, b);
            if constexpr (kSeg) {
                if (kDelta && dheads) {
                    decode_stage_seg<kDelta>(p, t, S, S.dbytes[b], dha, dhe);
                } else {
                    decode_stage<kDelta, false>(p, t, TileView{S.vals, S.dcnt, S.dsum}, S.dbytes[b], ra);
                    if (lane == 0) {
                        S.dflag[warp] = 0u;
                        S.dhf[warp] = 0xFFFFFFFFu;
                    }
                }
            } else {
                decode_stage<kDelta, true>(p, t, TileView{S.vals, S.dcnt, S.dsum}, S.dbytes[b], ra);
            }
        }
        __syncthreads();   // count partials, decode partials and the prefix are in place
        long long pend_c = -1;
        unsigned int pend_old = 0;
        if (k < ntiles && warp == kWarps - 1) {
            if constexpr (kSeg)
                pend_old = count_publish_seg<kDelta>(p, k, S, lane);
            else
                pend_old = count_publish<kDelta>(p, k, S, lane);
            pend_c = static_cast<long long>(k / kChunk);
        }
        if (dec) {
            if constexpr (kSeg) {
                decode_emit_seg<kDelta>(p, S);
                if (dheads) check_heads(p, t, S, S.dbytes[b], dha, dhe, S.R0);
            } else {
                decode_emit<kDelta, kRank>(p, TileView{S.vals, S.dcnt, S.dsum}, S.R0, S.S0, ra,
                                           S.dbytes[b] + kHalo + warp * kWarpBytes);
            }
        }
        // did this count complete its chunk?  (read after the emission, so the
        // atomic has had time to return); the scan runs after the next barrier,
        // before any decode of this CTA waits
        if (warp == kWarps - 1 && lane == 0)
            S.scan_c = (pend_c >= 0 && static_cast<uint64_t>(pend_old) + 1 == chunk_tiles(p, pend_c)) ? pend_c : -1;
        if (tid == 0) S.tnext = knn;
#pragma unroll
        for (int j = 0; j < kStages - 2; ++j) q[j] = q[j + 1];
        q[kStages - 2] = kn;
    }
    __syncthreads();
    if (S.scan_c >= 0) chunk_scan<kSeg>(p, static_cast<uint64_t>(S.scan_c), S);
    cp_async_wait_all();
}


// ---- single pass: decoupled look-back, two tiles in flight per CTA
//
// Ticket k is tile k.  In each iteration a CTA stages (decodes into shared
// memory) the tile whose bytes it holds and publishes that tile's own value
// count and sum; then it resolves the prefix of the tile it staged in the
// previous iteration by looking back over earlier tiles' words -- one
// iteration after that tile's own words went out, so the tiles before it
// have usually published by then -- and writes that tile out.  The input is
// read from HBM once and every value is assembled once.  Every wait is on a
// tile with a smaller ticket, which a running CTA holds (its own words go out
// before its CTA waits on anything); each wait is bounded.
//
// Words (bit 0 = written; one 64-bit relaxed access each):
//   lagg[t]      sum << 32 | count << 1 | 1     tile t's own values (count <= 4096)
//   linc[2t]     count << 1 | 1                 values up to and including tile t
//   linc[2t+1]   x << 32 | 1                    running x after tile t

struct Shared1 {
    alignas(16) uint8_t bytes[2][kByteBuf];             // staged tiles: the one decoded now, the next
    alignas(16) uint32_t vals[2][kWarps][kWarpValBuf];  // staged values: this tile's, the previous one's
    uint32_t dcnt[2][kWarps], dsum[2][kWarps];          // per-warp totals of both
    unsigned long long R0[2];                           // values before the previous tile
    uint32_t S0[2];                                     // running x before it
    uint32_t tcur, tnext;                               // first tickets
};
static_assert(offsetof(Shared1, bytes) % 16 == 0 && offsetof(Shared1, vals) % 16 == 0, "Shared1 alignment");

// Warp 0: the values before tile t and the running x before it, from the
// words of earlier tiles, 32 at a time (lane i reads tile jb - i); then
// tile t's inclusive words.  Tiles before the stream act as one inclusive
// word with no values and x = prev.  After a timeout R0 = n (nothing is
// written) and tile t publishes nothing.
__device__ __forceinline__ void lookback(const Params &p, uint32_t t, uint32_t own_c, uint32_t own_s,
                                         unsigned long long *R0, uint32_t *S0)
{
    const int lane = threadIdx.x & 31;
    uint64_t cacc = 0;
    uint32_t sacc = 0;
    long long jb = static_cast<long long>(t) - 1;
    uint64_t t0 = 0;
    bool ok = true;
    for (int spin = 0;; ++spin) {
        const long long j = jb - lane;
        int kind = 0;   // 0: nothing published yet, 1: own words, 2: inclusive words
        uint64_t c = 0;
        uint32_t sv = 0;
        if (j < 0) {
            kind = 2;
            sv = p.prev;
        } else {
            const uint64_t ic = ld_relaxed_u64(p.linc + 2 * j);
            const uint64_t ix = ld_relaxed_u64(p.linc + 2 * j + 1);
            const uint64_t a = ld_relaxed_u64(p.lagg + j);
            if (ic & ix & 1u) {
                kind = 2;
                c = ic >> 1;
                sv = word_hi(ix);
            } else if (a & 1u) {
                kind = 1;
                c = desc_count(a);
                sv = word_hi(a);
            }
        }
        const uint32_t inc = __ballot_sync(~0u, kind == 2);
        const uint32_t upto = inc ? (inc ^ (inc - 1u)) : ~0u;   // lanes up to the nearest inclusive word
        if (__ballot_sync(~0u, kind == 0) & upto) {             // a word we need is not out yet
            int stop = 0;
            if (lane == 0) {
                const uint64_t now = global_ns();
                if (t0 == 0) t0 = now;
                if (now - t0 > p.wait_ns) {
                    atomicOr(p.status, VBYTE_ERR_TIMEOUT);
                    stop = 1;
                } else if (spin > 4) {
                    if (*reinterpret_cast<volatile uint32_t *>(p.status) & VBYTE_ERR_TIMEOUT) stop = 1;
                    __nanosleep(100);
                }
            }
            if (__shfl_sync(~0u, stop, 0)) {
                ok = false;
                break;
            }
            continue;
        }
        const bool mine = (upto >> lane) & 1u;
        sacc += __reduce_add_sync(~0u, mine ? sv : 0u);
        cacc += __reduce_add_sync(~0u, (mine && kind == 1) ? static_cast<uint32_t>(c) : 0u);
        if (inc) {
            const int k = __ffs(inc) - 1;
            const uint32_t lo = __shfl_sync(~0u, static_cast<uint32_t>(c), k);
            const uint32_t hi = __shfl_sync(~0u, static_cast<uint32_t>(c >> 32), k);
            cacc += (static_cast<uint64_t>(hi) << 32) | lo;
            break;
        }
        jb -= 32;
        spin = 0;
        t0 = 0;
    }
    if (lane == 0) {
        if (ok) {
            *R0 = cacc;
            *S0 = sacc;
            if (t != p.skip_tile) {
                st_relaxed_u64(p.linc + 2 * static_cast<uint64_t>(t) + 1,
                               (static_cast<uint64_t>(sacc + own_s) << 32) | 1u);
                st_relaxed_u64(p.linc + 2 * static_cast<uint64_t>(t), ((cacc + own_c) << 1) | 1u);
            }
            if (t == p.ntiles - 1 && cacc + own_c != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
        } else {
            *R0 = p.n;
            *S0 = 0u;
        }
    }
}

template <bool kDelta, bool kRank>
__global__ void __launch_bounds__(kThreads, 5) onepass_kernel(const Params p)
{
    __shared__ Shared1 S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ntiles = static_cast<uint32_t>(p.ntiles);   // tickets fit 32 bits (checked by the host)
    if (tid < 2) *reinterpret_cast<uint4 *>(S.bytes[tid] + kHalo + kTile) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        S.tcur = atomicAdd(p.ctr, 1u);
        S.tnext = atomicAdd(p.ctr, 1u);
    }
    __syncthreads();
    uint32_t cur = S.tcur, prev = 0xFFFFFFFFu;
    if (cur < ntiles) issue_stage(p, cur, tid, S.bytes[0]);
    cp_async_commit();
    RegA rp;
    rp.on = false;
    int b = 0;
    for (;;) {
        cp_async_wait_all();
        __syncthreads();   // cur's bytes are in S.bytes[b]; the previous iteration is over
        const uint32_t nx = S.tnext;
        const bool hc = cur < ntiles, hp = prev < ntiles;
        if (!hc && !hp) break;   // CTA-uniform
        uint32_t nnx = 0xFFFFFFFFu;
        if (tid == 0 && nx < ntiles) nnx = atomicAdd(p.ctr, 1u);
        if (nx < ntiles) issue_stage(p, nx, tid, S.bytes[b ^ 1]);
        cp_async_commit();
        const TileView vc{S.vals[b], S.dcnt[b], S.dsum[b]};
        const TileView vp{S.vals[b ^ 1], S.dcnt[b ^ 1], S.dsum[b ^ 1]};
        RegA rc;
        rc.on = false;
        if (hc) decode_stage<kDelta, true, true, true>(p, cur, vc, S.bytes[b], rc);
        __syncthreads();   // cur's per-warp totals are in place
        if (hc && warp == kWarps - 1) {
            const uint32_t tc = __reduce_add_sync(~0u, lane < kWarps ? vc.dcnt[lane] : 0u);
            const uint32_t ts = kDelta ? __reduce_add_sync(~0u, lane < kWarps ? vc.dsum[lane] : 0u) : 0u;
            if (lane == 0 && cur != p.skip_tile) st_relaxed_u64(p.lagg + cur, desc_word(tc, 0u, ts));
        }
        if (hp && warp == 0) {
            const uint32_t pc = __reduce_add_sync(~0u, lane < kWarps ? vp.dcnt[lane] : 0u);
            const uint32_t ps = kDelta ? __reduce_add_sync(~0u, lane < kWarps ? vp.dsum[lane] : 0u) : 0u;
            lookback(p, prev, pc, ps, &S.R0[b ^ 1], &S.S0[b ^ 1]);
        }
        __syncthreads();   // prev's prefix is in place
        if (hp)
            decode_emit<kDelta, kRank>(p, vp, S.R0[b ^ 1], S.S0[b ^ 1], rp,
                                       reinterpret_cast<const uint8_t *>(vp.vals[warp]) + 16);
        if (tid == 0) S.tnext = nnx;
        prev = cur;
        rp = rc;
        cur = nx;
        b ^= 1;
    }
    cp_async_wait_all();
}

// ---- host

// Workspace of one launch: status head, ticket counter, per chunk its
// totals words and counter, per tile a descriptor and a prefix word, and
// (batched lists) per tile a head range.  Everything before the head ranges
// is cleared before each launch.  Prefix words are read in 16-byte pairs; the
// padding after them covers the pair of an odd last tile.
struct Layout {
    size_t ctr, cnext, cdone, tdesc, tpre, hr, total, clear, total_b;
};

Layout layout(uint64_t ntiles)
{
    Layout L;
    const uint64_t nchunks = (ntiles + kChunk - 1) / kChunk;
    L.ctr = 256;   // after the status head
    L.cnext = L.ctr + 16;
    L.cdone = L.cnext + 16 * nchunks;
    L.tdesc = (L.cdone + 4 * nchunks + 15) / 16 * 16;
    L.tpre = (L.tdesc + 8 * ntiles + 15) / 16 * 16;   // 16-byte copies read it
    L.hr = (L.tpre + 8 * ntiles + 15) / 16 * 16;
    L.total = L.hr;
    L.clear = L.hr - L.ctr;
    L.total_b = L.hr + 16 * ntiles;
    return L;
}

// Workspace of a single-pass launch: status head, ticket counter, per tile its
// own word and two inclusive words; all but the head cleared before each
// launch.
struct Layout1 {
    size_t ctr, lagg, linc, total, clear;
};

Layout1 layout1(uint64_t ntiles)
{
    Layout1 L;
    L.ctr = 256;
    L.lagg = L.ctr + 16;
    L.linc = (L.lagg + 8 * ntiles + 15) / 16 * 16;
    L.total = L.linc + 16 * ntiles;
    L.clear = L.total - L.ctr;
    return L;
}

// Tiles [t_in_lo, t_in_hi) lie wholly inside [in, in + nbytes).
void inside_range(Params &p, uintptr_t in, size_t nbytes)
{
    p.t_in_lo = p.base == in ? 0u : 1u;
    p.t_in_hi = static_cast<uint32_t>((in + nbytes - p.base) / kTile);
}

// Tickets (tiles plus lead, plus those the CTAs draw past the end) are
// counted in 32 bits.
bool tickets_fit(uint64_t ntiles, uint64_t lead, uint64_t grid)
{
    return ntiles + lead + grid * (kStages + 1) < (1ull << 32);
}

// Every array read with 16-byte copies starts on a 16-byte boundary (the
// workspace itself is at least 256-byte aligned).
bool aligned(const Layout &L) { return ((L.cnext | L.tdesc | L.tpre | L.hr) & 15u) == 0; }

uint64_t tiles_for(uintptr_t addr, size_t nbytes) { return nbytes ? ((addr & 15u) + nbytes + kTile - 1) / kTile : 0; }

struct Dev {
    int sms = 0;
    int occ[2] = {0, 0};       // single stream: plain, delta
    int occ_seg[2] = {0, 0};   // batched lists: plain, delta
    int occ1[2] = {0, 0};      // single pass: plain, delta
};
std::mutex g_mu;
std::map<int, Dev> g_dev;

int dev_info(Dev *out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    Dev &d = g_dev[dev];
    if (d.sms == 0) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VBYTE_ECUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[0], sdecode_kernel<false, false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[1], sdecode_kernel<true, false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ_seg[0], sdecode_kernel<false, true>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ_seg[1], sdecode_kernel<true, true>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ1[0], onepass_kernel<false, false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ1[1], onepass_kernel<true, false>, kThreads, 0);
        for (int &o : d.occ) o = std::max(o, 1);
        for (int &o : d.occ_seg) o = std::max(o, 1);
        for (int &o : d.occ1) o = std::max(o, 1);
    }
    *out = d;
    return VBYTE_OK;
}

}  // namespace sd

size_t stream_workspace_bytes(const uint8_t *in, size_t nbytes)
{
    return sd::layout(sd::tiles_for(reinterpret_cast<uintptr_t>(in), nbytes)).total;
}

size_t stream_workspace_bytes_any(const uint8_t *in, size_t nbytes)
{
    const uint64_t ntiles = sd::tiles_for(reinterpret_cast<uintptr_t>(in), nbytes);
    return std::max({sd::layout(ntiles).total, sd::layout1(ntiles).total, split_workspace_bytes(in, nbytes)});
}

int launch_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                  cudaStream_t s, bool rank)
{
    if (nbytes == 0 && n == 0) return VBYTE_OK;
    if ((nbytes && !in) || (n && !out)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(out) & 3u) return VBYTE_EINVAL;
    uint8_t *ws = nullptr;
    const int rc = stream_workspace(s, stream_workspace_bytes_any(in, nbytes), &ws);
    if (rc != VBYTE_OK) return rc;
    uint32_t *status = reinterpret_cast<uint32_t *>(ws);
    if (nbytes == 0) return set_status_async(status, VBYTE_ERR_COUNT_MISMATCH, s);   // n > 0 from no bytes
    return enqueue_stream(in, nbytes, out, n, delta, prev, ws, status, s, rank, choose_passes(nbytes, n, delta));
}

// The single-pass kernel (decoupled look-back).
int enqueue_onepass(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                    uint8_t *ws, uint32_t *status, cudaStream_t s, bool rank)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    const uint64_t ntiles = sd::tiles_for(a, nbytes);
    const sd::Layout1 L = sd::layout1(ntiles);
    if (reinterpret_cast<uintptr_t>(ws) & 15u) return VBYTE_EINVAL;
    sd::Dev di;
    const int rc = sd::dev_info(&di);
    if (rc != VBYTE_OK) return rc;
    if (cudaMemsetAsync(ws + L.ctr, 0, L.clear, s) != cudaSuccess) return VBYTE_ECUDA;
    sd::Params p = {};
    p.in = in;
    p.nbytes = nbytes;
    p.out = out;
    p.n = n;
    p.ntiles = ntiles;
    p.base = a & ~static_cast<uintptr_t>(15);
    sd::inside_range(p, a, nbytes);
    p.ctr = reinterpret_cast<unsigned int *>(ws + L.ctr);
    p.lagg = reinterpret_cast<uint64_t *>(ws + L.lagg);
    p.linc = reinterpret_cast<uint64_t *>(ws + L.linc);
    p.status = status;
    p.prev = prev;
    const FaultCfg fc = fault_cfg();
    p.wait_ns = fc.wait_ns;
    p.skip_tile = fc.skip_tile;
    const uint64_t grid = std::min<uint64_t>(ntiles, static_cast<uint64_t>(di.sms) * di.occ1[delta]);
    if (ntiles + 3 * grid >= (1ull << 32)) return VBYTE_EINVAL;
    if (rank)
        sd::onepass_kernel<true, true><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    else if (delta)
        sd::onepass_kernel<true, false><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    else
        sd::onepass_kernel<false, false><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int enqueue_stream(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                   uint8_t *ws, uint32_t *status, cudaStream_t s, bool rank, int passes)
{
    if (rank && !delta) return VBYTE_EINVAL;
    if (passes == 1) return enqueue_onepass(in, nbytes, out, n, delta, prev, ws, status, s, rank);
    if (passes == 3) return enqueue_split(in, nbytes, out, n, delta, prev, ws, status, s, rank);
    if (passes == 4) return enqueue_split(in, nbytes, out, n, delta, prev, ws, status, s, rank, nullptr, !rank);
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    const uint64_t ntiles = sd::tiles_for(a, nbytes);
    const sd::Layout L = sd::layout(ntiles);
    if (!sd::aligned(L) || (reinterpret_cast<uintptr_t>(ws) & 15u)) return VBYTE_EINVAL;
    sd::Dev di;
    const int rc = sd::dev_info(&di);
    if (rc != VBYTE_OK) return rc;
    if (cudaMemsetAsync(ws + L.ctr, 0, L.clear, s) != cudaSuccess) return VBYTE_ECUDA;
    sd::Params p = {};
    p.in = in;
    p.nbytes = nbytes;
    p.out = out;
    p.n = n;
    p.ntiles = ntiles;
    p.base = a & ~static_cast<uintptr_t>(15);
    sd::inside_range(p, a, nbytes);
    p.tdesc = reinterpret_cast<uint64_t *>(ws + L.tdesc);
    p.tpre = reinterpret_cast<uint64_t *>(ws + L.tpre);
    p.cnext = reinterpret_cast<uint64_t *>(ws + L.cnext);
    p.cdone = reinterpret_cast<unsigned int *>(ws + L.cdone);
    p.ctr = reinterpret_cast<unsigned int *>(ws + L.ctr);
    p.status = status;
    p.prev = prev;
    p.lead = std::min<uint64_t>(sd::kChunk + sd::kSlack, ntiles);
    const FaultCfg fc = fault_cfg();
    p.wait_ns = fc.wait_ns;
    p.skip_tile = fc.skip_tile;
    const uint64_t grid = std::min<uint64_t>(ntiles + p.lead, static_cast<uint64_t>(di.sms) * di.occ[delta]);
    if (!sd::tickets_fit(ntiles, p.lead, grid)) return VBYTE_EINVAL;
    if (rank)
        sd::sdecode_kernel<true, false, true><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    else if (delta)
        sd::sdecode_kernel<true, false><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    else
        sd::sdecode_kernel<false, false><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

// ---- batched lists

size_t workspace_bound(size_t nbytes)
{
    const uint64_t ntiles = sd::tiles_for(15, nbytes);   // the worst alignment
    return std::max({sd::layout(ntiles).total_b, sd::layout1(ntiles).total, split_workspace_bound(nbytes)});
}

int load_kernels()
{
    sd::Dev di;
    return sd::dev_info(&di);
}

int sbatched_max_ctas(bool delta)
{
    sd::Dev di;
    return sd::dev_info(&di) == VBYTE_OK ? di.occ_seg[delta] : 1;
}

size_t sbatched_workspace_bytes(const BatchArgs &a)
{
    return sd::layout(sd::tiles_for(reinterpret_cast<uintptr_t>(a.in), a.nbytes)).total_b;
}

int enqueue_sbatched(const BatchArgs &a, uint8_t *ws, const LaunchCfg &cfg, cudaStream_t s)
{
    sd::Dev di;
    int rc = sd::dev_info(&di);
    if (rc != VBYTE_OK) return rc;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(a.in);
    const uint64_t ntiles = sd::tiles_for(addr, a.nbytes);
    const sd::Layout Y = sd::layout(ntiles);
    if (!sd::aligned(Y) || (reinterpret_cast<uintptr_t>(ws) & 15u)) return VBYTE_EINVAL;
    uint32_t *status = reinterpret_cast<uint32_t *>(ws);
    uint64_t *hr = reinterpret_cast<uint64_t *>(ws + Y.hr);
    rc = enqueue_head_ranges(a.in, a.nbytes, a.bo, a.vo, a.L, a.n, hr, status, di.sms, s);
    if (rc != VBYTE_OK) return rc;
    if (a.nbytes == 0) return a.n > 0 ? set_status_async(status, VBYTE_ERR_COUNT_MISMATCH, s) : VBYTE_OK;
    if (cudaMemsetAsync(ws + Y.ctr, 0, Y.clear, s) != cudaSuccess) return VBYTE_ECUDA;
    sd::Params p = {};
    p.in = a.in;
    p.nbytes = a.nbytes;
    p.out = a.out;
    p.n = a.n;
    p.ntiles = ntiles;
    p.base = addr & ~static_cast<uintptr_t>(15);
    sd::inside_range(p, addr, a.nbytes);
    p.tdesc = reinterpret_cast<uint64_t *>(ws + Y.tdesc);
    p.tpre = reinterpret_cast<uint64_t *>(ws + Y.tpre);
    p.cnext = reinterpret_cast<uint64_t *>(ws + Y.cnext);
    p.cdone = reinterpret_cast<unsigned int *>(ws + Y.cdone);
    p.ctr = reinterpret_cast<unsigned int *>(ws + Y.ctr);
    p.status = status;
    p.prev = 0u;
    p.lead = std::min<uint64_t>(sd::kChunk + cfg.lead_slack, ntiles);
    p.bo = a.bo;
    p.vo = a.vo;
    p.prevs = a.prevs;
    p.L = a.L;
    p.hr = hr;
    const FaultCfg fc = fault_cfg();
    p.wait_ns = fc.wait_ns;
    p.skip_tile = fc.skip_tile;
    const int occ = di.occ_seg[a.delta];
    const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, occ) : occ;
    const uint64_t grid = std::min<uint64_t>(ntiles + p.lead, static_cast<uint64_t>(di.sms) * per_sm);
    if (!sd::tickets_fit(ntiles, p.lead, grid)) return VBYTE_EINVAL;
    if (a.delta)
        sd::sdecode_kernel<true, true><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    else
        sd::sdecode_kernel<false, true><<<static_cast<unsigned>(grid), sd::kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace vbk
