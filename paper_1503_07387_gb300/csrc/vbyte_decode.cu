// libvbyte: GPU decoder for VByte-coded uint32 streams (sm_103a).
//
// Operation (arXiv 1503.07387): the result of Algorithm 1 (Sec. 2) on the
// byte stream -- seven data bits per byte, least significant group first,
// high bit set on every byte of an integer except its last (Sec. 1, Table 1)
// -- optionally followed by the prefix sum that undoes differential coding
// (Sec. 1 "Differential coding", Sec. 4 "Differential Coding").
//
// GPU design: count, then decode, chunk by chunk, with the input read from
// HBM once.
//   * The stream is cut into 4 KiB tiles aligned to 16 bytes in absolute
//     address space.  A tile owns exactly the integers whose terminator byte
//     (high bit clear) lies inside it; the 16 bytes before the tile are
//     staged too, so an integer that starts up to four bytes earlier is
//     assembled by the tile holding its terminator.
//   * Tiles are grouped into chunks of kChunkTiles (8 MiB).  Persistent CTAs
//     take tickets; ticket k counts tile k and, after the first chunk and a
//     slack, also decodes tile k - (kChunkTiles + kLeadSlack), so a tile is
//     decoded a little over one chunk after it was counted.
//   * (a) count: a CTA forms the terminator mask of its tile (the GPU
//     counterpart of pmovmskb, Sec. 3/4), its terminator count and, in delta
//     mode, the sum of its gaps; publishes both in the tile's descriptor and
//     adds them to its group's accumulators (32 tiles per group).  The CTA
//     that finishes a chunk last scans the chunk's group aggregates into
//     group prefixes and raises the chunk's ready flag.  This pass checks the
//     data-error contract.
//   * (b, c) decode: once its chunk is ready, a CTA's tile prefix is its
//     group prefix plus the aggregates of the earlier tiles of its group (one
//     L2 round trip).  It re-reads its tile -- from L2: the count read it one
//     chunk earlier -- and assembles every integer branch-free
//     from the (up to) five bytes ending at its terminator.  The work splits
//     by the longest code, the GPU counterpart of the paper's case split on
//     the 12-bit mask (Sec. 4): tiles of one-byte integers only (class A)
//     write their bytes straight out as values; codes of at most two bytes
//     use a SWAR byte-pair merge over 4-byte words; longer codes use
//     per-terminator assembly.  Values, prefix-summed in delta mode (uint32
//     wrap-around, seeded with `prev`), are staged in shared memory at their
//     rank shifted so that output quads are 16-byte aligned, and leave with
//     16-byte stores clamped to [0, n).
// The only waits are on chunk ready flags raised by CTAs holding earlier
// tickets (counting never waits, except a chunk's last CTA on the chunk
// before), so every wait ends; each is bounded by the global timer.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "vbyte.h"
#include "vbyte_internal.h"
#include "vbyte_device.cuh"

namespace vbk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = kThreads * kBPT;        // input bytes per tile (4 KiB)
constexpr int kRoundVals = kThreads * 4;      // values per copy-out round
constexpr int kGroup = 32;                    // tiles per group
constexpr uint64_t kChunkTiles = 2048;        // tiles per chunk (8 MiB)
constexpr int kGroupsPerChunk = static_cast<int>(kChunkTiles / kGroup);   // 64
constexpr int kByteBuf = kHalo + kTile + 16;
constexpr int kValBuf = kTile + 16;
constexpr uint64_t kLeadSlack = kDefaultLeadSlack;   // extra tickets between a chunk's last count and first decode
static_assert(kGroupsPerChunk <= kThreads && kGroupsPerChunk % 32 == 0, "chunk scan: one thread per group");

enum : uint32_t { kClassA = 0, kClassB = 1, kClassC = 2 };

struct Params {
    const uint8_t *in;
    uint64_t nbytes;
    uint32_t *out;
    uint64_t n;
    uint64_t ntiles;
    uintptr_t base;            // 16-byte aligned address of tile 0
    uint64_t *tdesc;           // per tile: count, gap sum
    unsigned long long *gagg;  // per group: count, gap sum (atomic accumulators)
    uint64_t *gpre;            // per group: exclusive prefix count, running x before it
    uint64_t *cnext;           // per chunk: prefix count and running x after it
    unsigned int *cdone;       // per chunk: CTAs that finished counting
    unsigned int *cready;      // per chunk: group prefixes published
    unsigned long long *ctr;   // work tickets
    uint32_t *status;          // data-error bits
    uint32_t prev;             // x_0 for differential decoding
    uint64_t lead;             // tickets [0, lead) only count; ticket k >= lead also decodes k - lead
    // segmented (batched) decoding only
    const uint64_t *bo;        // list byte offsets [L + 1], relative to in
    const uint64_t *vo;        // list value offsets [L + 1]
    const uint32_t *prevs;     // per-list x_0 (nullptr: 0)
    uint64_t L;                // number of lists
    const uint64_t *hr;        // per tile: [first, end) of the lists whose head may own a terminator in it
    uint64_t *tpre;            // per tile: values before it, running x before it
};

static_assert(kHeadTile == kTile, "head helpers assume 4 KiB tiles");

// Thread 0 waits until *flag != 0 (bounded by the global timer; on expiry the
// status word gets VBYTE_ERR_TIMEOUT and the caller carries on), then the CTA
// syncs.  The flag is set after __threadfence() by a CTA that holds a ticket
// taken before the waiter's, so the wait always ends.
__device__ __forceinline__ void wait_flag(const unsigned int *flag, uint32_t *status)
{
    if (threadIdx.x == 0) spin_flag(flag, status);
    __syncthreads();
}

// Stage tile t into `bytes`: bytes[16 + 16*tid ..] gets tid's 16-byte slice
// (zero bytes outside the stream), bytes[0..16) the 16 bytes before the tile
// (zero before tile 0, i.e. terminators of earlier, uncounted integers; for
// t > 0 they always lie inside the stream).  Whole slices travel with
// cp.async; the ragged first and last slices of the stream are loaded byte
// by byte.  The caller commits, waits for the copies and syncs the CTA.
__device__ __forceinline__ void issue_stage(const Params &p, uint64_t t, int tid, uint8_t *bytes)
{
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
    uint8_t *dst = bytes + kHalo + tid * kBPT;
    if (va >= lo && va + kBPT <= hi) {
        cp_async16(dst, reinterpret_cast<const void *>(va));
    } else {
        uint32_t wb[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const uintptr_t ad = va + j;
            if (ad >= lo && ad < hi)
                wb[j >> 2] |= static_cast<uint32_t>(*reinterpret_cast<const uint8_t *>(ad))
                              << (8 * (j & 3));
        }
        *reinterpret_cast<uint4 *>(dst) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
    }
    if (tid == 0) {
        if (t > 0)
            cp_async16(bytes, reinterpret_cast<const void *>(tstart - 16));
        else
            *reinterpret_cast<uint4 *>(bytes) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == kThreads - 1)
        *reinterpret_cast<uint4 *>(bytes + kHalo + kTile) = make_uint4(0u, 0u, 0u, 0u);
}

struct Shared {
    uint8_t cbytes[2][kByteBuf];     // staged tiles to count (double-buffered)
    uint8_t dbytes[2][kByteBuf];     // staged tiles to decode (double-buffered)
    uint32_t vals[kValBuf];          // decode: staged values at rank + sh
    uint32_t wcnt[kWarps];           // count: per-warp partials
    uint32_t wsum[kWarps];
    uint32_t dcnt[kWarps];           // decode: per-warp partials
    uint32_t dsum[kWarps];
    unsigned long long R0;           // decode: values before the tile
    uint32_t S0;                     // decode: running x before the tile
    unsigned long long gsc[kWarps];  // chunk scan: per-warp count totals
    uint32_t gss[kWarps];            // chunk scan: per-warp sum totals
    unsigned long long tnext;        // the ticket after the prefetched one
    unsigned long long pR0[2];       // prefetched tile prefixes (per buffer)
    uint32_t pS0[2];
    uint32_t pok[2];                 // prefetch valid
    // segmented decoding
    alignas(16) unsigned long long hrc[2][2];   // head ranges of the staged count tiles (cp.async targets)
    alignas(16) unsigned long long hrd[2][2];   // head ranges of the staged decode tiles
    HeadTab heads;                   // list heads of the tile being worked on
    uint32_t wsf[kWarps];            // count: per-warp "crossed a list head" flags
    uint32_t dsf[kWarps];            // decode: the same
    unsigned long long csc[kWarps];  // segmented chunk scan: per-warp count totals
    uint32_t css[kWarps], csf[kWarps];
};
// 16-byte cp.async and vector accesses need 16-byte aligned shared addresses
static_assert(offsetof(Shared, cbytes) % 16 == 0 && kByteBuf % 16 == 0, "cbytes alignment");
static_assert(offsetof(Shared, dbytes) % 16 == 0, "dbytes alignment");
static_assert(offsetof(Shared, vals) % 16 == 0, "vals alignment");
static_assert(offsetof(Shared, hrc) % 16 == 0 && offsetof(Shared, hrd) % 16 == 0, "head range alignment");

// --------------------------------------------------------------- counting --

template <bool kDelta, bool kSeg>
__device__ void count_tile(const Params &p, uint64_t t, Shared &S, const uint8_t *bytes, int b)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;

    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = tstart >= lo && tstart + kTile <= hi;
    const uint4 w0 = *reinterpret_cast<const uint4 *>(bytes + kHalo + tid * kBPT);
    const uint32_t wp0 = reinterpret_cast<const uint32_t *>(bytes)[(kHalo + tid * kBPT) / 4 - 1];
    uint32_t cnt, vsum = 0;
    if (interior && !((w0.x | w0.y | w0.z | w0.w) & 0x80808080u) && !(wp0 & 0x80000000u)) {
        // one-byte integers only
        cnt = kBPT;
        if (kDelta) vsum = byte_sum4(w0);
    } else {
        const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
        const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
        cnt = __popc(m.tc);
        // the data-error contract, checked once per byte here
        const uint32_t c20 = ~m.t20 & 0xFFFFFu;   // continuation bytes
        if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
            atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
        if (t == p.ntiles - 1 && hi - 1 >= va && hi - 1 < va + kBPT && !((m.tl >> (hi - 1 - va)) & 1u))
            atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        if (kDelta) {
            if (interior && !(c20 & (c20 << 1) & 0xFFFF8u)) {
                vsum = sum_le2_fast(m.w, m.wprev);
            } else {
                assemble_all(reinterpret_cast<const uint32_t *>(bytes), tid, m.tl, m.t20, m.tc,
                             [&](uint32_t v) { vsum += v; });
            }
        }
    }

    if constexpr (kSeg) {
        // batched: the tile's sum restarts at every list head it holds
        uint32_t segf = 0;
        if constexpr (kDelta) {
            const uint64_t ha = S.hrc[b][0], he = S.hrc[b][1];
            if (ha < he) {   // CTA-uniform
                const long long trel = static_cast<long long>(tstart) - static_cast<long long>(lo);
                build_heads(HeadSrc{p.bo, p.vo, p.prevs}, trel, ha, he, S.heads, true, false);
                const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
                const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
                const uint32_t *const sw = reinterpret_cast<const uint32_t *>(bytes);
                const HeadWin h = head_window(sw, S.heads.bits, tid, m.tl);
                const uint32_t ht = head_terms(h, m.tc);
                if (ht) {
                    segf = 1u;
                    vsum = slice_seg_sum(HeadSrc{p.bo, p.vo, p.prevs}, S.heads, sw, tid, m.tl, m.t20, m.tc, h, ht, trel + tid * kBPT, ha,
                                         he);
                }
            }
        }
        Seg sg;
        sg.f = segf;
        sg.s = vsum;
        sg = warp_seg_incl(sg, lane);
        const uint32_t wc = __reduce_add_sync(~0u, cnt);
        if (lane == 31) {
            S.wcnt[warp] = wc;
            S.wsum[warp] = sg.s;
            S.wsf[warp] = sg.f;
        }
        __syncthreads();
        if (warp == 0) {
            Seg ws;
            ws.f = lane < kWarps ? S.wsf[lane] : 0u;
            ws.s = lane < kWarps ? S.wsum[lane] : 0u;
            ws = warp_seg_incl(ws, lane);
            const uint32_t tcnt = __reduce_add_sync(~0u, lane < kWarps ? S.wcnt[lane] : 0u);
            if (lane == 31) {
                p.tdesc[2 * t] = tcnt;
                p.tdesc[2 * t + 1] = (static_cast<uint64_t>(ws.f) << 32) | ws.s;
                red_release_add(p.cdone + t / kChunkTiles, 1u);
            }
        }
        return;
    }

    const uint32_t wc = __reduce_add_sync(~0u, cnt);
    const uint32_t wsm = kDelta ? __reduce_add_sync(~0u, vsum) : 0u;
    if (lane == 0) {
        S.wcnt[warp] = wc;
        S.wsum[warp] = wsm;
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t cw = lane < kWarps ? S.wcnt[lane] : 0u;
        const uint32_t sw = lane < kWarps ? S.wsum[lane] : 0u;
        const uint32_t tcnt = __reduce_add_sync(~0u, cw);
        const uint32_t tsum = __reduce_add_sync(~0u, sw);
        if (lane == 0) {
            const uint64_t g = t / kGroup;
            p.tdesc[2 * t] = tcnt;
            p.tdesc[2 * t + 1] = tsum;
            atomicAdd(p.gagg + 2 * g, static_cast<unsigned long long>(tcnt));
            if (kDelta) atomicAdd(p.gagg + 2 * g + 1, static_cast<unsigned long long>(tsum));
            red_release_add(p.cdone + t / kChunkTiles, 1u);
        }
    }
}

// The group prefixes of chunk c, computed by the CTA that decodes the chunk's
// first tile: wait until every tile of the chunk has been counted and the
// chunk before has been scanned (both by CTAs holding earlier tickets), scan
// the chunk's group aggregates, publish, and raise the chunk's ready flag.
template <bool kDelta>
__device__ void chunk_scan(const Params &p, uint64_t c, Shared &S)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uint64_t c0 = c * kChunkTiles;
    const uint64_t c1 = (c0 + kChunkTiles < p.ntiles) ? c0 + kChunkTiles : p.ntiles;
    if (tid == 0) {
        uint64_t t0 = 0;
        for (int spin = 0;; ++spin) {
            unsigned int done;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(done) : "l"(p.cdone + c) : "memory");
            if (done >= static_cast<unsigned int>(c1 - c0)) break;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > kWaitLimitNs) {
                atomicOr(p.status, VBYTE_ERR_TIMEOUT);
                break;
            }
            if (spin > 4) __nanosleep(200);
        }
    }
    uint64_t pc = 0;
    uint32_t ps = p.prev;
    if (c > 0) {
        wait_flag(p.cready + (c - 1), p.status);
        pc = *reinterpret_cast<volatile uint64_t *>(p.cnext + 2 * (c - 1));
        ps = static_cast<uint32_t>(*reinterpret_cast<volatile uint64_t *>(p.cnext + 2 * (c - 1) + 1));
    } else {
        __syncthreads();
    }
    const uint64_t g0 = c * kGroupsPerChunk;
    const uint64_t ng = (p.ntiles + kGroup - 1) / kGroup;
    const uint64_t g = g0 + tid;
    uint64_t ac = 0;
    uint32_t as = 0;
    if (tid < kGroupsPerChunk && g < ng) {
        ac = *reinterpret_cast<volatile unsigned long long *>(p.gagg + 2 * g);
        as = static_cast<uint32_t>(*reinterpret_cast<volatile unsigned long long *>(p.gagg + 2 * g + 1));
    }
    const uint64_t ic = warp_incl_scan64(ac, lane);
    const uint32_t is = warp_incl_scan(as, lane);
    if (lane == 31) {
        S.gsc[warp] = ic;
        S.gss[warp] = is;
    }
    __syncthreads();
    uint64_t wc0 = 0, tc_all = 0;
    uint32_t ws0 = 0, ts_all = 0;
#pragma unroll
    for (int q = 0; q < kGroupsPerChunk / 32; ++q) {
        wc0 += (q < warp) ? S.gsc[q] : 0ull;
        ws0 += (q < warp) ? S.gss[q] : 0u;
        tc_all += S.gsc[q];
        ts_all += S.gss[q];
    }
    if (tid < kGroupsPerChunk && g < ng) {
        p.gpre[2 * g] = pc + wc0 + ic - ac;
        p.gpre[2 * g + 1] = static_cast<uint32_t>(ps + ws0 + is - as);
    }
    __syncthreads();
    if (tid == 0) {
        p.cnext[2 * c] = pc + tc_all;
        p.cnext[2 * c + 1] = static_cast<uint32_t>(ps + ts_all);
        if (c1 == p.ntiles && pc + tc_all != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
        __threadfence();
        *reinterpret_cast<volatile unsigned int *>(p.cready + c) = 1u;
    }
    __syncthreads();
}

// Batched form: the per-tile prefixes of chunk c, computed from the tile
// descriptors by the CTA that decodes the chunk's first tile (same waits as
// chunk_scan).  Each thread scans eight consecutive tiles; the running value
// restarts at list heads (segmented sums).
template <bool kDelta>
__device__ void chunk_scan_seg(const Params &p, uint64_t c, Shared &S)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    constexpr int kPer = static_cast<int>(kChunkTiles / kThreads);   // 8
    const uint64_t c0 = c * kChunkTiles;
    const uint64_t c1 = (c0 + kChunkTiles < p.ntiles) ? c0 + kChunkTiles : p.ntiles;
    if (tid == 0) {
        uint64_t t0 = 0;
        for (int spin = 0;; ++spin) {
            if (ld_acquire_u32(p.cdone + c) >= static_cast<unsigned int>(c1 - c0)) break;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > kWaitLimitNs) {
                atomicOr(p.status, VBYTE_ERR_TIMEOUT);
                break;
            }
            if (spin > 4) __nanosleep(200);
        }
    }
    uint64_t pc = 0;
    uint32_t ps = 0;
    if (c > 0) {
        wait_flag(p.cready + (c - 1), p.status);
        pc = __ldcg(reinterpret_cast<const unsigned long long *>(p.cnext + 2 * (c - 1)));
        ps = static_cast<uint32_t>(__ldcg(reinterpret_cast<const unsigned long long *>(p.cnext + 2 * (c - 1) + 1)));
    } else {
        __syncthreads();
    }
    const uint64_t tb = c0 + static_cast<uint64_t>(kPer) * tid;
    uint64_t cn[kPer];
    Seg sg[kPer];
    uint64_t tcn = 0;
    Seg ts;
    ts.f = 0u;
    ts.s = 0u;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        cn[i] = 0;
        sg[i].f = 0u;
        sg[i].s = 0u;
        if (tb + i < c1) {
            const ulonglong2 d = __ldcg(reinterpret_cast<const ulonglong2 *>(p.tdesc + 2 * (tb + i)));
            cn[i] = d.x;
            sg[i].f = static_cast<uint32_t>(d.y >> 32);
            sg[i].s = static_cast<uint32_t>(d.y);
        }
        tcn += cn[i];
        ts = seg_op(ts, sg[i]);
    }
    const uint64_t icn = warp_incl_scan64(tcn, lane);
    const Seg is = warp_seg_incl(ts, lane);
    if (lane == 31) {
        S.csc[warp] = icn;
        S.css[warp] = is.s;
        S.csf[warp] = is.f;
    }
    __syncthreads();
    uint64_t wc0 = 0, call = 0;
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
    // state before my first tile: chunk start, earlier warps, earlier lanes
    Seg ex;
    ex.f = __shfl_up_sync(~0u, is.f, 1);
    ex.s = __shfl_up_sync(~0u, is.s, 1);
    if (lane == 0) ex.f = ex.s = 0u;
    uint64_t rc = pc + wc0 + icn - tcn;
    uint32_t x = seg_apply(ps, seg_op(w0, ex));
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        if (tb + i < c1) {
            *reinterpret_cast<ulonglong2 *>(p.tpre + 2 * (tb + i)) = make_ulonglong2(rc, x);
        }
        rc += cn[i];
        x = seg_apply(x, sg[i]);
    }
    __syncthreads();
    if (tid == 0) {
        p.cnext[2 * c] = pc + call;
        p.cnext[2 * c + 1] = seg_apply(ps, wall);
        if (c1 == p.ntiles && pc + call != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
        __threadfence();
        *reinterpret_cast<volatile unsigned int *>(p.cready + c) = 1u;
    }
    __syncthreads();
}

// --------------------------------------------------------------- decoding --

// Warp 0's loads of a tile's prefix: the group prefix (lane 0) and the
// aggregates of the earlier tiles of the group (one per lane).
struct PrefixLoads {
    uint64_t pa, pb, ga, gb;
    bool ok;   // loaded after the tile's chunk was seen ready (warp-uniform)
};

template <bool kSeg>
__device__ __forceinline__ PrefixLoads load_prefix(const Params &p, uint64_t t, int lane)
{
    PrefixLoads r;
    r.pa = r.pb = r.ga = r.gb = 0;
    r.ok = true;
    if constexpr (kSeg) {   // the chunk scan wrote the tile's own prefix
        if (lane == 0) {
            const ulonglong2 d = __ldcg(reinterpret_cast<const ulonglong2 *>(p.tpre + 2 * t));
            r.ga = d.x;
            r.gb = d.y;
        }
        return r;
    }
    const uint64_t g = t / kGroup;
    const uint64_t j = g * kGroup + lane;
    if (j < t) {
        r.pa = *reinterpret_cast<const volatile uint64_t *>(p.tdesc + 2 * j);
        r.pb = *reinterpret_cast<const volatile uint64_t *>(p.tdesc + 2 * j + 1);
    }
    if (lane == 0) {
        r.ga = *reinterpret_cast<const volatile uint64_t *>(p.gpre + 2 * g);
        r.gb = *reinterpret_cast<const volatile uint64_t *>(p.gpre + 2 * g + 1);
    }
    return r;
}

// Warp 0: if tile t's chunk is already published (and t is not the chunk's
// first tile, whose CTA scans the chunk), issue its prefix loads now, to be
// consumed an iteration later.
template <bool kSeg>
__device__ __forceinline__ PrefixLoads try_prefetch_prefix(const Params &p, uint64_t t, int lane)
{
    PrefixLoads r;
    r.pa = r.pb = r.ga = r.gb = 0;
    r.ok = false;
    if (t >= p.ntiles || t % kChunkTiles == 0) return r;
    unsigned int ready = 0;
    if (lane == 0) ready = ld_acquire_u32(p.cready + t / kChunkTiles);
    ready = __shfl_sync(~0u, ready, 0);   // the warp sync orders lane 0's acquire before the loads
    if (!ready) return r;
    return load_prefix<kSeg>(p, t, lane);
}

template <bool kDelta, bool kSeg>
__device__ void decode_tile(const Params &p, uint64_t t, Shared &S, const uint8_t *bytes, int b)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);

    // tile prefix: group prefix + the earlier tiles of the group, once the
    // chunk's group prefixes are published -- usually prefetched an iteration
    // ago into S.pR0 / S.pS0; otherwise warp 0 loads it now and folds it into
    // S.R0 / S.S0 before the CTA's second barrier.
    PrefixLoads pre;
    pre.pa = pre.pb = pre.ga = pre.gb = 0;
    const bool prefetched = S.pok[b] != 0u && t % kChunkTiles != 0;
    if (t % kChunkTiles == 0) {
        if constexpr (kSeg)
            chunk_scan_seg<kDelta>(p, t / kChunkTiles, S);
        else
            chunk_scan<kDelta>(p, t / kChunkTiles, S);
        if (warp == 0) pre = load_prefix<kSeg>(p, t, lane);
    } else if (warp == 0 && !prefetched) {
        if (lane == 0) spin_flag(p.cready + t / kChunkTiles, p.status);
        __syncwarp();
        pre = load_prefix<kSeg>(p, t, lane);
    }
    auto fold_prefix = [&]() {
        if (warp == 0) {
            if (prefetched) {
                if (lane == 0) {
                    S.R0 = S.pR0[b];
                    S.S0 = S.pS0[b];
                }
            } else {
                const uint64_t ec = warp_sum64(pre.pa);
                const uint64_t es = warp_sum64(pre.pb & 0xFFFFFFFFull);
                if (lane == 0) {
                    S.R0 = pre.ga + ec;
                    S.S0 = static_cast<uint32_t>(pre.gb + es);
                }
            }
        }
    };

    const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
    const bool interior = tstart >= lo && tstart + kTile <= hi;
    const uint4 w0 = *reinterpret_cast<const uint4 *>(bytes + kHalo + tid * kBPT);
    const uint32_t wp0 = reinterpret_cast<const uint32_t *>(bytes)[(kHalo + tid * kBPT) / 4 - 1];
    bool mineA = interior && !((w0.x | w0.y | w0.z | w0.w) & 0x80808080u) && !(wp0 & 0x80000000u);
    uint64_t ha = 0, he = 0;
    if constexpr (kSeg) {
        ha = S.hrd[b][0];
        he = S.hrd[b][1];
        if (ha < he) mineA = false;   // tiles with list heads take the general path
    }

    if (!__syncthreads_or(!mineA)) {
        // ---- class A: every byte is a one-byte integer; tile rank 16*tid + i is
        // my byte i.  I rebuild the 3 values before my bytes as well, so every
        // aligned output quad that starts among my ranks is complete here.
        uint32_t base = 0;
        uint32_t mine = 0, incs = 0;
        if (kDelta) {
            mine = byte_sum4(w0);
            incs = warp_incl_scan(mine, lane);
            if (lane == 31) S.dsum[warp] = incs;
        }
        fold_prefix();
        __syncthreads();
        if (kDelta) {
            uint32_t wsbase = 0;
#pragma unroll
            for (int q = 0; q < kWarps; ++q) wsbase += (q < warp) ? S.dsum[q] : 0u;
            base = S.S0 + wsbase + incs - mine;
        }
        const unsigned long long R0 = S.R0;
        const uint32_t sh = (out_word + static_cast<uint32_t>(R0)) & 3u;
        uint32_t v[19];
        const uint4 q0 = bytes_as_values(w0.x), q1 = bytes_as_values(w0.y);
        const uint4 q2 = bytes_as_values(w0.z), q3 = bytes_as_values(w0.w);
        v[3] = q0.x; v[4] = q0.y; v[5] = q0.z; v[6] = q0.w;
        v[7] = q1.x; v[8] = q1.y; v[9] = q1.z; v[10] = q1.w;
        v[11] = q2.x; v[12] = q2.y; v[13] = q2.z; v[14] = q2.w;
        v[15] = q3.x; v[16] = q3.y; v[17] = q3.z; v[18] = q3.w;
        const uint4 pv = bytes_as_values(wp0);   // pv.y, pv.z, pv.w: ranks -3, -2, -1
        if (kDelta) {
            v[2] = base;
            v[1] = base - pv.w;
            v[0] = v[1] - pv.z;
            uint32_t run = base;
#pragma unroll
            for (int i = 3; i < 19; ++i) {
                run += v[i];
                v[i] = run;
            }
        } else {
            v[0] = pv.y;
            v[1] = pv.z;
            v[2] = pv.w;
        }
        const long long gq = static_cast<long long>(R0) - sh + 16 * tid;   // output rank of my first quad
        const int kq = 16 * tid - static_cast<int>(sh);                    // tile rank of it
        const bool whole = tid > 0 && gq + 20 <= static_cast<long long>(p.n);
        auto put = [&](int j, uint32_t e0, uint32_t e1, uint32_t e2, uint32_t e3) {
            const int k0 = kq + 4 * j;
            const long long g0 = gq + 4 * j;
            if ((whole && j < 4) ||
                (k0 >= 0 && k0 + 4 <= kTile && g0 + 4 <= static_cast<long long>(p.n))) {
                st_quad(p.out + g0, make_uint4(e0, e1, e2, e3));
            } else {
                const uint32_t e4[4] = {e0, e1, e2, e3};
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
                    if (k0 + mm >= 0 && k0 + mm < kTile && g0 + mm < static_cast<long long>(p.n))
                        p.out[g0 + mm] = e4[mm];
            }
        };
        const bool tail = tid == kThreads - 1 && sh != 0u;
        switch (sh) {
        case 0:
            put(0, v[3], v[4], v[5], v[6]);
            put(1, v[7], v[8], v[9], v[10]);
            put(2, v[11], v[12], v[13], v[14]);
            put(3, v[15], v[16], v[17], v[18]);
            break;
        case 1:
            put(0, v[2], v[3], v[4], v[5]);
            put(1, v[6], v[7], v[8], v[9]);
            put(2, v[10], v[11], v[12], v[13]);
            put(3, v[14], v[15], v[16], v[17]);
            if (tail) put(4, v[18], 0u, 0u, 0u);
            break;
        case 2:
            put(0, v[1], v[2], v[3], v[4]);
            put(1, v[5], v[6], v[7], v[8]);
            put(2, v[9], v[10], v[11], v[12]);
            put(3, v[13], v[14], v[15], v[16]);
            if (tail) put(4, v[17], v[18], 0u, 0u);
            break;
        default:
            put(0, v[0], v[1], v[2], v[3]);
            put(1, v[4], v[5], v[6], v[7]);
            put(2, v[8], v[9], v[10], v[11]);
            put(3, v[12], v[13], v[14], v[15]);
            if (tail) put(4, v[16], v[17], v[18], 0u);
            break;
        }
        return;
    }

    // ---- general tiles: ranks and (delta) gap offsets by block scans
    const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;
    const uint32_t *const sw = reinterpret_cast<const uint32_t *>(bytes);
    const SliceMasks m = slice_masks(bytes, tid, interior, va, lo, hi);
    uint32_t cnt, vsum;
    bool notB;
    slice_count_sum<kDelta>(m, sw, tid, interior, cnt, vsum, notB);
    const long long trel = static_cast<long long>(tstart) - static_cast<long long>(lo);
    const long long srel = trel + tid * kBPT;
    HeadWin hw;
    hw.t24 = hw.h24 = 0u;
    uint32_t ht = 0;
    if constexpr (kSeg) {
        if (ha < he) {   // CTA-uniform
            build_heads(HeadSrc{p.bo, p.vo, p.prevs}, trel, ha, he, S.heads, kDelta, true);
            hw = head_window(sw, S.heads.bits, tid, m.tl);
            if constexpr (kDelta) {
                ht = head_terms(hw, m.tc);
                if (ht) {
                    vsum = slice_seg_sum(HeadSrc{p.bo, p.vo, p.prevs}, S.heads, sw, tid, m.tl, m.t20, m.tc, hw, ht, srel, ha, he);
                    notB = true;   // values with restarts take the per-terminator path
                }
            }
        }
    }
    const uint32_t inc = warp_incl_scan(cnt, lane);
    Seg isg;
    isg.f = ht ? 1u : 0u;
    isg.s = vsum;
    if constexpr (kSeg && kDelta) {
        isg = warp_seg_incl(isg, lane);
    } else if constexpr (kDelta) {
        isg.s = warp_incl_scan(vsum, lane);
    }
    if (lane == 31) {
        S.dcnt[warp] = inc;
        S.dsum[warp] = isg.s;
        if constexpr (kSeg) S.dsf[warp] = isg.f;
    }
    fold_prefix();
    __syncthreads();
    uint32_t wbase = 0, wsbase = 0, tcnt = 0;
    Seg wseg;
    wseg.f = wseg.s = 0u;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
        const uint32_t c = S.dcnt[q];
        wbase += (q < warp) ? c : 0u;
        if constexpr (kSeg && kDelta) {
            if (q < warp) {
                Seg e;
                e.f = S.dsf[q];
                e.s = S.dsum[q];
                wseg = seg_op(wseg, e);
            }
        } else if constexpr (kDelta) {
            wsbase += (q < warp) ? S.dsum[q] : 0u;
        }
        tcnt += c;
    }
    const unsigned long long R0 = S.R0;
    const uint32_t sh = (out_word + static_cast<uint32_t>(R0)) & 3u;

    if constexpr (kSeg) {
        // each list head in my slice: its first integer's rank must be vo[j],
        // and the byte before it must end the previous list's last integer
        const uint32_t hs = (hw.h24 >> kHeadBack) & 0xFFFFu;
        if (hs) {
            uint32_t mm = hs;
            while (mm) {
                const int k = __ffs(mm) - 1;
                mm &= mm - 1u;
                const long long pos = srel + k;
                if (pos < 0 || pos >= static_cast<long long>(p.nbytes)) continue;
                if (pos > 0 && !((hw.t24 >> (kHeadBack + k - 1)) & 1u)) atomicOr(p.status, VBYTE_ERR_TRUNCATED);
                const uint64_t rank = R0 + wbase + inc - cnt + __popc(m.tc & ((1u << k) - 1u));
                if (he - ha <= static_cast<uint64_t>(kMaxHeadList)) {
                    const int qs = kHalo + tid * kBPT + k;
                    for (int i = tab_last_le(S.heads, static_cast<int>(he - ha), qs); i >= 0; --i) {
                        if (S.heads.pos[i] != qs) break;
                        if (S.heads.vo[i] != rank) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
                    }
                } else {
                    for (long long j = last_list_at(HeadSrc{p.bo, p.vo, p.prevs}, ha, he, pos); j >= static_cast<long long>(ha); --j) {
                        if (static_cast<long long>(p.bo[j]) != pos) break;
                        if (p.vo[j] != rank) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
                    }
                }
            }
        }
    }

    // assemble my values into vals[sh + rank], prefix-summed in delta mode
    uint32_t *dst = S.vals + sh + wbase + inc - cnt;
    uint32_t run = 0u;
    if constexpr (kSeg && kDelta) {
        Seg ex;
        ex.f = __shfl_up_sync(~0u, isg.f, 1);
        ex.s = __shfl_up_sync(~0u, isg.s, 1);
        if (lane == 0) ex.f = ex.s = 0u;
        run = seg_apply(S.S0, seg_op(wseg, ex));
    } else if constexpr (kDelta) {
        run = S.S0 + wsbase + isg.s - vsum;
    }
    const bool warp_le2 = !__any_sync(~0u, notB);
    if (ht) {
        assemble_all_o(sw, tid, m.tl, m.t20, m.tc, [&](int o, uint32_t v) {
            if ((ht >> o) & 1u)
                run = head_prev(HeadSrc{p.bo, p.vo, p.prevs}, S.heads, hw, o, tid, srel, ha, he) + v;
            else
                run += v;
            *dst++ = run;
        });
    } else if (warp_le2) {
        const uint32_t c4[4] = {m.w.x, m.w.y, m.w.z, m.w.w};
        uint32_t wp = m.wprev;
        int q = 0;
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
                        dst[q++] = run;
                    } else {
                        dst[q++] = v4[i];
                    }
                }
            }
            wp = c4[j];
        }
    } else {
        assemble_all(sw, tid, m.tl, m.t20, m.tc, [&](uint32_t v) {
            if (kDelta) {
                run += v;
                *dst++ = run;
            } else {
                *dst++ = v;
            }
        });
    }
    __syncthreads();

    // copy-out: staging index 4i maps to a 16-byte aligned output address
    const uint32_t lim = sh + tcnt;   // staged indices [sh, lim)
    const long long rho0 = static_cast<long long>(R0) - sh;
    for (uint32_t idx = 4 * tid; idx < lim; idx += kRoundVals) {
        const uint4 o = *reinterpret_cast<const uint4 *>(S.vals + idx);
        const long long g0 = rho0 + idx;
        if (idx >= sh && idx + 4 <= lim && g0 + 4 <= static_cast<long long>(p.n)) {
            st_quad(p.out + g0, o);
        } else {
            const uint32_t e4[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (idx + j >= sh && idx + j < lim && g0 + j < static_cast<long long>(p.n))
                    p.out[g0 + j] = e4[j];
        }
    }
}

// ----------------------------------------------------------------- kernel --
//
// Persistent CTAs take tickets.  Ticket k counts tile k and, from ticket
// `lead` (one chunk plus kLeadSlack) on, also decodes tile k - lead, whose
// chunk was counted by tickets at least kLeadSlack earlier: a tile is read
// from HBM by its count and again, about 12 MiB of input later, from L2 by
// its decode.

template <bool kDelta, bool kSeg>
__global__ void __launch_bounds__(kThreads, 4) decode_kernel(const Params p)
{
    __shared__ __align__(16) Shared S;
    const int tid = threadIdx.x;
    const uint64_t total = p.ntiles + p.lead;
    // Tickets run two ahead: while ticket k is processed, the tiles of the next
    // ticket are in flight to the other buffers and the one after is taken.
    if (tid == 0) {
        S.R0 = atomicAdd(p.ctr, 1ull);
        S.tnext = atomicAdd(p.ctr, 1ull);
    }
    __syncthreads();
    uint64_t k = S.R0;
    uint64_t kn = S.tnext;
    auto stage = [&](uint64_t tk, int b) {
        if (tk < p.ntiles) issue_stage(p, tk, tid, S.cbytes[b]);
        if (tk >= p.lead && tk < total) issue_stage(p, tk - p.lead, tid, S.dbytes[b]);
        if constexpr (kSeg) {   // the tiles' list-head ranges travel with them
            if (kDelta && tid == 32 && tk < p.ntiles) cp_async16(S.hrc[b], p.hr + 2 * tk);
            if (tid == 64 && tk >= p.lead && tk < total) cp_async16(S.hrd[b], p.hr + 2 * (tk - p.lead));
        }
        cp_async_commit();
    };
    stage(k, 0);
    if (tid == 0) S.pok[0] = 0u;
    const int warp = tid >> 5, lane = tid & 31;
    for (int b = 0; k < total; b ^= 1) {
        unsigned long long knn = 0;
        if (tid == 0) knn = atomicAdd(p.ctr, 1ull);
        stage(kn, b ^ 1);
        // warp 0 issues the prefix loads of kn's decode tile now (if its chunk is
        // ready) and folds them into S.pR0 / S.pS0 at the end of the iteration
        PrefixLoads pn;
        pn.pa = pn.pb = pn.ga = pn.gb = 0;
        pn.ok = false;
        if (warp == 0 && kn >= p.lead && kn < total) pn = try_prefetch_prefix<kSeg>(p, kn - p.lead, lane);
        cp_async_wait_prior();
        __syncthreads();   // ticket k's tiles are staged
        if (k < p.ntiles) count_tile<kDelta, kSeg>(p, k, S, S.cbytes[b], b);
        if (k >= p.lead) decode_tile<kDelta, kSeg>(p, k - p.lead, S, S.dbytes[b], b);
        if (warp == 0) {
            const uint64_t ec = warp_sum64(pn.pa);
            const uint64_t es = warp_sum64(pn.pb & 0xFFFFFFFFull);
            if (lane == 0) {
                S.pR0[b ^ 1] = pn.ga + ec;
                S.pS0[b ^ 1] = static_cast<uint32_t>(pn.gb + es);
                S.pok[b ^ 1] = pn.ok ? 1u : 0u;
                S.tnext = knn;
            }
        }
        __syncthreads();   // buffers b are free; the next ticket is known
        k = kn;
        kn = S.tnext;
    }
    cp_async_wait_all();
}

__global__ void set_status_kernel(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// Batched form, before the decode: for every tile, the range [first, end) of
// list indices whose byte offset lies in [tile start - kHeadBack, tile end)
// (binary searches over bo), and the offset arrays' contract: bo and vo
// non-decreasing from 0 to nbytes and n; a list that starts at the end of the
// bytes holds no values.
__device__ __forceinline__ uint64_t lower_bound_bo(const uint64_t *bo, uint64_t L, long long x)
{
    if (x <= 0) return 0;
    uint64_t lo = 0, hi = L + 1;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (static_cast<long long>(bo[mid]) < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) head_range_kernel(const Params p)
{
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long long in0 = static_cast<long long>(reinterpret_cast<uintptr_t>(p.in));
    uint64_t *hr = const_cast<uint64_t *>(p.hr);
    for (uint64_t t = i0; t < p.ntiles; t += stride) {
        const long long trel = static_cast<long long>(p.base + t * kTile) - in0;
        uint64_t a = lower_bound_bo(p.bo, p.L, trel - kHeadBack);
        uint64_t e = lower_bound_bo(p.bo, p.L, trel + kTile);
        if (e > p.L) e = p.L;
        if (a > e) a = e;
        *reinterpret_cast<ulonglong2 *>(hr + 2 * t) = make_ulonglong2(a, e);
    }
    uint32_t bad = 0;
    for (uint64_t j = i0; j < p.L; j += stride) {
        if (p.bo[j] > p.bo[j + 1] || p.vo[j] > p.vo[j + 1]) bad |= VBYTE_ERR_BAD_OFFSETS;
        if (p.bo[j] == p.nbytes && p.vo[j] != p.n) bad |= VBYTE_ERR_COUNT_MISMATCH;
    }
    if (i0 == 0 && (p.bo[0] != 0 || p.vo[0] != 0 || p.bo[p.L] != p.nbytes || p.vo[p.L] != p.n))
        bad |= VBYTE_ERR_BAD_OFFSETS;
    if (bad) atomicOr(p.status, bad);
}

// Launch head_range_kernel for a batch decoded by another kernel with the
// same 4 KiB tiling (tile 0 at `in` rounded down to 16 bytes).
int enqueue_head_ranges(const uint8_t *in, size_t nbytes, const uint64_t *bo, const uint64_t *vo, size_t L,
                        size_t n, uint64_t *hr, uint32_t *status, int sms, cudaStream_t s)
{
    Params p = {};
    p.in = in;
    p.nbytes = nbytes;
    p.n = n;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    p.ntiles = nbytes ? ((a & 15u) + nbytes + kTile - 1) / kTile : 0;
    p.base = a & ~static_cast<uintptr_t>(15);
    p.bo = bo;
    p.vo = vo;
    p.L = L;
    p.hr = hr;
    p.status = status;
    const uint64_t work = std::max<uint64_t>(p.ntiles, L);
    const unsigned grid = static_cast<unsigned>(std::min<uint64_t>((work + 255) / 256, static_cast<uint64_t>(sms) * 8));
    head_range_kernel<<<std::max(grid, 1u), 256, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

// ------------------------------------------------------------- workspace --

// Workspace layout: [0,4) status word; [256, ...) the ticket counter, per
// chunk two words of cnext and one each of cdone and cready, then per group
// two words of gagg and two of gpre, then per tile two words of tdesc.  All
// but gpre and tdesc (written before they are read) is cleared before each
// decode.
constexpr size_t kWsHead = 256;

struct Workspace {
    uint8_t *ptr = nullptr;
    size_t cap = 0;
};

struct HostBuffers {
    uint8_t *d_in = nullptr;
    size_t cap_in = 0;
    uint32_t *d_out = nullptr;
    size_t cap_out = 0;
};

std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, Workspace> g_ws;
std::map<std::pair<int, uintptr_t>, HostBuffers> g_hb;

struct Layout {
    uint64_t ntiles, ngroups, nchunks;
    size_t ctr, cnext, cdone, cready, gagg, gpre, tdesc, total, clear;
};

Layout layout(uint64_t ntiles)
{
    Layout L;
    L.ntiles = ntiles;
    L.ngroups = (ntiles + kGroup - 1) / kGroup;
    L.nchunks = (ntiles + kChunkTiles - 1) / kChunkTiles;
    L.ctr = kWsHead;
    L.cnext = L.ctr + 16;
    L.cdone = L.cnext + 16 * L.nchunks;
    L.cready = L.cdone + 4 * L.nchunks;
    L.gagg = (L.cready + 4 * L.nchunks + 15) / 16 * 16;
    L.gpre = L.gagg + 16 * L.ngroups;
    L.tdesc = L.gpre + 16 * L.ngroups;
    L.total = L.tdesc + 16 * ntiles;
    L.clear = L.gpre - L.ctr;   // ticket counter, chunk words and gagg
    return L;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

// Returns the workspace of (current device, s) with at least `need` bytes.
int get_workspace(cudaStream_t s, size_t need, Workspace **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &w = g_ws[{dev, reinterpret_cast<uintptr_t>(s)}];
    if (w.cap < need) {
        if (capturing(s)) return VBYTE_ENOMEM;
        size_t cap = std::max<size_t>(need, std::max<size_t>(2 * w.cap, size_t(1) << 20));
        void *np = nullptr;
        if (cudaMallocAsync(&np, cap, s) != cudaSuccess) {
            cudaGetLastError();
            return VBYTE_ENOMEM;
        }
        if (w.ptr) {
            cudaMemcpyAsync(np, w.ptr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
            cudaFreeAsync(w.ptr, s);
        } else {
            cudaMemsetAsync(np, 0, sizeof(uint32_t), s);
        }
        w.ptr = static_cast<uint8_t *>(np);
        w.cap = cap;
    }
    *out = &w;
    return VBYTE_OK;
}

// Batched workspace: after the single-stream head, ticket counter and chunk
// words, per tile two words of tdesc, two of tpre and two of hr.
struct LayoutSeg {
    uint64_t ntiles, nchunks;
    size_t ctr, cnext, cdone, cready, tdesc, tpre, hr, total, clear;
};

LayoutSeg layout_seg(uint64_t ntiles)
{
    LayoutSeg L;
    L.ntiles = ntiles;
    L.nchunks = (ntiles + kChunkTiles - 1) / kChunkTiles;
    L.ctr = kWsHead;
    L.cnext = L.ctr + 16;
    L.cdone = L.cnext + 16 * L.nchunks;
    L.cready = L.cdone + 4 * L.nchunks;
    L.tdesc = (L.cready + 4 * L.nchunks + 15) / 16 * 16;
    L.tpre = L.tdesc + 16 * ntiles;
    L.hr = L.tpre + 16 * ntiles;
    L.total = L.hr + 16 * ntiles;
    L.clear = L.tdesc - L.ctr;   // ticket counter and chunk words
    return L;
}

std::map<int, DeviceInfo> g_dev;

int device_info(DeviceInfo *di)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo &d = g_dev[dev];
    if (d.sms == 0) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return VBYTE_ECUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[0], decode_kernel<false, false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[1], decode_kernel<true, false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ_seg[0], decode_kernel<false, true>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ_seg[1], decode_kernel<true, true>, kThreads, 0);
        for (int &o : d.occ) o = std::max(o, 1);
        for (int &o : d.occ_seg) o = std::max(o, 1);
    }
    *di = d;
    return VBYTE_OK;
}

int stream_workspace(cudaStream_t s, size_t need, uint8_t **ptr)
{
    Workspace *w = nullptr;
    const int rc = get_workspace(s, need, &w);
    if (rc == VBYTE_OK) *ptr = w->ptr;
    return rc;
}

int set_status_async(uint32_t *status, uint32_t bits, cudaStream_t s)
{
    set_status_kernel<<<1, 1, 0, s>>>(status, bits);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

// Batched decoding: lists j in [0, L) are bytes [bo[j], bo[j+1]) of in and
// values [vo[j], vo[j+1]) of out; the concatenation is decoded as one stream
// whose running value (delta) restarts at prevs[j] at each list head.
int check_batch(const BatchArgs &a)
{
    if ((a.nbytes && !a.in) || (a.n && !a.out) || !a.bo || !a.vo) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(a.out) & 3u) return VBYTE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.bo) | reinterpret_cast<uintptr_t>(a.vo)) & 7u) return VBYTE_EINVAL;
    if (a.prevs && (reinterpret_cast<uintptr_t>(a.prevs) & 3u)) return VBYTE_EINVAL;
    if (a.L == 0 && (a.nbytes || a.n)) return VBYTE_EINVAL;
    return VBYTE_OK;
}

uint64_t batch_tiles(const BatchArgs &a)
{
    const uintptr_t addr = reinterpret_cast<uintptr_t>(a.in);
    return a.nbytes ? ((addr & 15u) + a.nbytes + kTile - 1) / kTile : 0;
}

size_t batch_workspace_bytes(const BatchArgs &a) { return layout_seg(batch_tiles(a)).total; }

// Queue the batched decode of a (already checked, L > 0) on s, with its
// scratch in ws (layout_seg of the batch's tile count).
int enqueue_batched(const BatchArgs &a, uint8_t *ws, const LaunchCfg &cfg, const DeviceInfo &di, cudaStream_t s)
{
    const uintptr_t addr = reinterpret_cast<uintptr_t>(a.in);
    const uint64_t ntiles = batch_tiles(a);
    const LayoutSeg Y = layout_seg(ntiles);
    Params p = {};
    p.in = a.in;
    p.nbytes = a.nbytes;
    p.out = a.out;
    p.n = a.n;
    p.ntiles = ntiles;
    p.base = addr & ~static_cast<uintptr_t>(15);
    p.tdesc = reinterpret_cast<uint64_t *>(ws + Y.tdesc);
    p.cnext = reinterpret_cast<uint64_t *>(ws + Y.cnext);
    p.cdone = reinterpret_cast<unsigned int *>(ws + Y.cdone);
    p.cready = reinterpret_cast<unsigned int *>(ws + Y.cready);
    p.ctr = reinterpret_cast<unsigned long long *>(ws + Y.ctr);
    p.status = reinterpret_cast<uint32_t *>(ws);
    p.lead = std::min<uint64_t>(kChunkTiles + cfg.lead_slack, ntiles);
    p.bo = a.bo;
    p.vo = a.vo;
    p.prevs = a.prevs;
    p.L = a.L;
    p.hr = reinterpret_cast<const uint64_t *>(ws + Y.hr);
    p.tpre = reinterpret_cast<uint64_t *>(ws + Y.tpre);
    const uint64_t work = std::max<uint64_t>(ntiles, a.L);
    const unsigned pre_grid = static_cast<unsigned>(
        std::min<uint64_t>((work + 255) / 256, static_cast<uint64_t>(di.sms) * 8));
    head_range_kernel<<<std::max(pre_grid, 1u), 256, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return VBYTE_ECUDA;
    if (a.nbytes == 0) {
        if (a.n > 0) set_status_kernel<<<1, 1, 0, s>>>(p.status, VBYTE_ERR_COUNT_MISMATCH);
        return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
    }
    if (cudaMemsetAsync(ws + Y.ctr, 0, Y.clear, s) != cudaSuccess) return VBYTE_ECUDA;
    const int occ = di.occ_seg[a.delta];
    const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, occ) : occ;
    const uint64_t grid = std::min<uint64_t>(ntiles + p.lead, static_cast<uint64_t>(di.sms) * per_sm);
    if (a.delta)
        decode_kernel<true, true><<<static_cast<unsigned>(grid), kThreads, 0, s>>>(p);
    else
        decode_kernel<false, true><<<static_cast<unsigned>(grid), kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int reserve_workspace(cudaStream_t s, size_t nbytes)
{
    const uint64_t ntiles = (15 + nbytes + kTile - 1) / kTile;
    const size_t need = std::max(wdecode_workspace_bytes(nbytes), layout_seg(ntiles).total + 16 * ntiles);
    Workspace *w = nullptr;
    return get_workspace(s, need, &w);
}

int status_word(cudaStream_t s, uint32_t **word)
{
    Workspace *w = nullptr;
    const int rc = get_workspace(s, kWsHead, &w);
    if (rc == VBYTE_OK) *word = reinterpret_cast<uint32_t *>(w->ptr);
    return rc;
}

void release_workspace(cudaStream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find({dev, reinterpret_cast<uintptr_t>(s)});
    if (it != g_ws.end()) {
        if (it->second.ptr) cudaFreeAsync(it->second.ptr, s);
        g_ws.erase(it);
    }
    auto ih = g_hb.find({dev, reinterpret_cast<uintptr_t>(s)});
    if (ih != g_hb.end()) {
        if (ih->second.d_in) cudaFreeAsync(ih->second.d_in, s);
        if (ih->second.d_out) cudaFreeAsync(ih->second.d_out, s);
        g_hb.erase(ih);
    }
}

int launch_decode_batched(const BatchArgs &a, cudaStream_t s)
{
    int rc = check_batch(a);
    if (rc != VBYTE_OK || a.L == 0) return rc;
    Workspace *w = nullptr;
    rc = get_workspace(s, sbatched_workspace_bytes(a), &w);
    if (rc != VBYTE_OK) return rc;
    return enqueue_sbatched(a, w->ptr, LaunchCfg(), s);
}

// ---- scratch for vbyte_decode_noalloc -----------------------------------
// A file-scope device array replaces the per-stream workspace for callers
// that cannot allocate device memory.  It holds the layout() of an input of
// up to VBYTE_NOALLOC_MAX_BYTES bytes (about 545 KiB); every call on a device
// shares it.
constexpr size_t kStaticScratchBytes = size_t(576) << 10;
static __device__ __align__(256) uint8_t g_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
struct StaticDevice {
    bool ready = false;
    uint8_t *scratch = nullptr;
    int sms = 0;
    int occ[2] = {0, 0};
};
std::mutex g_static_mu;
StaticDevice g_static[kMaxStaticDevices];

// Set-up, once per device, with that device current: the address of
// g_scratch on it, its SM count and the kernels' occupancy.  No allocation.
int static_device(StaticDevice *out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    if (dev < 0 || dev >= kMaxStaticDevices) return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice &d = g_static[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return VBYTE_ECUDA;
        }
        int sms = 0, occ0 = 0, occ1 = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, decode_kernel<false, false>, kThreads, 0) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, decode_kernel<true, false>, kThreads, 0) !=
                cudaSuccess) {
            cudaGetLastError();
            return VBYTE_ECUDA;
        }
        d.scratch = static_cast<uint8_t *>(ptr);
        d.sms = sms;
        d.occ[0] = std::max(occ0, 1);
        d.occ[1] = std::max(occ1, 1);
        d.ready = true;
    }
    *out = d;
    return VBYTE_OK;
}

int launch_decode_noalloc(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta,
                          uint32_t prev, uint32_t *status, cudaStream_t s)
{
    if (nbytes > VBYTE_NOALLOC_MAX_BYTES) return VBYTE_ETOOBIG;
    if ((nbytes && !in) || (n && !out)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(out) & 3u) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(status) & 3u) return VBYTE_EINVAL;
    StaticDevice d;
    int rc = static_device(&d);
    if (rc != VBYTE_OK) return rc;
    if (nbytes == 0 && n == 0) return VBYTE_OK;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    const uint64_t ntiles = nbytes ? ((a & 15u) + nbytes + kTile - 1) / kTile : 0;
    const Layout L = layout(ntiles);
    if (L.total > kStaticScratchBytes) return VBYTE_ETOOBIG;
    // without a caller status word, data errors go to the array's own head
    if (status == nullptr) status = reinterpret_cast<uint32_t *>(d.scratch);
    if (nbytes == 0) {   // n > 0 values expected from an empty stream
        set_status_kernel<<<1, 1, 0, s>>>(status, VBYTE_ERR_COUNT_MISMATCH);
        return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
    }
    // the ticket counter, the chunk words and the group accumulators start at 0
    if (cudaMemsetAsync(d.scratch + L.ctr, 0, L.clear, s) != cudaSuccess) return VBYTE_ECUDA;
    Params p = {};
    p.in = in;
    p.nbytes = nbytes;
    p.out = out;
    p.n = n;
    p.ntiles = ntiles;
    p.base = a & ~static_cast<uintptr_t>(15);
    p.tdesc = reinterpret_cast<uint64_t *>(d.scratch + L.tdesc);
    p.gagg = reinterpret_cast<unsigned long long *>(d.scratch + L.gagg);
    p.gpre = reinterpret_cast<uint64_t *>(d.scratch + L.gpre);
    p.cnext = reinterpret_cast<uint64_t *>(d.scratch + L.cnext);
    p.cdone = reinterpret_cast<unsigned int *>(d.scratch + L.cdone);
    p.cready = reinterpret_cast<unsigned int *>(d.scratch + L.cready);
    p.ctr = reinterpret_cast<unsigned long long *>(d.scratch + L.ctr);
    p.status = status;
    p.prev = prev;
    p.lead = std::min<uint64_t>(kChunkTiles + kLeadSlack, ntiles);
    const uint64_t grid = std::min<uint64_t>(ntiles + p.lead, static_cast<uint64_t>(d.sms) * d.occ[delta]);
    if (delta)
        decode_kernel<true, false><<<static_cast<unsigned>(grid), kThreads, 0, s>>>(p);
    else
        decode_kernel<false, false><<<static_cast<unsigned>(grid), kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace vbk

extern "C" {

int vbyte_decode(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, false, 0u, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, uint32_t prev,
                       void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, true, prev, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_batched(const uint8_t *d_in, size_t nbytes, const uint64_t *d_byte_off, uint32_t *d_out,
                         size_t n, const uint64_t *d_val_off, size_t num_lists, void *stream)
{
    const vbk::BatchArgs a{d_in, nbytes, d_byte_off, d_out, n, d_val_off, num_lists, nullptr, false};
    return vbk::launch_decode_batched(a, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta_batched(const uint8_t *d_in, size_t nbytes, const uint64_t *d_byte_off, uint32_t *d_out,
                               size_t n, const uint64_t *d_val_off, size_t num_lists, const uint32_t *d_prev,
                               void *stream)
{
    const vbk::BatchArgs a{d_in, nbytes, d_byte_off, d_out, n, d_val_off, num_lists, d_prev, true};
    return vbk::launch_decode_batched(a, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_host(const uint8_t *h_in, size_t nbytes, uint32_t *h_out, size_t n, int delta,
                      uint32_t prev, void *stream)
{
    if ((nbytes && !h_in) || (n && !h_out)) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    vbk::HostBuffers *hb;
    {
        std::lock_guard<std::mutex> lk(vbk::g_mu);
        hb = &vbk::g_hb[{dev, reinterpret_cast<uintptr_t>(s)}];
        if (hb->cap_in < nbytes) {
            if (hb->d_in) cudaFreeAsync(hb->d_in, s);
            hb->d_in = nullptr;
            hb->cap_in = 0;
            void *p = nullptr;
            if (cudaMallocAsync(&p, nbytes, s) != cudaSuccess) return VBYTE_ENOMEM;
            hb->d_in = static_cast<uint8_t *>(p);
            hb->cap_in = nbytes;
        }
        if (hb->cap_out < n) {
            if (hb->d_out) cudaFreeAsync(hb->d_out, s);
            hb->d_out = nullptr;
            hb->cap_out = 0;
            void *p = nullptr;
            if (cudaMallocAsync(&p, n * sizeof(uint32_t), s) != cudaSuccess) return VBYTE_ENOMEM;
            hb->d_out = static_cast<uint32_t *>(p);
            hb->cap_out = n;
        }
    }
    if (nbytes && cudaMemcpyAsync(hb->d_in, h_in, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VBYTE_ECUDA;
    int rc = vbk::launch_decode(hb->d_in, nbytes, hb->d_out, n, delta != 0, prev, s);
    if (rc != VBYTE_OK) return rc;
    if (n && cudaMemcpyAsync(h_out, hb->d_out, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VBYTE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int vbyte_decode_noalloc(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, int delta,
                         uint32_t prev, uint32_t *d_status, void *stream)
{
    return vbk::launch_decode_noalloc(d_in, nbytes, d_out, n, delta != 0, prev, d_status,
                                      static_cast<cudaStream_t>(stream));
}

int vbyte_get_status(void *stream, uint32_t *status_out)
{
    if (!status_out) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vbk::Workspace *w = nullptr;
    int rc = vbk::get_workspace(s, vbk::kWsHead, &w);
    if (rc != VBYTE_OK) return rc;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, w->ptr, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaMemsetAsync(w->ptr, 0, sizeof(uint32_t), s) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VBYTE_ECUDA;
    *status_out = v;
    return VBYTE_OK;
}

const char *vbyte_strerror(int code)
{
    switch (code) {
    case VBYTE_OK: return "ok";
    case VBYTE_EINVAL: return "invalid argument (null pointer with nonzero size or misaligned output)";
    case VBYTE_ECUDA: return "CUDA runtime error or kernel launch failure";
    case VBYTE_ENOMEM: return "workspace allocation failed (or needed during stream capture)";
    case VBYTE_ETOOBIG: return "input larger than VBYTE_NOALLOC_MAX_BYTES (vbyte_decode_noalloc)";
    default: return "unknown vbyte error code";
    }
}

size_t vbyte_workspace_size(size_t nbytes)
{
    const uint64_t ntiles = (15 + nbytes + vbk::kTile - 1) / vbk::kTile;
    return std::max(vbk::wdecode_workspace_bytes(nbytes), vbk::layout_seg(ntiles).total);
}

}  // extern "C"
