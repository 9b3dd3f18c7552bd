// Split single-stream decoder: count, scan, decode -- three launches and no
// wait between CTAs anywhere.
//
// Operation (arXiv 1503.07387): Algorithm 1 (Sec. 2) on a VByte byte stream
// (Sec. 1, Table 1), optionally followed by the prefix sum that undoes
// differential coding (Sec. 1 "Differential coding", Sec. 4).
//
// Design:
//   * The stream is cut into 2 KiB warp tiles aligned to 16 bytes in absolute
//     address space (tile 0 starts at the input rounded down to 16 bytes).
//     A warp tile owns the integers whose terminator byte lies in it and in
//     the stream.
//   * count: CTA c owns the contiguous warp tiles [c T, (c + 1) T) (a range);
//     its warps take every eighth tile, four 512-byte units of one 16-byte
//     slice per lane.  Per warp tile, its integers and (delta) their sum -- a
//     popc of the terminator mask and, for the sum, the byte-weight formula
//     for codes of at most two bytes, else every byte weighted by 128^place
//     with the tile's two ends corrected (no assembly).  The CTA scans its
//     range in shared memory and writes, per tile, the count and sum of the
//     range's tiles before it, and the range's totals.  The data-error
//     contract is checked here.
//   * scan: one CTA turns the range totals into each range's prefix: values
//     before it and the running x before it (from prev).
//   * decode (decode2_kernel): persistent CTAs whose warps take warp tiles
//     round-robin and work alone -- no CTA barrier, no wait on another CTA.
//     A step is 1 KiB (32 bytes per lane), loaded into registers a step
//     ahead; values are staged at their output positions in a padded
//     per-warp buffer and written with coalesced 16-byte stores.  The
//     blocked-difference and table-driven settings keep the earlier launch
//     (decode_kernel: 512-byte units through a cp.async ring), whose unit
//     functions the batched list items also use.
// The input is read twice (count, decode); the per-tile words add 8 bytes per
// 2 KiB.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "vbyte.h"
#include "vbyte_device.cuh"
#include "vbyte_emit.cuh"
#include "vbyte_internal.h"
#include "vbyte_table.cuh"

namespace vbk {
namespace sp {

constexpr int kLanes = 32;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * kLanes;
constexpr int kUnit = kLanes * kBPT;            // 512 bytes per warp step
constexpr int kUnits = 4;                       // units per warp tile
constexpr int kWT = kUnit * kUnits;             // 2 KiB warp tile
constexpr uint32_t kMaxT = 1024;                // warp tiles per CTA range
constexpr int kRing = 4;                        // unit buffers per warp (kRing - 1 in flight)
constexpr int kSlot = kHalo + kUnit + 16;       // a unit, the 16 bytes before and after it
constexpr int kVal = kUnit + 16;                // staged values of one unit
constexpr uint32_t kMaxRanges = 8192;           // bound on the ranges beyond nwt / kMaxT
static_assert(kWT == 1 << 11, "warp tile addresses are t << 11");

struct Params {
    const uint8_t *in;
    uint64_t nbytes;
    uint32_t *out;
    uint64_t n;
    uintptr_t base;     // 16-byte aligned address of warp tile 0
    uint64_t nwt;       // warp tiles
    uint64_t in_lo;     // warp tiles [in_lo, in_hi) lie wholly inside the stream
    uint64_t in_hi;
    uint32_t T;         // warp tiles per range
    uint32_t G;         // ranges (CTAs of the count and decode launches)
    uint32_t range0;    // the first range of a launch (pieces of a pipelined decode; else 0)
    uint2 *ent;         // per warp tile: (count, sum) before it within its range
    uint2 *ctot;        // per range: (count, sum) of the range
    uint4 *cpre;        // per range: values before it (lo, hi), running x before it, 0
    uint32_t *status;
    uint32_t prev;      // x_0
    // blocked differences (x_i = g_i + x_{i-4}): per class of rank modulo 4
    uint4 prev4;        // x_{-4} .. x_{-1}, the seeds of classes 0..3
    uint4 *ent4;        // per warp tile: sums before it within its range, by class relative to the range
    uint4 *ctot4;       // per range: its sums by class relative to its start
    uint4 *cpre4;       // per range: the running value of each class (by rank modulo 4) before it
};

// ---- blocked differences: segments of (count, per-class sums)
//
// A segment's sums are indexed by class relative to its first rank.  r =
// rot4(s, c) re-indexes them for a start c ranks later: r[m] = s[(m - c) & 3].
__device__ __forceinline__ uint4 rot4(uint4 s, uint32_t c)
{
    switch (c & 3u) {
    case 0: return s;
    case 1: return make_uint4(s.w, s.x, s.y, s.z);
    case 2: return make_uint4(s.z, s.w, s.x, s.y);
    default: return make_uint4(s.y, s.z, s.w, s.x);
    }
}

__device__ __forceinline__ uint4 add4(uint4 a, uint4 b) { return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

struct Seg4 {
    uint32_t c;   // values (mod 2^32: only the class shift c & 3 and relative counts are used)
    uint4 s;      // sums by class relative to the segment's start
};

// a, then b
__device__ __forceinline__ Seg4 cat4(Seg4 a, Seg4 b)
{
    Seg4 r;
    r.c = a.c + b.c;
    r.s = add4(a.s, rot4(b.s, a.c));
    return r;
}

__device__ __forceinline__ Seg4 shfl_up4(Seg4 x, int o)
{
    Seg4 y;
    y.c = __shfl_up_sync(~0u, x.c, o);
    y.s.x = __shfl_up_sync(~0u, x.s.x, o);
    y.s.y = __shfl_up_sync(~0u, x.s.y, o);
    y.s.z = __shfl_up_sync(~0u, x.s.z, o);
    y.s.w = __shfl_up_sync(~0u, x.s.w, o);
    return y;
}

__device__ __forceinline__ Seg4 warp_incl_scan4(Seg4 x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Seg4 y = shfl_up4(x, o);
        if (lane >= o) x = cat4(y, x);
    }
    return x;
}

// Lane-level: f(v) for each value of a slice whose terminator is marked in
// tc, in order (codes of any length; bytes outside the stream are zero).
template <typename F>
__device__ __forceinline__ void slice_values(uint4 w, uint32_t wp, uint32_t tl, uint32_t t20, uint32_t tc, bool in,
                                             F f)
{
    const uint32_t c20 = ~t20 & 0xFFFFFu;
    if (!(c20 & (c20 << 1) & 0xFFFF8u)) {   // codes of at most two bytes
        const uint32_t c4[4] = {w.x, w.y, w.z, w.w};
        uint32_t wpp = wp;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const Pairs pr = pairs_le2(wpp, c4[j]);
            uint32_t q01 = prmt(pr.lob, pr.hib, 0x5140u);
            uint32_t q23 = prmt(pr.lob, pr.hib, 0x7362u);
            q01 -= (q01 & 0xFF00FF00u) >> 1;
            q23 -= (q23 & 0xFF00FF00u) >> 1;
            const uint32_t v4[4] = {q01 & 0xFFFFu, q01 >> 16, q23 & 0xFFFFu, q23 >> 16};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((tc >> (4 * j + i)) & 1u) f(v4[i]);
            wpp = c4[j];
        }
    } else if (in && !dense_words(tl)) {
        uint32_t v[4];
        const uint32_t nz = words4(wp, w, tl, t20, v);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((nz >> j) & 1u) f(v[j]);
    } else {
        assemble_regs(wp, w, tl, t20, tc, f);
    }
}

__device__ __forceinline__ bool interior(const Params &p, uint64_t t) { return t >= p.in_lo && t < p.in_hi; }

// A 16-byte slice at va; bytes outside [lo, hi) read as zero.
__device__ __forceinline__ uint4 load_slice(uintptr_t va, bool inside, uintptr_t lo, uintptr_t hi)
{
    if (inside || (va >= lo && va + kBPT <= hi)) return __ldg(reinterpret_cast<const uint4 *>(va));
    uint32_t wb[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const uintptr_t ad = va + j;
        if (ad >= lo && ad < hi) wb[j >> 2] |= static_cast<uint32_t>(*reinterpret_cast<const uint8_t *>(ad)) << (8 * (j & 3));
    }
    return make_uint4(wb[0], wb[1], wb[2], wb[3]);
}

// ---- count

// One warp: the integers of warp tile t and (delta) their sum, or (blocked
// differences, kD4) their sums by class relative to the tile's first rank.
template <bool kDelta, bool kD4>
__device__ __forceinline__ void count_wt(const Params &p, uint64_t t, int lane, uint32_t &cnt_out, uint32_t &sum_out,
                                         uint4 &s4_out)
{
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const bool in = interior(p, t);
    const uintptr_t w0 = p.base + (static_cast<uintptr_t>(t) << 11);
    uint4 w[kUnits];
#pragma unroll
    for (int u = 0; u < kUnits; ++u) w[u] = load_slice(w0 + u * kUnit + lane * kBPT, in, lo, hi);
    // the 4 bytes before the tile (inside the stream for t > 0; none before tile 0)
    uint32_t before = 0;
    if (lane == 0 && t > 0) before = __ldg(reinterpret_cast<const uint32_t *>(w0 - 4));
    uint32_t cnt = 0, sum = 0;
    uint32_t wps[kUnits];                          // kDelta: the 4 bytes before each slice
    uint32_t tl3 = 0;                              // kDelta: terminators of the last slice
    bool all_le2 = true;                           // kDelta: codes of at most two bytes in every unit
    uint32_t ub = 0;                               // kD4: values of the tile's earlier units
    uint4 s4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
        uint32_t wp = __shfl_up_sync(~0u, w[u].w, 1);
        const uint32_t last = (u == 0) ? before : __shfl_sync(~0u, w[u - 1].w, kLanes - 1);
        if (lane == 0) wp = last;
        const uintptr_t va = w0 + u * kUnit + lane * kBPT;
        const uint32_t tl = term4(w[u].x) | (term4(w[u].y) << 4) | (term4(w[u].z) << 8) | (term4(w[u].w) << 12);
        const uint32_t t20 = term4(wp) | (tl << 4);
        const uint32_t tc = in ? tl : (tl & slice_valid(va, lo, hi));
        const uint32_t cu = __popc(tc);
        cnt += cu;
        const uint32_t c20 = ~t20 & 0xFFFFFu;
        if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
            atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
        if (kD4) {
            // the lane's values by lane-relative class: add to a.x, then rotate,
            // so a holds class (k + cu) & 3 in component k at the end
            uint4 a = make_uint4(0u, 0u, 0u, 0u);
            slice_values(w[u], wp, tl, t20, tc, in, [&](uint32_t v) { a = make_uint4(a.y, a.z, a.w, a.x + v); });
            const uint32_t inc = warp_incl_scan(cu, lane);
            // lane class k is tile class (ub + inc - cu + k) & 3
            s4 = add4(s4, rot4(a, ub + inc));
            ub += __shfl_sync(~0u, inc, 31);
        }
        if (t == p.nwt - 1 && hi - 1 >= va && hi - 1 < va + kBPT && !((tl >> (hi - 1 - va)) & 1u))
            atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        if (kDelta) {
            wps[u] = wp;
            if (u == kUnits - 1) tl3 = tl;
            const bool le2 = __all_sync(~0u, !(c20 & (c20 << 1) & 0xFFFF8u));
            all_le2 = all_le2 && le2;
            if (!in)   // the stream's end tiles: per-integer assembly
                assemble_regs(wp, w[u], tl, t20, tc, [&](uint32_t v) { sum += v; });
        }
    }
    if (kDelta && in) {
        if (all_le2) {
            // codes of at most two bytes: the byte-weight formula per lane
#pragma unroll
            for (int u = 0; u < kUnits; ++u) sum += sum_le2_fast(w[u], wps[u]);
        } else {
            // any codes: every byte of the tile weighted by 128^place, with
            // the bytes after the tile's last terminator (the next tile's
            // first integer, lane 31's last slice) left out and the bytes
            // before the tile that start its first integer (after the last
            // terminator of the 4 bytes before it, lane 0) taken in
            uint32_t a[3] = {0u, 0u, 0u};
#pragma unroll
            for (int u = 0; u < kUnits; ++u) {
                uint32_t keep = 0xFFFFu;
                if (u == kUnits - 1 && lane == kLanes - 1) keep = tl3 ? (2u << (31 - __clz(tl3))) - 1u : 0u;
                const uint32_t W4[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
                uint32_t cpv = cont_flags(wps[u]);
#pragma unroll
                for (int j = 0; j < 4; ++j) cpv = place_sums(cpv, W4[j], nibble_to_bytes((keep >> (4 * j)) & 0xFu), a);
            }
            if (lane == 0) {
                const uint32_t tb = term4(before);
                const uint32_t head = tb ? 0xFu & ~((2u << (31 - __clz(tb))) - 1u) : 0xFu;
                place_sums(0u, before, nibble_to_bytes(head), a);
            }
            sum += a[0] + 127u * (a[1] + 16384u * a[2]);
        }
    }
    cnt_out = __reduce_add_sync(~0u, cnt);
    sum_out = kDelta ? __reduce_add_sync(~0u, sum) : 0u;
    if (kD4)
        s4_out = make_uint4(__reduce_add_sync(~0u, s4.x), __reduce_add_sync(~0u, s4.y), __reduce_add_sync(~0u, s4.z),
                            __reduce_add_sync(~0u, s4.w));
}

// Blocked differences: the range's entries scanned with cat4 (per-class sums
// re-indexed by the counts before them).
__device__ __forceinline__ void range_scan4(const Params &p, uint64_t t0, uint32_t nt, const uint2 *E, const uint4 *E4)
{
    __shared__ Seg4 wq[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t per = (nt + kThreads - 1) / kThreads;
    const uint32_t a = min(nt, tid * per), e = min(nt, a + per);
    Seg4 mine = {0u, make_uint4(0u, 0u, 0u, 0u)};
    for (uint32_t i = a; i < e; ++i) mine = cat4(mine, Seg4{E[i].x, E4[i]});
    const Seg4 inc = warp_incl_scan4(mine, lane);
    if (lane == kLanes - 1) wq[warp] = inc;
    __syncthreads();
    Seg4 x = {0u, make_uint4(0u, 0u, 0u, 0u)}, tot = {0u, make_uint4(0u, 0u, 0u, 0u)};
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
        if (q < warp) x = cat4(x, wq[q]);
        tot = cat4(tot, wq[q]);
    }
    Seg4 ex = shfl_up4(inc, 1);
    if (lane == 0) ex = Seg4{0u, make_uint4(0u, 0u, 0u, 0u)};
    x = cat4(x, ex);
    for (uint32_t i = a; i < e; ++i) {
        p.ent[t0 + i] = make_uint2(x.c, 0u);
        p.ent4[t0 + i] = x.s;
        x = cat4(x, Seg4{E[i].x, E4[i]});
    }
    if (tid == 0) {
        p.ctot[blockIdx.x + p.range0] = make_uint2(tot.c, 0u);
        p.ctot4[blockIdx.x + p.range0] = tot.s;
    }
}

template <bool kDelta, bool kD4>
__global__ void __launch_bounds__(kThreads, 5) count_kernel(const Params p)
{
    __shared__ uint2 E[kMaxT];
    __shared__ uint4 E4[kD4 ? kMaxT : 1];
    __shared__ uint32_t wcnt[kWarps], wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t t0 = static_cast<uint64_t>(blockIdx.x + p.range0) * p.T;
    const uint32_t nt = static_cast<uint32_t>(min(static_cast<uint64_t>(p.T), p.nwt - t0));
    for (uint32_t i = warp; i < nt; i += kWarps) {
        uint32_t c, s;
        uint4 s4;
        count_wt<kDelta, kD4>(p, t0 + i, lane, c, s, s4);
        if (lane == 0) {
            E[i] = make_uint2(c, s);
            if (kD4) E4[i] = s4;
        }
    }
    __syncthreads();
    if (kD4) {
        range_scan4(p, t0, nt, E, E4);
        return;
    }
    // exclusive scan of the range's entries: thread i takes [i per, (i + 1) per)
    const uint32_t per = (nt + kThreads - 1) / kThreads;
    const uint32_t a = min(nt, tid * per), e = min(nt, a + per);
    uint32_t c = 0, s = 0;
    for (uint32_t i = a; i < e; ++i) {
        c += E[i].x;
        s += E[i].y;
    }
    const uint32_t ic = warp_incl_scan(c, lane), is = warp_incl_scan(s, lane);
    if (lane == kLanes - 1) {
        wcnt[warp] = ic;
        wsum[warp] = is;
    }
    __syncthreads();
    uint32_t bc = 0, bs = 0, tc = 0, ts = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
        if (q < warp) {
            bc += wcnt[q];
            bs += wsum[q];
        }
        tc += wcnt[q];
        ts += wsum[q];
    }
    uint32_t xc = bc + ic - c, xs = bs + is - s;
    for (uint32_t i = a; i < e; ++i) {
        const uint2 v = E[i];
        p.ent[t0 + i] = make_uint2(xc, xs);
        xc += v.x;
        xs += v.y;
    }
    if (tid == 0) p.ctot[blockIdx.x + p.range0] = make_uint2(tc, ts);
}

// ---- scan of the range totals (one CTA)

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) scan_kernel(const Params p)
{
    __shared__ unsigned long long wc[kScanThreads / 32];
    __shared__ uint32_t wsm[kScanThreads / 32];
    __shared__ unsigned long long carry_c;
    __shared__ uint32_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry_c = 0;
        carry_s = p.prev;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < p.G; b0 += kScanThreads) {
        const uint32_t i = b0 + tid;
        const uint2 v = i < p.G ? p.ctot[i] : make_uint2(0u, 0u);
        // counts of a range fit 32 bits, those of 32 ranges too (T <= 1024 tiles of 2048 values)
        const uint32_t ic = warp_incl_scan(v.x, lane), is = warp_incl_scan(v.y, lane);
        if (lane == 31) {
            wc[warp] = ic;
            wsm[warp] = is;
        }
        __syncthreads();
        unsigned long long bc = carry_c, tc = 0;
        uint32_t bs = carry_s, ts = 0;
        for (int q = 0; q < kScanThreads / 32; ++q) {
            if (q < warp) {
                bc += wc[q];
                bs += wsm[q];
            }
            tc += wc[q];
            ts += wsm[q];
        }
        const unsigned long long xc = bc + ic - v.x;
        const uint32_t xs = bs + is - v.y;
        if (i < p.G)
            p.cpre[i] = make_uint4(static_cast<uint32_t>(xc), static_cast<uint32_t>(xc >> 32), xs, 0u);
        __syncthreads();
        if (tid == 0) {
            carry_c += tc;
            carry_s += ts;
        }
        __syncthreads();
    }
    if (tid == 0 && carry_c != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
}

// A piece of a pipelined decode: the prefixes of ranges [range0, r1), from
// the carry the earlier pieces left (values before the piece, running x;
// the first piece starts from none and prev); then the carry after the
// piece.  The last piece checks the total against n.
__global__ void __launch_bounds__(kScanThreads) scan_piece_kernel(const Params p, uint32_t r1,
                                                                  unsigned long long *carry, bool first, bool last)
{
    __shared__ unsigned long long wc[kScanThreads / 32];
    __shared__ uint32_t wsm[kScanThreads / 32];
    __shared__ unsigned long long carry_c;
    __shared__ uint32_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry_c = first ? 0ull : carry[0];
        carry_s = first ? p.prev : static_cast<uint32_t>(carry[1]);
    }
    __syncthreads();
    for (uint32_t b0 = p.range0; b0 < r1; b0 += kScanThreads) {
        const uint32_t i = b0 + tid;
        const uint2 v = i < r1 ? p.ctot[i] : make_uint2(0u, 0u);
        const uint32_t ic = warp_incl_scan(v.x, lane), is = warp_incl_scan(v.y, lane);
        if (lane == 31) {
            wc[warp] = ic;
            wsm[warp] = is;
        }
        __syncthreads();
        unsigned long long bc = carry_c, tc = 0;
        uint32_t bs = carry_s, ts = 0;
        for (int q = 0; q < kScanThreads / 32; ++q) {
            if (q < warp) {
                bc += wc[q];
                bs += wsm[q];
            }
            tc += wc[q];
            ts += wsm[q];
        }
        const unsigned long long xc = bc + ic - v.x;
        const uint32_t xs = bs + is - v.y;
        if (i < r1) p.cpre[i] = make_uint4(static_cast<uint32_t>(xc), static_cast<uint32_t>(xc >> 32), xs, 0u);
        __syncthreads();
        if (tid == 0) {
            carry_c += tc;
            carry_s += ts;
        }
        __syncthreads();
    }
    if (tid == 0) {
        carry[0] = carry_c;
        carry[1] = carry_s;
        if (last && carry_c != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
    }
}

// The blocked-difference form: cat4 over the ranges from the seed (no
// values, each class at its x_{-4..-1}); per range the count before it and
// each class's running value before it.
__global__ void __launch_bounds__(kScanThreads) scan4_kernel(const Params p)
{
    __shared__ Seg4 wq[kScanThreads / 32];
    __shared__ Seg4 carry;                 // the seed, then every range before the block
    __shared__ unsigned long long carry_c; // values before the block
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Seg4 zero = {0u, make_uint4(0u, 0u, 0u, 0u)};
    if (tid == 0) {
        carry = Seg4{0u, p.prev4};
        carry_c = 0;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < p.G; b0 += kScanThreads) {
        const uint32_t i = b0 + tid;
        const Seg4 v = i < p.G ? Seg4{p.ctot[i].x, p.ctot4[i]} : zero;
        const Seg4 inc = warp_incl_scan4(v, lane);   // a warp's count fits 32 bits
        if (lane == 31) wq[warp] = inc;
        __syncthreads();
        Seg4 x = carry;
        unsigned long long xc = carry_c;
        for (int q = 0; q < warp; ++q) {
            x = cat4(x, wq[q]);
            xc += wq[q].c;
        }
        Seg4 ex = shfl_up4(inc, 1);
        if (lane == 0) ex = zero;
        x = cat4(x, ex);
        xc += ex.c;
        if (i < p.G) {
            p.cpre[i] = make_uint4(static_cast<uint32_t>(xc), static_cast<uint32_t>(xc >> 32), 0u, 0u);
            p.cpre4[i] = x.s;
        }
        __syncthreads();
        if (tid == 0) {
            Seg4 c = carry;
            unsigned long long cc = carry_c;
            for (int q = 0; q < kScanThreads / 32; ++q) {
                c = cat4(c, wq[q]);
                cc += wq[q].c;
            }
            carry = c;
            carry_c = cc;
        }
        __syncthreads();
    }
    if (tid == 0 && carry_c != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
}

// ---- decode (every warp on its own)

struct WarpSmem {
    alignas(16) uint8_t ring[kRing][kSlot];   // units staged with their 16 bytes before
    alignas(16) uint32_t vals[kVal];          // a unit's values at rank + 4
};
static_assert(sizeof(WarpSmem) % 16 == 0 && kSlot % 16 == 0, "unit buffers keep 16-byte alignment");

// Stage unit u of warp tile t into `slot` (the 16 bytes before the unit at
// slot[0..16), the unit at slot[16..528)); bytes outside the stream as zero.
// The caller commits.
// Stage the unit at ua (16-byte aligned) and the 16 bytes before it into
// `slot`; bytes outside [lo, hi) as zero.  inside: all of them lie in
// [lo, hi).  The caller commits.
__device__ __forceinline__ void stage_unit(uintptr_t ua, int lane, uint8_t *slot, uintptr_t lo, uintptr_t hi,
                                           bool inside)
{
    const uintptr_t va = ua + lane * kBPT;
    uint8_t *dst = slot + kHalo + lane * kBPT;
    if (inside) {
        cp_async16(dst, reinterpret_cast<const void *>(va));
        if (lane == 0) cp_async16(slot, reinterpret_cast<const void *>(ua - 16));
        return;
    }
    if (va >= lo && va + kBPT <= hi) {
        cp_async16(dst, reinterpret_cast<const void *>(va));
    } else {
        const uint4 v = load_slice(va, false, lo, hi);
        *reinterpret_cast<uint4 *>(dst) = v;
    }
    if (lane == 0) {
        const uintptr_t ha = ua - 16;
        if (ha >= lo && ua <= hi)
            cp_async16(slot, reinterpret_cast<const void *>(ha));
        else
            *reinterpret_cast<uint4 *>(slot) = load_slice(ha, false, lo, hi);
    }
}

__device__ __forceinline__ void issue_unit(const Params &p, uint64_t t, int u, int lane, uint8_t *slot)
{
    const uintptr_t ua = p.base + (static_cast<uintptr_t>(t) << 11) + u * kUnit;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    // the unit and the 16 bytes before it are inside the stream
    const bool inside = interior(p, t) && (t > 0 || u > 0);
    stage_unit(ua, lane, slot, lo, lo + p.nbytes, inside);
}

// One warp: decode the staged unit ub into vals (warp rank r at vals[4 + r];
// delta: running sums from the unit's first value).  The unit owns the
// integers whose terminators lie in [lo, hi); in: it owns all its bytes.
// Returns the unit's value count and sum; one = every slice holds one-byte
// integers only (the values stay as bytes and vals is untouched).  kCheck:
// also record runs of five continuation bytes and (dend != 0) a stream that
// ends at dend inside an integer.
// The table-driven step (Sec. 4) for one lane: from the first byte of its
// first integer, the high-bit mask of the next 12 bytes picks (bytes
// consumed, case) from T; the case's lengths D give its integers; those whose
// terminators lie in the lane's slice and in tc are emitted in order.  An
// entry with nothing consumed (an integer of more than five bytes) hands the
// rest of the slice to per-terminator assembly.
template <typename F>
__device__ __forceinline__ void table_steps(const uint32_t *sw, int lane, const SliceMasks &m, const uint16_t *T,
                                            const uint32_t *D, F emit)
{
    const uint32_t q0 = kHalo + lane * kBPT;
    const uint32_t n0 = sw[q0 / 4 + 4], n1 = sw[q0 / 4 + 5], n2 = sw[q0 / 4 + 6];   // the 12 bytes after the slice
    // bit b: byte b - 4 of the slice has its high bit set
    const uint32_t cont =
        ~(term4(m.wprev) | (m.tl << 4) | (term4(n0) << 20) | (term4(n1) << 24) | (term4(n2) << 28));
    if (!m.tl) return;
    const uint32_t low = m.t20 & 0xFu;
    uint32_t b = low ? 32u - __clz(low) : 0u;   // first byte of the first integer
    const uint32_t endb = 31u - __clz(m.tl) + 4u;   // the slice's last terminator
    while (b <= endb) {
        const uint32_t e = T[(cont >> b) & 0xFFFu];
        const uint32_t c = e & 15u, id = e >> 4;
        if (!c) {   // malformed: the remaining terminators one by one
            const uint32_t keep = b >= 4 ? ~((1u << (b - 4)) - 1u) : ~0u;
            assemble_all(sw, lane, m.tl, m.t20, m.tc & keep, emit);
            return;
        }
        if (id == tab::kTwelve) {
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const int t = static_cast<int>(b) + i - 4;   // slice position of the one-byte integer
                if (t >= 0 && t < kBPT && ((m.tc >> t) & 1u)) {
                    const uint32_t q = q0 + t;
                    emit((sw[q >> 2] >> (8 * (q & 3))) & 0xFFu);
                }
            }
        } else {
            const uint32_t d = D[id];
            uint32_t o = b;
            for (uint32_t t = 0; t < tab::case_k(d); ++t) {
                const uint32_t L = tab::case_len(d, static_cast<int>(t));
                const int tp = static_cast<int>(o + L) - 5;   // slice position of the terminator
                if (tp >= 0 && tp < kBPT && ((m.tc >> tp) & 1u)) {
                    const uint32_t q = q0 + tp;
                    const uint32_t A = sw[(q >> 2) - 1];
                    const uint32_t B = sw[q >> 2];
                    emit(assemble(__funnelshift_r(A, B, 8 * q), prmt(B, 0u, 0x4440u | (q & 3u)), static_cast<int>(L)));
                }
                o += L;
            }
        }
        b += c;
    }
}

template <bool kDelta, bool kCheck = false, bool kTable = false>
__device__ __forceinline__ void unit_stage(const uint8_t *ub, bool in, uintptr_t ua, uintptr_t lo, uintptr_t hi,
                                           uint32_t *vals, int lane, uint32_t &wc, uint32_t &ws, bool &one,
                                           uint32_t *status = nullptr, uintptr_t dend = 0,
                                           const uint16_t *T = nullptr, const uint32_t *D = nullptr)
{
    const uint4 w0 = *reinterpret_cast<const uint4 *>(ub + kHalo + lane * kBPT);
    const uint32_t wp0 = reinterpret_cast<const uint32_t *>(ub)[(kHalo + lane * kBPT) / 4 - 1];
    const bool mineA = in && !((w0.x | w0.y | w0.z | w0.w) & 0x80808080u) && !(wp0 & 0x80000000u);
    ws = 0;
    one = __all_sync(~0u, mineA);
    if (one) {
        if (kDelta) ws = __reduce_add_sync(~0u, byte_sum4(w0));
        wc = kUnit;
        return;
    }
    const uintptr_t va = ua + lane * kBPT;
    const uint32_t *const sw = reinterpret_cast<const uint32_t *>(ub);
    const SliceMasks m = slice_masks(ub, lane, in, va, lo, hi);
    const uint32_t cnt = __popc(m.tc);
    const uint32_t c20 = ~m.t20 & 0xFFFFFu;
    const bool notB = (c20 & (c20 << 1) & 0xFFFF8u) != 0;
    if (kCheck) {
        if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
            atomicOr(status, VBYTE_ERR_MALFORMED_LONG);
        if (dend && dend - 1 >= va && dend - 1 < va + kBPT && !((m.tl >> (dend - 1 - va)) & 1u))
            atomicOr(status, VBYTE_ERR_TRUNCATED);
    }
    const uint32_t inc = warp_incl_scan(cnt, lane);
    wc = __shfl_sync(~0u, inc, 31);
    uint32_t *dst = vals + 4 + inc - cnt;
    uint32_t vsum = 0;
    if (kTable) {
        // the table-driven steps for every code length, then running sums
        table_steps(sw, lane, m, T, D, [&](uint32_t v) {
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
    } else if (!__any_sync(~0u, notB)) {
        // codes of at most two bytes: the lane's sum by the byte-weight
        // formula, then the values (with running sums) in one SWAR pass
        uint32_t run = 0;
        if (kDelta) {
            vsum = in ? sum_le2_fast(m.w, m.wprev) : sum_le2(m.w, m.wprev, m.tc);
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
        // longer codes: each value assembled once -- in registers, one fixed
        // step per word, when no word holds two terminators (running sums
        // from this lane's offset within the unit taken there too), else one
        // terminator at a time through the value buffer
        if (in && !__any_sync(~0u, dense_words(m.tl))) {
            uint32_t v[4];
            const uint32_t nz = words4(m.wprev, m.w, m.tl, m.t20, v);
            uint32_t run = 0;
            if (kDelta) {
#pragma unroll
                for (int j = 0; j < 4; ++j) vsum += ((nz >> j) & 1u) ? v[j] : 0u;
                const uint32_t incs = warp_incl_scan(vsum, lane);
                ws = __shfl_sync(~0u, incs, 31);
                run = incs - vsum;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((nz >> j) & 1u) {
                    if (kDelta) {
                        run += v[j];
                        *dst++ = run;
                    } else {
                        *dst++ = v[j];
                    }
                }
            }
            return;
        }
        assemble_all(sw, lane, m.tl, m.t20, m.tc, [&](uint32_t v) {
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

// One warp: a staged unit's values to out[G0 ..], coalesced, clamped to n.
template <bool kDelta, bool kRank>
__device__ __forceinline__ void unit_emit(const Params &p, const uint8_t *ub, uint32_t *vals, bool one, uint32_t wc,
                                          unsigned long long G0l, uint32_t add, int lane)
{
    const long long n = static_cast<long long>(p.n);
    const long long G0 = static_cast<long long>(G0l);
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
    const int sh = static_cast<int>((out_word + static_cast<uint32_t>(G0)) & 3u);
    uint32_t *const oq = p.out + (G0 - sh);   // 16-byte aligned; quad q at oq + 4q
    if (one) {   // warp-uniform
        const uint8_t *wb = ub + kHalo;
        if (G0 + kUnit <= n) {
            const uint32_t rb = static_cast<uint32_t>(G0);
            switch (sh) {
            case 0: emit_bytes_a<0, kDelta, kRank>(oq, wb, add, rb, lane); break;
            case 1: emit_bytes_a<1, kDelta, kRank>(oq, wb, add, rb, lane); break;
            case 2: emit_bytes_a<2, kDelta, kRank>(oq, wb, add, rb, lane); break;
            default: emit_bytes_a<3, kDelta, kRank>(oq, wb, add, rb, lane); break;
            }
            return;
        }
        // near the end of the output: through the value buffer, with the checks
        const uint4 w = *reinterpret_cast<const uint4 *>(wb + lane * kBPT);
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
    emit_staged<kRank>(oq, vals, static_cast<int>(wc), kDelta ? add : 0u, static_cast<uint32_t>(G0), n - G0, lane,
                       sh);
}

// Blocked differences: per-class running sums in place over a unit's staged
// values (quad j holds ranks 4j .. 4j + 3 of the unit, component k the class
// k relative to the unit's first rank); returns each class's total.  Ranks
// past wc count as zero.
__device__ __forceinline__ uint4 class_scan(uint32_t *vals, uint32_t wc, int lane)
{
    const uint32_t nq = (wc + 3u) >> 2;
    uint4 *v4 = reinterpret_cast<uint4 *>(vals + 4);
    uint4 carry = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t j0 = 0; j0 < nq; j0 += kLanes) {
        const uint32_t j = j0 + lane;
        uint4 v = j < nq ? v4[j] : make_uint4(0u, 0u, 0u, 0u);
        if (j + 1 == nq) {   // the last quad: ranks past wc
            const uint32_t r = wc - 4u * j;
            if (r < 2) v.y = 0u;
            if (r < 3) v.z = 0u;
            if (r < 4) v.w = 0u;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a = __shfl_up_sync(~0u, v.x, o), b = __shfl_up_sync(~0u, v.y, o);
            const uint32_t c = __shfl_up_sync(~0u, v.z, o), d = __shfl_up_sync(~0u, v.w, o);
            if (lane >= o) {
                v.x += a;
                v.y += b;
                v.z += c;
                v.w += d;
            }
        }
        if (j < nq) v4[j] = add4(carry, v);
        carry = add4(carry, make_uint4(__shfl_sync(~0u, v.x, 31), __shfl_sync(~0u, v.y, 31),
                                       __shfl_sync(~0u, v.z, 31), __shfl_sync(~0u, v.w, 31)));
    }
    return carry;
}

// The table and case descriptors of the table-driven step, built by the CTA.
struct TableSmem {
    uint16_t T[4096];
    uint32_t D[tab::kCases];
};

__device__ __forceinline__ void fill_table(TableSmem &S)
{
    for (uint32_t i = threadIdx.x; i < 4096; i += blockDim.x) S.T[i] = static_cast<uint16_t>(tab::table_entry(i));
    for (uint32_t i = threadIdx.x; i < static_cast<uint32_t>(tab::kCases); i += blockDim.x) S.D[i] = tab::case_desc(i);
}

template <bool kDelta, bool kRank, bool kD4 = false, bool kTable = false>
__global__ void __launch_bounds__(kThreads, 5) decode_kernel(const Params p)
{
    __shared__ WarpSmem Wsm[kWarps];
    extern __shared__ __align__(16) unsigned char dsm[];   // kTable: the table (dynamic shared memory)
    TableSmem &Tab = *reinterpret_cast<TableSmem *>(dsm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpSmem &M = Wsm[warp];
    if (kTable) {
        fill_table(Tab);
        __syncthreads();
    }
    if (lane < kRing) *reinterpret_cast<uint4 *>(M.ring[lane] + kHalo + kUnit) = make_uint4(0u, 0u, 0u, 0u);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uint64_t t0 = static_cast<uint64_t>(blockIdx.x + p.range0) * p.T;
    const uint32_t nt = static_cast<uint32_t>(min(static_cast<uint64_t>(p.T), p.nwt - t0));
    const uint32_t mine = nt > static_cast<uint32_t>(warp) ? (nt - warp + kWarps - 1) / kWarps : 0u;
    const uint32_t K = mine * kUnits;   // units of this warp: tiles warp, warp + 8, ... of the range
    const uint4 cp = p.cpre[blockIdx.x + p.range0];
    const unsigned long long C0 = cp.x | (static_cast<unsigned long long>(cp.y) << 32);
    auto issue = [&](uint32_t k) {
        if (k < K) issue_unit(p, t0 + warp + (k / kUnits) * kWarps, static_cast<int>(k % kUnits), lane,
                              M.ring[k % kRing]);
        cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < kRing - 1; ++i) issue(i);
    unsigned long long R = 0;
    uint32_t X = 0;
    uint4 B = make_uint4(0u, 0u, 0u, 0u);   // kD4: each class's running value (class = rank mod 4)
    uint4 cp4 = make_uint4(0u, 0u, 0u, 0u);
    if (kD4) cp4 = p.cpre4[blockIdx.x + p.range0];
    uint2 e_next = make_uint2(0u, 0u);
    if (K) e_next = p.ent[t0 + warp];
    for (uint32_t k = 0; k < K; ++k) {
        cp_async_wait_prior<kRing - 2>();   // unit k has landed (for this lane)
        __syncwarp();                       // ... for every lane
        issue(k + kRing - 1);
        const uint32_t u = k % kUnits;
        const uint64_t t = t0 + warp + (k / kUnits) * kWarps;
        if (u == 0) {
            R = C0 + e_next.x;
            X = cp.z + e_next.y;
            if (kD4) B = add4(cp4, rot4(p.ent4[t], static_cast<uint32_t>(C0)));
            if (k + kUnits < K) e_next = p.ent[t + kWarps];   // the next tile's prefix travels meanwhile
        }
        const uint8_t *ub = M.ring[k % kRing];
        const uintptr_t ua = p.base + (static_cast<uintptr_t>(t) << 11) + u * kUnit;
        uint32_t wc, ws;
        bool one;
        unit_stage<kDelta, false, kTable>(ub, interior(p, t), ua, lo, hi, M.vals, lane, wc, ws, one, nullptr, 0,
                                          Tab.T, Tab.D);
        __syncwarp();
        if (kD4) {
            if (one) {   // one-byte integers: the bytes become the staged values
                const uint4 w = *reinterpret_cast<const uint4 *>(ub + kHalo + lane * kBPT);
                uint4 *d4 = reinterpret_cast<uint4 *>(M.vals + 4 + 16 * lane);
                d4[0] = bytes_as_values(w.x);
                d4[1] = bytes_as_values(w.y);
                d4[2] = bytes_as_values(w.z);
                d4[3] = bytes_as_values(w.w);
                __syncwarp();
            }
            const uint4 T = class_scan(M.vals, wc, lane);
            __syncwarp();
            const uint32_t ow = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
            const int sh = static_cast<int>((ow + static_cast<uint32_t>(R)) & 3u);
            // the output word at position j of a 16-byte quad holds class (j - ow) & 3
            emit_staged4(p.out + (static_cast<long long>(R) - sh), M.vals, static_cast<int>(wc), rot4(B, ow),
                         static_cast<long long>(p.n) - static_cast<long long>(R), lane, sh);
            B = add4(B, rot4(T, static_cast<uint32_t>(R)));
        } else {
            unit_emit<kDelta, kRank>(p, ub, M.vals, one, wc, R, X, lane);
        }
        R += wc;
        X += ws;
        __syncwarp();   // the value buffer and this unit's slot are free again
    }
    cp_async_wait_all();
}

// ---- decode in 1 KiB warp steps (the stream decode launch)
//
// A warp step is 1 KiB of a warp tile, 32 bytes per lane, loaded straight
// into registers one step ahead: no shared-memory staging of the input.
// Each lane's values come from its eight words and the four bytes before
// them; they are staged, with running sums in differential mode, at their
// output positions -- step rank r at position s = r + sh, sh the output
// misalignment of the step's first value -- so that every output quad is one
// aligned 16-byte load, and one padding quad follows every 32 positions, so
// that lanes whose runs start 32 positions apart write different banks.  The
// launch's warps take the warp tiles of its interval round-robin; a tile's
// prefix comes from the count and scan launches.  A step of one-byte
// integers only is staged as bytes and written by the byte copy-out.

constexpr int kW2 = 4;                               // warps per CTA
constexpr int kThreads2 = kW2 * kLanes;
constexpr int kStep = 1024;                          // bytes per warp step
constexpr int kPos = kStep + 8;                      // positions: sh, the values, the last quad
constexpr int kVals2 = kPos + 4 * (kPos / 32 + 1);   // padded words per warp
static_assert(kVals2 * 4 >= 16 + kStep + 16, "the byte stage fits the value buffer");

__device__ __forceinline__ uint32_t pidx(uint32_t s) { return s + ((s >> 5) << 2); }

struct Step2 {
    uint4 a, b;        // the lane's 32 bytes
    uint32_t before;   // lane 0, first step of a tile: the 4 bytes before the tile (0 before tile 0)
};

__device__ __forceinline__ void load_step(const Params &p, uint64_t t, int h, int lane, uintptr_t lo, uintptr_t hi,
                                          Step2 &st)
{
    const bool in = interior(p, t);
    const uintptr_t va = p.base + (static_cast<uintptr_t>(t) << 11) + h * kStep + lane * 32;
    st.a = load_slice(va, in, lo, hi);
    st.b = load_slice(va + 16, in, lo, hi);
    st.before = 0u;
    if (h == 0 && lane == 0 && t > 0) st.before = __ldg(reinterpret_cast<const uint32_t *>(va - 4));
}

// Exclusive warp scan; *tot gets the warp's total.
__device__ __forceinline__ uint32_t warp_excl(uint32_t x, int lane, uint32_t *tot)
{
    const uint32_t inc = warp_incl_scan(x, lane);
    *tot = __shfl_sync(~0u, inc, 31);
    return inc - x;
}

template <bool kDelta, bool kRank>
__global__ void __launch_bounds__(kThreads2, 7) decode2_kernel(const Params p, uint64_t tb, uint64_t te)
{
    __shared__ __align__(16) uint32_t Vs[kW2][kVals2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *const V = Vs[warp];
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uint64_t NW = static_cast<uint64_t>(gridDim.x) * kW2;
    const uint64_t t0 = tb + static_cast<uint64_t>(blockIdx.x) * kW2 + warp;
    if (t0 >= te) return;
    const uint64_t K = 2 * ((te - t0 + NW - 1) / NW);   // steps of this warp
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
    const long long n = static_cast<long long>(p.n);
    Step2 cur, nxt;
    load_step(p, t0, 0, lane, lo, hi, nxt);
    uint2 e_nxt = p.ent[t0];
    uint4 c_nxt = p.cpre[static_cast<uint32_t>(t0) / p.T];
    unsigned long long R = 0;   // rank of the step's first value
    uint32_t X = 0;             // running x before it
    uint32_t last = 0;          // the previous step's last word (lane 31), same tile
    for (uint64_t k = 0; k < K; ++k) {
        const uint64_t t = t0 + (k >> 1) * NW;
        const int h = static_cast<int>(k & 1u);
        cur = nxt;
        if (h == 0) {
            R = (c_nxt.x | (static_cast<unsigned long long>(c_nxt.y) << 32)) + e_nxt.x;
            X = c_nxt.z + e_nxt.y;
        }
        if (k + 1 < K) {   // the next step's bytes (and the next tile's prefix) travel meanwhile
            const uint64_t tn = t0 + ((k + 1) >> 1) * NW;
            load_step(p, tn, static_cast<int>((k + 1) & 1u), lane, lo, hi, nxt);
            if (h == 1) {
                e_nxt = p.ent[tn];
                c_nxt = p.cpre[static_cast<uint32_t>(tn) / p.T];
            }
        }
        const bool in = interior(p, t);
        uint32_t wprev = __shfl_up_sync(~0u, cur.b.w, 1);
        if (lane == 0) wprev = h ? last : cur.before;
        last = __shfl_sync(~0u, cur.b.w, kLanes - 1);
        const uintptr_t va = p.base + (static_cast<uintptr_t>(t) << 11) + h * kStep + lane * 32;
        const uint32_t tlA = term4(cur.a.x) | (term4(cur.a.y) << 4) | (term4(cur.a.z) << 8) | (term4(cur.a.w) << 12);
        const uint32_t tlB = term4(cur.b.x) | (term4(cur.b.y) << 4) | (term4(cur.b.z) << 8) | (term4(cur.b.w) << 12);
        uint32_t tcA = tlA, tcB = tlB;
        if (!in) {   // warp-uniform: only the tiles at the stream's ends
            tcA &= slice_valid(va, lo, hi);
            tcB &= slice_valid(va + 16, lo, hi);
        }
        const uint32_t t20A = term4(wprev) | (tlA << 4);
        const uint32_t t20B = (tlA >> 12) | (tlB << 4);
        const uint32_t cnt = __popc(tcA) + __popc(tcB);
        uint32_t wc;
        const uint32_t base = warp_excl(cnt, lane, &wc);
        const uint32_t sh = (out_word + static_cast<uint32_t>(R)) & 3u;
        uint32_t ws = 0;
        const bool one = in && (tlA & tlB) == 0xFFFFu && !(wprev & 0x80000000u);
        if (__all_sync(~0u, one) && static_cast<long long>(R) + kStep <= n) {
            // one-byte integers only: the bytes themselves, written by the byte
            // copy-out (two 512-byte halves), with the 4 bytes before them
            uint8_t *const sb = reinterpret_cast<uint8_t *>(V) + 16;
            *reinterpret_cast<uint4 *>(sb + 32 * lane) = cur.a;
            *reinterpret_cast<uint4 *>(sb + 32 * lane + 16) = cur.b;
            if (lane == 0) reinterpret_cast<uint32_t *>(sb)[-1] = wprev;
            uint32_t s0 = 0;
            if (kDelta) {
                const uint32_t bs = byte_sum4(cur.a) + byte_sum4(cur.b);
                const uint32_t inc = warp_incl_scan(bs, lane);
                s0 = __shfl_sync(~0u, inc, 15);   // the first half's sum
                ws = __shfl_sync(~0u, inc, 31);
            }
            __syncwarp();
            uint32_t *const oq = p.out + (static_cast<long long>(R) - sh);
            const uint32_t rb = static_cast<uint32_t>(R);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t *const o = oq + half * (kStep / 2);
                const uint8_t *const wb = sb + half * (kStep / 2);
                const uint32_t ad = kDelta ? X + (half ? s0 : 0u) : 0u;
                const uint32_t r0 = rb + half * (kStep / 2);
                switch (sh) {
                case 0: emit_bytes_a<0, kDelta, kRank>(o, wb, ad, r0, lane); break;
                case 1: emit_bytes_a<1, kDelta, kRank>(o, wb, ad, r0, lane); break;
                case 2: emit_bytes_a<2, kDelta, kRank>(o, wb, ad, r0, lane); break;
                default: emit_bytes_a<3, kDelta, kRank>(o, wb, ad, r0, lane); break;
                }
            }
        } else {
            uint32_t s = sh + base;   // the lane's next position
            const uint32_t c20A = ~t20A & 0xFFFFFu, c20B = ~t20B & 0xFFFFFu;
            const bool le2 = !((c20A & (c20A << 1) & 0xFFFF8u) | (c20B & (c20B << 1) & 0xFFFF8u));
            if (__all_sync(~0u, le2)) {
                // codes of at most two bytes: the lane's sum by the byte-weight
                // formula, then the values (running sums) in one SWAR pass
                uint32_t run = 0;
                if (kDelta) {
                    const uint32_t vs = in ? sum_le2_fast(cur.a, wprev) + sum_le2_fast(cur.b, cur.a.w)
                                           : sum_le2(cur.a, wprev, tcA) + sum_le2(cur.b, cur.a.w, tcB);
                    run = warp_excl(vs, lane, &ws);
                }
                const uint32_t w8[8] = {cur.a.x, cur.a.y, cur.a.z, cur.a.w, cur.b.x, cur.b.y, cur.b.z, cur.b.w};
                const uint32_t tc = tcA | (tcB << 16);
                uint32_t wp = wprev;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const Pairs pr = pairs_le2(wp, w8[j]);
                    uint32_t q01 = prmt(pr.lob, pr.hib, 0x5140u);
                    uint32_t q23 = prmt(pr.lob, pr.hib, 0x7362u);
                    q01 -= (q01 & 0xFF00FF00u) >> 1;
                    q23 -= (q23 & 0xFF00FF00u) >> 1;
                    const uint32_t v4[4] = {q01 & 0xFFFFu, q01 >> 16, q23 & 0xFFFFu, q23 >> 16};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if ((tc >> (4 * j + i)) & 1u) {
                            run += v4[i];
                            V[pidx(s)] = kDelta ? run : v4[i];
                            ++s;
                        }
                    }
                    wp = w8[j];
                }
            } else if (in && !__any_sync(~0u, dense_words(tlA) | dense_words(tlB))) {
                // codes in separate words: every word's value in registers
                uint32_t vA[4], vB[4];
                const uint32_t nz = words4(wprev, cur.a, tlA, t20A, vA) | (words4(cur.a.w, cur.b, tlB, t20B, vB) << 4);
                const uint32_t v8[8] = {vA[0], vA[1], vA[2], vA[3], vB[0], vB[1], vB[2], vB[3]};
                uint32_t run = 0;
                if (kDelta) {
                    uint32_t vs = 0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) vs += ((nz >> j) & 1u) ? v8[j] : 0u;
                    run = warp_excl(vs, lane, &ws);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if ((nz >> j) & 1u) {
                        run += v8[j];
                        V[pidx(s)] = kDelta ? run : v8[j];
                        ++s;
                    }
                }
            } else {
                // anything else: one terminator at a time, then running sums
                uint32_t vs = 0;
                auto put = [&](uint32_t v) {
                    V[pidx(s)] = v;
                    ++s;
                    vs += v;
                };
                assemble_regs(wprev, cur.a, tlA, t20A, tcA, put);
                assemble_regs(cur.a.w, cur.b, tlB, t20B, tcB, put);
                if (kDelta) {
                    uint32_t run = warp_excl(vs, lane, &ws);
                    for (uint32_t q = sh + base; q < s; ++q) {
                        run += V[pidx(q)];
                        V[pidx(q)] = run;
                    }
                }
            }
            __syncwarp();
            // copy-out: positions [sh, sh + lim) hold ranks [0, lim)
            const long long room = n - static_cast<long long>(R);
            const uint32_t lim = room < static_cast<long long>(wc) ? (room > 0 ? static_cast<uint32_t>(room) : 0u)
                                                                    : wc;
            const uint32_t np = sh + lim;
            const uint32_t qa = sh ? 1u : 0u;   // quads [qa, qb) are whole
            const uint32_t qb = np >> 2;
            uint32_t *const oq = p.out + (static_cast<long long>(R) - sh);
            const uint32_t ad = kDelta ? X : 0u;
            const uint32_t rk = static_cast<uint32_t>(R) - sh;   // kRank: position 0's rank
            for (uint32_t q = qa + lane; q < qb; q += kLanes) {
                uint4 e = *reinterpret_cast<const uint4 *>(V + 4 * q + ((q >> 3) << 2));
                const uint32_t a0 = ad + (kRank ? rk + 4 * q : 0u);
                e.x += a0;
                e.y += a0 + (kRank ? 1u : 0u);
                e.z += a0 + (kRank ? 2u : 0u);
                e.w += a0 + (kRank ? 3u : 0u);
                st_quad(oq + 4 * q, e);
            }
            // the positions outside whole quads: lanes 0..3 the first quad's,
            // lanes 4..7 the last one's (when it is another quad)
            if (lane < 8) {
                const uint32_t ps = lane < 4 ? static_cast<uint32_t>(lane) : 4 * qb + lane - 4;
                const bool edge = lane < 4 ? ps < 4 * qa || qb < qa : qb >= qa;
                if (edge && ps >= sh && ps < np) oq[ps] = V[pidx(ps)] + ad + (kRank ? rk + ps : 0u);
            }
        }
        R += wc;
        X += ws;
        __syncwarp();   // the value buffer is free again
    }
}

// ---- batched lists as work items (tuned plans)
//
// A plan cuts the batch into items: a whole list of at most C bytes, or a
// C-byte chunk of a longer list (chunks start on 16-byte boundaries of the
// input).  One warp decodes one item by itself, taking items from a queue,
// longest first: a whole list in a single pass (its first value's rank and
// x_0 are vo[j] and prev[j]), a chunk from the count and sum of its list's
// earlier chunks (a count launch over the chunks, then one warp per chunked
// list scans them).  Per-list data errors are checked by the decode launch;
// a chunked list's count by the scan.

using Item = ListItem;
constexpr uint32_t kOnly = kItemOnly, kLast = kItemLast;

struct LParams {
    const uint8_t *in;
    uint32_t *out;
    const uint64_t *bo, *vo;     // list byte and value offsets
    const uint32_t *prevs;       // per-list x_0, or null (zeros)
    const Item *items;           // in decode order
    uint32_t nitems;
    const uint32_t *citem;       // the items of chunked lists, list by list, chunk by chunk
    const uint32_t *cfirst;      // per chunked list: its first citem entry; cfirst[ncl] = the entries
    uint32_t ncl;
    uint2 *cs;                   // per item: its count and sum (chunked lists)
    uint2 *rel;                  // per item: count and sum of its list's earlier chunks (zero for first chunks)
    unsigned int *queue;         // the decode launch's next item (cleared before it)
    uint32_t *status;
};

// One warp: the integers whose terminators lie in [c0, c1) and (delta) their
// sum; the bytes of the list are [lo, hi) (others read as zero).
template <bool kDelta>
__device__ __forceinline__ void count_range(uintptr_t c0, uintptr_t c1, uintptr_t lo, uintptr_t hi, int lane,
                                            uint32_t &cnt_out, uint32_t &sum_out)
{
    uint32_t cnt = 0, sum = 0;
    const uintptr_t a0 = c0 & ~static_cast<uintptr_t>(15);
    // the 4 bytes before the first unit
    uint32_t last = 0;
    if (lane == 0) last = load_slice(a0 - 16, a0 - 16 >= lo && a0 <= hi, lo, hi).w;
    for (uintptr_t g = a0; g < c1; g += kUnits * kUnit) {
        uint4 w[kUnits];
#pragma unroll
        for (int u = 0; u < kUnits; ++u) {
            const uintptr_t va = g + u * kUnit + lane * kBPT;
            w[u] = va < c1 ? load_slice(va, va >= lo && va + kBPT <= hi, lo, hi) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kUnits; ++u) {
            uint32_t wp = __shfl_up_sync(~0u, w[u].w, 1);
            if (lane == 0) wp = last;
            last = __shfl_sync(~0u, w[u].w, kLanes - 1);
            const uintptr_t va = g + u * kUnit + lane * kBPT;
            const uint32_t tl = term4(w[u].x) | (term4(w[u].y) << 4) | (term4(w[u].z) << 8) | (term4(w[u].w) << 12);
            const uint32_t t20 = term4(wp) | (tl << 4);
            const bool own = va >= c0 && va + kBPT <= c1;
            const uint32_t tc = own ? tl : (tl & slice_valid(va, c0, c1));
            cnt += __popc(tc);
            if (kDelta) {
                const uint32_t c20 = ~t20 & 0xFFFFFu;
                if (own && !(c20 & (c20 << 1) & 0xFFFF8u))
                    sum += sum_le2_fast(w[u], wp);
                else if (own)
                    sum += sum_any_fast(w[u], wp, tl, t20);
                else
                    assemble_regs(wp, w[u], tl, t20, tc, [&](uint32_t v) { sum += v; });
            }
        }
    }
    cnt_out = __reduce_add_sync(~0u, cnt);
    sum_out = kDelta ? __reduce_add_sync(~0u, sum) : 0u;
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads) lists_count_kernel(const LParams p)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t nci = p.ncl ? p.cfirst[p.ncl] : 0u;
    const uintptr_t base = reinterpret_cast<uintptr_t>(p.in);
    for (uint32_t e = gw; e < nci; e += nwarps) {
        const uint32_t i = p.citem[e];
        const Item it = p.items[i];
        uint32_t c, s;
        count_range<kDelta>(base + it.b0, base + it.b1, base + p.bo[it.list], base + p.bo[it.list + 1], lane, c, s);
        if (lane == 0) p.cs[i] = make_uint2(c, s);
    }
}

// One warp per chunked list: the count and sum of each chunk's earlier
// chunks, and the list's count against its value offsets.
__global__ void __launch_bounds__(kThreads) lists_scan_kernel(const LParams p)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (uint32_t c = gw; c < p.ncl; c += nwarps) {
        const uint32_t e0 = p.cfirst[c], e1 = p.cfirst[c + 1];
        uint32_t cc = 0, cx = 0;
        for (uint32_t b = e0; b < e1; b += kLanes) {
            const uint32_t e = b + lane;
            const uint2 v = e < e1 ? p.cs[p.citem[e]] : make_uint2(0u, 0u);
            const uint32_t ic = warp_incl_scan(v.x, lane), is = warp_incl_scan(v.y, lane);
            if (e < e1) p.rel[p.citem[e]] = make_uint2(cc + ic - v.x, cx + is - v.y);
            cc += __shfl_sync(~0u, ic, 31);
            cx += __shfl_sync(~0u, is, 31);
        }
        if (lane == 0) {
            const uint32_t j = p.items[p.citem[e0]].list;
            if (cc != p.vo[j + 1] - p.vo[j]) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
        }
    }
}

template <bool kDelta, bool kTable = false>
__global__ void __launch_bounds__(kThreads, 5) lists_decode_kernel(const LParams p)
{
    extern __shared__ __align__(16) unsigned char lsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &M = reinterpret_cast<WarpSmem *>(lsm)[warp];
    TableSmem &Tb = *reinterpret_cast<TableSmem *>(lsm + (blockDim.x >> 5) * sizeof(WarpSmem));
    if (kTable) {
        fill_table(Tb);
        __syncthreads();
    }
    if (lane < kRing) *reinterpret_cast<uint4 *>(M.ring[lane] + kHalo + kUnit) = make_uint4(0u, 0u, 0u, 0u);
    const uintptr_t base = reinterpret_cast<uintptr_t>(p.in);
    const uint32_t ow = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
    (void)ow;
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(p.queue, 1u);
        i = __shfl_sync(~0u, i, 0);
        if (i >= p.nitems) break;
        const Item it = p.items[i];
        const uint2 r = p.rel[i];
        const uint32_t j = it.list;
        unsigned long long R = p.vo[j] + r.x;
        uint32_t X = (kDelta && p.prevs ? p.prevs[j] : 0u) + r.y;
        const uintptr_t c0 = base + it.b0, c1 = base + it.b1;
        const uintptr_t lo = base + p.bo[j], hi = base + p.bo[j + 1];
        const uintptr_t a0 = c0 & ~static_cast<uintptr_t>(15);
        const uint32_t K = c1 > c0 ? static_cast<uint32_t>((c1 - a0 + kUnit - 1) / kUnit) : 0u;
        auto issue = [&](uint32_t k) {
            if (k < K) {
                const uintptr_t ua = a0 + static_cast<uintptr_t>(k) * kUnit;
                stage_unit(ua, lane, M.ring[k % kRing], lo, hi, ua - 16 >= lo && ua + kUnit <= hi);
            }
            cp_async_commit();
        };
        issue(0);
        issue(1);
        for (uint32_t k = 0; k < K; ++k) {
            cp_async_wait_prior<1>();
            __syncwarp();
            issue(k + 2);
            const uint8_t *ub = M.ring[k % kRing];
            const uintptr_t ua = a0 + static_cast<uintptr_t>(k) * kUnit;
            const bool in = ua >= c0 && ua + kUnit <= c1 && ua - 16 >= lo;
            uint32_t wc, ws;
            bool one;
            unit_stage<kDelta, true, kTable>(ub, in, ua, c0, c1, M.vals, lane, wc, ws, one, p.status,
                                             (it.flags & kLast) ? hi : 0, Tb.T, Tb.D);
            __syncwarp();
            // the output's end: this list's last value (a count beyond it is an error)
            Params q;
            q.out = p.out;
            q.n = p.vo[j + 1];
            unit_emit<kDelta, false>(q, ub, M.vals, one, wc, R, X, lane);
            R += wc;
            X += ws;
            __syncwarp();
        }
        cp_async_wait_all();
        if (lane == 0 && (it.flags & kOnly) && R != p.vo[j + 1]) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
    }
}

// ---- host

size_t lists_smem(int warps_per_cta, bool table)
{
    return warps_per_cta * sizeof(WarpSmem) + (table ? sizeof(TableSmem) : 0);
}

int lists_occupancy(int warps_per_cta, bool table)
{
    int occ = 0;
    if (table)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lists_decode_kernel<true, true>, warps_per_cta * kLanes,
                                                      lists_smem(warps_per_cta, true));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lists_decode_kernel<true>, warps_per_cta * kLanes,
                                                      lists_smem(warps_per_cta, false));
    return occ > 0 ? occ : 1;
}

struct Layout {
    size_t ent, ctot, cpre, ent4, ctot4, cpre4, total;
};

uint64_t wtiles_for(uintptr_t addr, size_t nbytes) { return nbytes ? ((addr & 15u) + nbytes + kWT - 1) / kWT : 0; }

uint32_t max_ranges(uint64_t nwt)
{
    return static_cast<uint32_t>(std::min<uint64_t>(nwt, kMaxRanges + nwt / kMaxT));
}

// d4: with the per-class arrays of blocked differences.
Layout layout(uint64_t nwt, uint64_t G, bool d4)
{
    Layout L;
    L.ent = 256;   // after the status head
    L.ctot = (L.ent + 8 * nwt + 15) / 16 * 16;
    L.cpre = (L.ctot + 8 * G + 15) / 16 * 16;
    L.ent4 = L.cpre + 16 * G;
    L.ctot4 = L.ent4 + (d4 ? 16 * nwt : 0);
    L.cpre4 = L.ctot4 + (d4 ? 16 * G : 0);
    L.total = L.cpre4 + (d4 ? 16 * G : 0);
    return L;
}

struct Dev {
    int sms = 0;
    int occ = 0;    // resident CTAs per SM of decode_kernel (the count launch's ranges follow it)
    int occ2 = 0;   // ... of decode2_kernel
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ, decode_kernel<true, false>, kThreads, 0);
        d.occ = std::max(d.occ, 1);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ2, decode2_kernel<true, false>, kThreads2, 0);
        d.occ2 = std::max(d.occ2, 1);
    }
    *out = d;
    return VBYTE_OK;
}

// The stream decode launch over warp tiles [tb, te): persistent CTAs, at
// most one wave.
template <bool kDelta, bool kRank>
void launch_decode2(const Params &p, const Dev &di, uint64_t tb, uint64_t te, cudaStream_t s)
{
    if (te <= tb) return;
    const uint64_t want = (te - tb + kW2 - 1) / kW2;
    const unsigned g = static_cast<unsigned>(std::min<uint64_t>(want, static_cast<uint64_t>(di.sms) * di.occ2));
    decode2_kernel<kDelta, kRank><<<g, kThreads2, 0, s>>>(p, tb, te);
}

}  // namespace sp

size_t split_workspace_bytes(const uint8_t *in, size_t nbytes)
{
    const uint64_t nwt = sp::wtiles_for(reinterpret_cast<uintptr_t>(in), nbytes);
    return sp::layout(nwt, sp::max_ranges(nwt), true).total;
}

int enqueue_list_plan(const BatchArgs &a, const ListPlan &lp, int warps_per_cta, uint32_t *status, cudaStream_t s,
                      bool table)
{
    if (warps_per_cta != 4 && warps_per_cta != 8) return VBYTE_EINVAL;
    sp::Dev di;
    int rc = sp::dev_info(&di);
    if (rc != VBYTE_OK) return rc;
    sp::LParams p = {};
    p.in = a.in;
    p.out = a.out;
    p.bo = a.bo;
    p.vo = a.vo;
    p.prevs = a.delta ? a.prevs : nullptr;
    p.items = lp.items;
    p.nitems = lp.nitems;
    p.citem = lp.citem;
    p.cfirst = lp.cfirst;
    p.ncl = lp.ncl;
    p.cs = lp.cs;
    p.rel = lp.rel;
    p.queue = lp.queue;
    p.status = status;
    if (cudaMemsetAsync(lp.queue, 0, sizeof(unsigned int), s) != cudaSuccess) return VBYTE_ECUDA;
    if (lp.ncl) {
        const unsigned g = static_cast<unsigned>(std::max(1, di.sms * 4));
        if (a.delta)
            sp::lists_count_kernel<true><<<g, sp::kThreads, 0, s>>>(p);
        else
            sp::lists_count_kernel<false><<<g, sp::kThreads, 0, s>>>(p);
        const unsigned gs = static_cast<unsigned>((lp.ncl + sp::kWarps - 1) / sp::kWarps);
        sp::lists_scan_kernel<<<gs, sp::kThreads, 0, s>>>(p);
    }
    const int occ = sp::lists_occupancy(warps_per_cta, table);
    const unsigned g = static_cast<unsigned>(std::min<uint64_t>(static_cast<uint64_t>(di.sms) * occ,
                                                                (lp.nitems + warps_per_cta - 1) / warps_per_cta));
    const size_t smem = sp::lists_smem(warps_per_cta, table);
    const unsigned nt = static_cast<unsigned>(warps_per_cta * sp::kLanes);
    if (g) {
        if (table && a.delta)
            sp::lists_decode_kernel<true, true><<<g, nt, smem, s>>>(p);
        else if (table)
            sp::lists_decode_kernel<false, true><<<g, nt, smem, s>>>(p);
        else if (a.delta)
            sp::lists_decode_kernel<true><<<g, nt, smem, s>>>(p);
        else
            sp::lists_decode_kernel<false><<<g, nt, smem, s>>>(p);
    }
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

// ---- decoding from host buffers, pipelined
//
// The input is cut into pieces of whole ranges (R ranges of T warp tiles).
// A copy stream moves the pieces to the device one after another; the
// compute stream counts each piece once its bytes (and the 16 before) are
// there, scans its ranges from the carry of the pieces before it, decodes it,
// and records how many values precede the next piece; the host reads that and
// queues the piece's values back on a third stream as soon as they are
// decoded.  Copies in the two directions and the kernels overlap.

namespace {
struct PipeStreams {
    cudaStream_t up = nullptr, work = nullptr, down = nullptr;
    std::vector<cudaEvent_t> ev;
    unsigned long long *h_after = nullptr;   // pinned: values after each piece
    size_t pieces = 0;
};
std::mutex g_pipe_mu;
std::map<std::pair<int, uintptr_t>, PipeStreams> g_pipe;

int pipe_streams(cudaStream_t s, size_t pieces, PipeStreams **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    PipeStreams &P = g_pipe[{dev, reinterpret_cast<uintptr_t>(s)}];
    if (!P.up) {
        if (cudaStreamCreateWithFlags(&P.up, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&P.work, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&P.down, cudaStreamNonBlocking) != cudaSuccess)
            return VBYTE_ECUDA;
    }
    while (P.ev.size() < 3 * pieces + 3) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return VBYTE_ECUDA;
        P.ev.push_back(e);
    }
    if (P.pieces < pieces) {
        if (P.h_after) cudaFreeHost(P.h_after);
        P.h_after = nullptr;
        if (cudaMallocHost(&P.h_after, pieces * sizeof(unsigned long long)) != cudaSuccess) return VBYTE_ENOMEM;
        P.pieces = pieces;
    }
    *out = &P;
    return VBYTE_OK;
}
}  // namespace

size_t pipe_workspace_bytes(size_t nbytes)
{
    // ranges of at least one tile: an ent word per tile, ctot and cpre per range, the carry
    const uint64_t nwt = sp::wtiles_for(15, nbytes);
    return 256 + 8 * nwt + 16 + 24 * nwt + 64;
}

int decode_host_pipelined(const uint8_t *h_in, size_t nbytes, uint32_t *h_out, size_t n, bool delta, uint32_t prev,
                          uint8_t *d_in, uint32_t *d_out, uint8_t *ws, uint32_t *status, cudaStream_t s,
                          size_t piece_bytes)
{
    sp::Dev di;
    int rc = sp::dev_info(&di);
    if (rc != VBYTE_OK) return rc;
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_in);
    const uint64_t nwt = sp::wtiles_for(a, nbytes);
    const uint64_t R = static_cast<uint64_t>(di.sms) * di.occ;                  // ranges per piece
    const uint64_t T = std::max<uint64_t>(1, std::min<uint64_t>(sp::kMaxT, piece_bytes / sp::kWT / R));
    const uint64_t TP = T * R;                                                   // warp tiles per piece
    const uint64_t K = (nwt + TP - 1) / TP;                                      // pieces
    const uint64_t G = (nwt + T - 1) / T;
    PipeStreams *P = nullptr;
    if ((rc = pipe_streams(s, K, &P)) != VBYTE_OK) return rc;
    // workspace: ent per tile, ctot and cpre per range, the carry
    uint8_t *w = ws + 256;
    uint2 *ent = reinterpret_cast<uint2 *>(w);
    uint2 *ctot = reinterpret_cast<uint2 *>(w + (8 * nwt + 15) / 16 * 16);
    uint4 *cpre = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(ctot) + (8 * G + 15) / 16 * 16);
    unsigned long long *carry = reinterpret_cast<unsigned long long *>(cpre + G);
    sp::Params p = {};
    p.in = d_in;
    p.nbytes = nbytes;
    p.out = d_out;
    p.n = n;
    p.base = a & ~static_cast<uintptr_t>(15);
    p.nwt = nwt;
    p.in_lo = p.base == a ? 0u : 1u;
    p.in_hi = (a + nbytes - p.base) / sp::kWT;
    p.T = static_cast<uint32_t>(T);
    p.G = static_cast<uint32_t>(G);
    p.ent = ent;
    p.ctot = ctot;
    p.cpre = cpre;
    p.status = status;
    p.prev = prev;
    cudaEvent_t start = P->ev[3 * K], end_work = P->ev[3 * K + 1], end_down = P->ev[3 * K + 2];
    if (cudaEventRecord(start, s) != cudaSuccess) return VBYTE_ECUDA;
    for (cudaStream_t x : {P->up, P->work, P->down})
        if (cudaStreamWaitEvent(x, start, 0) != cudaSuccess) return VBYTE_ECUDA;
    // the input, piece by piece (piece i: its tiles, clipped to the input)
    const uint64_t skew = a - p.base;
    for (uint64_t i = 0; i < K; ++i) {
        const uint64_t b0 = i == 0 ? 0 : i * TP * sp::kWT - skew;
        const uint64_t b1 = std::min<uint64_t>(nbytes, (i + 1) * TP * sp::kWT - skew);
        if (b1 > b0 && cudaMemcpyAsync(d_in + b0, h_in + b0, b1 - b0, cudaMemcpyHostToDevice, P->up) != cudaSuccess)
            return VBYTE_ECUDA;
        if (cudaEventRecord(P->ev[i], P->up) != cudaSuccess) return VBYTE_ECUDA;
    }
    // count, scan and decode each piece once its bytes (and those before) are there
    for (uint64_t i = 0; i < K; ++i) {
        const uint64_t r0 = i * R, r1 = std::min<uint64_t>(G, (i + 1) * R);
        if (cudaStreamWaitEvent(P->work, P->ev[i], 0) != cudaSuccess) return VBYTE_ECUDA;
        p.range0 = static_cast<uint32_t>(r0);
        const unsigned g = static_cast<unsigned>(r1 - r0);
        if (delta)
            sp::count_kernel<true, false><<<g, sp::kThreads, 0, P->work>>>(p);
        else
            sp::count_kernel<false, false><<<g, sp::kThreads, 0, P->work>>>(p);
        sp::scan_piece_kernel<<<1, sp::kScanThreads, 0, P->work>>>(p, static_cast<uint32_t>(r1), carry, i == 0,
                                                                   i + 1 == K);
        if (cudaMemcpyAsync(P->h_after + i, carry, 8, cudaMemcpyDeviceToHost, P->work) != cudaSuccess)
            return VBYTE_ECUDA;
        if (cudaEventRecord(P->ev[K + i], P->work) != cudaSuccess) return VBYTE_ECUDA;
        const uint64_t tb = r0 * p.T, te = std::min<uint64_t>(r1 * p.T, p.nwt);
        if (delta)
            sp::launch_decode2<true, false>(p, di, tb, te, P->work);
        else
            sp::launch_decode2<false, false>(p, di, tb, te, P->work);
        if (cudaEventRecord(P->ev[2 * K + i], P->work) != cudaSuccess) return VBYTE_ECUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return VBYTE_ECUDA;
    // each piece's values back as soon as they are decoded
    unsigned long long before = 0;
    for (uint64_t i = 0; i < K; ++i) {
        if (cudaEventSynchronize(P->ev[K + i]) != cudaSuccess) return VBYTE_ECUDA;
        const unsigned long long after = std::min<unsigned long long>(P->h_after[i], n);
        if (cudaStreamWaitEvent(P->down, P->ev[2 * K + i], 0) != cudaSuccess) return VBYTE_ECUDA;
        if (after > before &&
            cudaMemcpyAsync(h_out + before, d_out + before, (after - before) * 4, cudaMemcpyDeviceToHost, P->down) !=
                cudaSuccess)
            return VBYTE_ECUDA;
        before = std::max(before, after);
    }
    if (cudaEventRecord(end_work, P->work) != cudaSuccess || cudaStreamWaitEvent(s, end_work, 0) != cudaSuccess ||
        cudaEventRecord(end_down, P->down) != cudaSuccess || cudaStreamWaitEvent(s, end_down, 0) != cudaSuccess)
        return VBYTE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

size_t split_workspace_bound(size_t nbytes)
{
    const uint64_t nwt = sp::wtiles_for(15, nbytes);   // the worst alignment
    return sp::layout(nwt, sp::max_ranges(nwt), true).total;
}

int enqueue_split(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                  uint8_t *ws, uint32_t *status, cudaStream_t s, bool rank, const uint32_t *prev4, bool table)
{
    if (rank && !delta) return VBYTE_EINVAL;
    const bool d4 = prev4 != nullptr;
    if (d4 && (delta || rank)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) & 15u) return VBYTE_EINVAL;
    sp::Dev di;
    int rc = sp::dev_info(&di);
    if (rc != VBYTE_OK) return rc;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    const uint64_t nwt = sp::wtiles_for(a, nbytes);
    // ranges: about one per resident CTA, at most kMaxT tiles each
    const uint64_t target = static_cast<uint64_t>(di.sms) * di.occ;
    uint64_t T = std::max<uint64_t>(1, (nwt + target - 1) / target);
    T = std::min<uint64_t>(T, sp::kMaxT);
    const uint64_t G = (nwt + T - 1) / T;
    if (G > sp::max_ranges(nwt) || nwt >= (uint64_t(1) << 32)) return VBYTE_EINVAL;   // 32-bit tile indices
    const sp::Layout L = sp::layout(nwt, G, d4);
    sp::Params p = {};
    p.in = in;
    p.nbytes = nbytes;
    p.out = out;
    p.n = n;
    p.base = a & ~static_cast<uintptr_t>(15);
    p.nwt = nwt;
    p.in_lo = p.base == a ? 0u : 1u;
    p.in_hi = (a + nbytes - p.base) / sp::kWT;
    p.T = static_cast<uint32_t>(T);
    p.G = static_cast<uint32_t>(G);
    p.ent = reinterpret_cast<uint2 *>(ws + L.ent);
    p.ctot = reinterpret_cast<uint2 *>(ws + L.ctot);
    p.cpre = reinterpret_cast<uint4 *>(ws + L.cpre);
    p.status = status;
    p.prev = prev;
    if (d4) {
        p.prev4 = make_uint4(prev4[0], prev4[1], prev4[2], prev4[3]);
        p.ent4 = reinterpret_cast<uint4 *>(ws + L.ent4);
        p.ctot4 = reinterpret_cast<uint4 *>(ws + L.ctot4);
        p.cpre4 = reinterpret_cast<uint4 *>(ws + L.cpre4);
        const unsigned dg = static_cast<unsigned>(G);
        sp::count_kernel<false, true><<<dg, sp::kThreads, 0, s>>>(p);
        sp::scan4_kernel<<<1, sp::kScanThreads, 0, s>>>(p);
        sp::decode_kernel<false, false, true><<<dg, sp::kThreads, 0, s>>>(p);
        return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
    }
    if (delta)
        sp::count_kernel<true, false><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    else
        sp::count_kernel<false, false><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    sp::scan_kernel<<<1, sp::kScanThreads, 0, s>>>(p);
    const unsigned g = static_cast<unsigned>(G);
    if (rank)   // the gaps-minus-one variant: no table-driven instance
        sp::launch_decode2<true, true>(p, di, 0, nwt, s);
    else if (table && delta)
        sp::decode_kernel<true, false, false, true><<<g, sp::kThreads, sizeof(sp::TableSmem), s>>>(p);
    else if (table)
        sp::decode_kernel<false, false, false, true><<<g, sp::kThreads, sizeof(sp::TableSmem), s>>>(p);
    else if (delta)
        sp::launch_decode2<true, false>(p, di, 0, nwt, s);
    else
        sp::launch_decode2<false, false>(p, di, 0, nwt, s);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace vbk
