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
//     the stream; it is four 512-byte units, one 16-byte slice per lane.
//   * CTA c of the count and the decode launch owns the contiguous warp
//     tiles [c T, (c + 1) T); its warps take every eighth tile.
//   * count: per warp tile, its integers and (delta) their sum -- a popc of
//     the terminator mask and, for the sum, the byte-weight formula for codes
//     of at most two bytes or per-integer assembly.  The CTA scans its range
//     in shared memory and writes, per tile, the count and sum of the range's
//     tiles before it, and the range's totals.  The data-error contract is
//     checked here.
//   * scan: one CTA turns the range totals into each range's prefix: values
//     before it and the running x before it (from prev).
//   * decode: every warp on its own.  Its units travel through a ring of
//     three shared-memory buffers with cp.async (two units ahead), each unit
//     is decoded into the warp's value buffer (one-byte units stay as bytes)
//     and written out with coalesced 16-byte stores.  No CTA barrier after
//     the start, no wait on another CTA.
// The input is read twice (count, decode); the per-tile words add 8 bytes per
// 2 KiB.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "vbyte.h"
#include "vbyte_device.cuh"
#include "vbyte_emit.cuh"
#include "vbyte_internal.h"

namespace vbk {
namespace sp {

constexpr int kLanes = 32;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * kLanes;
constexpr int kUnit = kLanes * kBPT;            // 512 bytes per warp step
constexpr int kUnits = 4;                       // units per warp tile
constexpr int kWT = kUnit * kUnits;             // 2 KiB warp tile
constexpr uint32_t kMaxT = 1024;                // warp tiles per CTA range
constexpr int kRing = 3;                        // unit buffers per warp
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
    uint2 *ent;         // per warp tile: (count, sum) before it within its range
    uint2 *ctot;        // per range: (count, sum) of the range
    uint4 *cpre;        // per range: values before it (lo, hi), running x before it, 0
    uint32_t *status;
    uint32_t prev;      // x_0
};

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

// One warp: the integers of warp tile t and (delta) their sum.
template <bool kDelta>
__device__ __forceinline__ void count_wt(const Params &p, uint64_t t, int lane, uint32_t &cnt_out, uint32_t &sum_out)
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
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
        uint32_t wp = __shfl_up_sync(~0u, w[u].w, 1);
        const uint32_t last = (u == 0) ? before : __shfl_sync(~0u, w[u - 1].w, kLanes - 1);
        if (lane == 0) wp = last;
        const uintptr_t va = w0 + u * kUnit + lane * kBPT;
        const uint32_t tl = term4(w[u].x) | (term4(w[u].y) << 4) | (term4(w[u].z) << 8) | (term4(w[u].w) << 12);
        const uint32_t t20 = term4(wp) | (tl << 4);
        const uint32_t tc = in ? tl : (tl & slice_valid(va, lo, hi));
        cnt += __popc(tc);
        const uint32_t c20 = ~t20 & 0xFFFFFu;
        if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
            atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
        if (t == p.nwt - 1 && hi - 1 >= va && hi - 1 < va + kBPT && !((tl >> (hi - 1 - va)) & 1u))
            atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        if (kDelta) {
            // codes of at most two bytes, codes in separate words, any codes
            // (warp-uniform choices), per-integer assembly at the stream's ends
            const bool le2 = !(c20 & (c20 << 1) & 0xFFFF8u);
            if (in && __all_sync(~0u, le2))
                sum += sum_le2_fast(w[u], wp);
            else if (in && !__any_sync(~0u, dense_words(tl)))
                assemble_words(wp, w[u], tl, t20, [&](uint32_t v) { sum += v; });
            else if (in)
                sum += sum_any_fast(w[u], wp, tl, t20);
            else
                assemble_regs(wp, w[u], tl, t20, tc, [&](uint32_t v) { sum += v; });
        }
    }
    cnt_out = __reduce_add_sync(~0u, cnt);
    sum_out = kDelta ? __reduce_add_sync(~0u, sum) : 0u;
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads, 5) count_kernel(const Params p)
{
    __shared__ uint2 E[kMaxT];
    __shared__ uint32_t wcnt[kWarps], wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t t0 = static_cast<uint64_t>(blockIdx.x) * p.T;
    const uint32_t nt = static_cast<uint32_t>(min(static_cast<uint64_t>(p.T), p.nwt - t0));
    for (uint32_t i = warp; i < nt; i += kWarps) {
        uint32_t c, s;
        count_wt<kDelta>(p, t0 + i, lane, c, s);
        if (lane == 0) E[i] = make_uint2(c, s);
    }
    __syncthreads();
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
    if (tid == 0) p.ctot[blockIdx.x] = make_uint2(tc, ts);
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

// ---- decode (every warp on its own)

struct WarpSmem {
    alignas(16) uint8_t ring[kRing][kSlot];   // units staged with their 16 bytes before
    alignas(16) uint32_t vals[kVal];          // a unit's values at rank + 4
};
static_assert(sizeof(WarpSmem) % 16 == 0 && kSlot % 16 == 0, "unit buffers keep 16-byte alignment");

// Stage unit u of warp tile t into `slot` (the 16 bytes before the unit at
// slot[0..16), the unit at slot[16..528)); bytes outside the stream as zero.
// The caller commits.
__device__ __forceinline__ void issue_unit(const Params &p, uint64_t t, int u, int lane, uint8_t *slot)
{
    const uintptr_t ua = p.base + (static_cast<uintptr_t>(t) << 11) + u * kUnit;
    const uintptr_t va = ua + lane * kBPT;
    uint8_t *dst = slot + kHalo + lane * kBPT;
    if (interior(p, t) && (t > 0 || u > 0)) {   // the unit and the 16 bytes before it are inside
        cp_async16(dst, reinterpret_cast<const void *>(va));
        if (lane == 0) cp_async16(slot, reinterpret_cast<const void *>(ua - 16));
        return;
    }
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
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

// One warp: decode the staged unit ub into vals (warp rank r at vals[4 + r];
// delta: running sums from the unit's first value).  Returns the unit's
// value count and sum; one = every slice holds one-byte integers only (the
// values stay as bytes and vals is untouched).
template <bool kDelta>
__device__ __forceinline__ void unit_stage(const uint8_t *ub, bool in, uintptr_t ua, uintptr_t lo, uintptr_t hi,
                                           uint32_t *vals, int lane, uint32_t &wc, uint32_t &ws, bool &one)
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
    const uint32_t inc = warp_incl_scan(cnt, lane);
    wc = __shfl_sync(~0u, inc, 31);
    uint32_t *dst = vals + 4 + inc - cnt;
    uint32_t vsum = 0;
    if (!__any_sync(~0u, notB)) {
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
        // longer codes: each value assembled once (one fixed step per word
        // when no word holds two terminators), then running sums from this
        // lane's offset within the unit
        if (in && !__any_sync(~0u, dense_words(m.tl)))
            assemble_words(m.wprev, m.w, m.tl, m.t20, [&](uint32_t v) {
                *dst++ = v;
                vsum += v;
            });
        else
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

template <bool kDelta, bool kRank>
__global__ void __launch_bounds__(kThreads, 5) decode_kernel(const Params p)
{
    __shared__ WarpSmem Wsm[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpSmem &M = Wsm[warp];
    if (lane < kRing) *reinterpret_cast<uint4 *>(M.ring[lane] + kHalo + kUnit) = make_uint4(0u, 0u, 0u, 0u);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uint64_t t0 = static_cast<uint64_t>(blockIdx.x) * p.T;
    const uint32_t nt = static_cast<uint32_t>(min(static_cast<uint64_t>(p.T), p.nwt - t0));
    const uint32_t mine = nt > static_cast<uint32_t>(warp) ? (nt - warp + kWarps - 1) / kWarps : 0u;
    const uint32_t K = mine * kUnits;   // units of this warp: tiles warp, warp + 8, ... of the range
    const uint4 cp = p.cpre[blockIdx.x];
    const unsigned long long C0 = cp.x | (static_cast<unsigned long long>(cp.y) << 32);
    auto issue = [&](uint32_t k) {
        if (k < K) issue_unit(p, t0 + warp + (k / kUnits) * kWarps, static_cast<int>(k % kUnits), lane,
                              M.ring[k % kRing]);
        cp_async_commit();
    };
    issue(0);
    issue(1);
    unsigned long long R = 0;
    uint32_t X = 0;
    uint2 e_next = make_uint2(0u, 0u);
    if (K) e_next = p.ent[t0 + warp];
    for (uint32_t k = 0; k < K; ++k) {
        cp_async_wait_prior<1>();   // unit k has landed (for this lane)
        __syncwarp();               // ... for every lane
        issue(k + 2);
        const uint32_t u = k % kUnits;
        const uint64_t t = t0 + warp + (k / kUnits) * kWarps;
        if (u == 0) {
            R = C0 + e_next.x;
            X = cp.z + e_next.y;
            if (k + kUnits < K) e_next = p.ent[t + kWarps];   // the next tile's prefix travels meanwhile
        }
        const uint8_t *ub = M.ring[k % kRing];
        const uintptr_t ua = p.base + (static_cast<uintptr_t>(t) << 11) + u * kUnit;
        uint32_t wc, ws;
        bool one;
        unit_stage<kDelta>(ub, interior(p, t), ua, lo, hi, M.vals, lane, wc, ws, one);
        __syncwarp();
        unit_emit<kDelta, kRank>(p, ub, M.vals, one, wc, R, X, lane);
        R += wc;
        X += ws;
        __syncwarp();   // the value buffer and this unit's slot are free again
    }
    cp_async_wait_all();
}

// ---- host

struct Layout {
    size_t ent, ctot, cpre, total;
};

uint64_t wtiles_for(uintptr_t addr, size_t nbytes) { return nbytes ? ((addr & 15u) + nbytes + kWT - 1) / kWT : 0; }

uint32_t max_ranges(uint64_t nwt)
{
    return static_cast<uint32_t>(std::min<uint64_t>(nwt, kMaxRanges + nwt / kMaxT));
}

Layout layout(uint64_t nwt, uint64_t G)
{
    Layout L;
    L.ent = 256;   // after the status head
    L.ctot = (L.ent + 8 * nwt + 15) / 16 * 16;
    L.cpre = (L.ctot + 8 * G + 15) / 16 * 16;
    L.total = L.cpre + 16 * G;
    return L;
}

struct Dev {
    int sms = 0;
    int occ = 0;
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
    }
    *out = d;
    return VBYTE_OK;
}

}  // namespace sp

size_t split_workspace_bytes(const uint8_t *in, size_t nbytes)
{
    const uint64_t nwt = sp::wtiles_for(reinterpret_cast<uintptr_t>(in), nbytes);
    return sp::layout(nwt, sp::max_ranges(nwt)).total;
}

size_t split_workspace_bound(size_t nbytes)
{
    const uint64_t nwt = sp::wtiles_for(15, nbytes);   // the worst alignment
    return sp::layout(nwt, sp::max_ranges(nwt)).total;
}

int enqueue_split(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                  uint8_t *ws, uint32_t *status, cudaStream_t s, bool rank)
{
    if (rank && !delta) return VBYTE_EINVAL;
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
    if (G > sp::max_ranges(nwt)) return VBYTE_EINVAL;
    const sp::Layout L = sp::layout(nwt, G);
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
    if (delta)
        sp::count_kernel<true><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    else
        sp::count_kernel<false><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    sp::scan_kernel<<<1, sp::kScanThreads, 0, s>>>(p);
    if (rank)
        sp::decode_kernel<true, true><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    else if (delta)
        sp::decode_kernel<true, false><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    else
        sp::decode_kernel<false, false><<<static_cast<unsigned>(G), sp::kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace vbk
