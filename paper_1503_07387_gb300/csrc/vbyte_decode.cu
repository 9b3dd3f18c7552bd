// libvbyte: single-pass GPU decoder for VByte-coded uint32 streams (sm_103a).
//
// Operation (arXiv 1503.07387): the result of Algorithm 1 (Sec. 2) on the
// byte stream -- seven data bits per byte, least significant group first,
// high bit set on every byte of an integer except its last (Sec. 1, Table 1)
// -- optionally followed by the prefix sum that undoes differential coding
// (Sec. 1 "Differential coding", Sec. 4 "Differential Coding").
//
// GPU design (one kernel, one pass over the input, persistent CTAs that take
// tiles from an atomic counter and prefetch the next tile while decoding):
//   (a) terminator mask + slot assignment.  A tile is 4 KiB of input aligned
//       to 16 bytes in absolute address space.  Each thread loads 16 bytes
//       with one vector load, forms a 16-bit mask of terminator bytes (high
//       bit clear -- the GPU counterpart of pmovmskb in Sec. 3/4) and counts
//       them; a block scan gives every thread its first rank inside the tile.
//       A tile owns exactly the integers whose terminator byte lies inside
//       it; the 16 bytes before the tile are staged too, so an integer that
//       starts up to four bytes before the tile is assembled by the tile
//       holding its terminator.
//   (b) value assembly.  Integers are assembled branch-free from the (up to)
//       five bytes ending at their terminator.  The work is split by the
//       longest code in the tile, the GPU counterpart of the paper's case
//       split on the 12-bit mask (Sec. 4): class A (every byte a terminator:
//       values are the bytes themselves), class B (codes of at most two
//       bytes: a SWAR byte-pair merge over 4-byte words) and class C (any
//       length: per-terminator assembly from shared memory).  Values are
//       staged in shared memory at their tile rank.
//   (c) fused delta prefix sum.  Staged gaps are scanned in place (four
//       consecutive values per thread, then a warp scan), and the per-warp
//       totals give each (round, warp) entry its offset inside the tile.
//   The tile's exclusive (count, gap sum) prefix comes from a two-level
//   decoupled look-back (tiles grouped 32 at a time through atomic group
//   accumulators), seeded with `prev`.  Output leaves in 16-byte aligned
//   quads; the alignment shift is applied with one lane shuffle, and every
//   write is clamped to [0, n).
//
// Every cross-tile wait is bounded by the global timer (about two seconds);
// on expiry the status word gets VBYTE_ERR_TIMEOUT and the kernel carries on.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "vbyte.h"

namespace vbk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBPT = 16;                      // input bytes per thread
constexpr int kTile = kThreads * kBPT;        // input bytes per tile (4 KiB)
constexpr int kHalo = 16;                     // bytes staged before the tile
constexpr int kRoundVals = kThreads * 4;      // values per copy-out round
constexpr int kGroup = 32;                    // tiles per look-back group

constexpr uint64_t kStateAgg = 1ull << 62;    // descriptor holds the tile aggregate
constexpr uint64_t kStateIncl = 2ull << 62;   // descriptor holds the inclusive prefix
constexpr uint64_t kPayload = (1ull << 62) - 1;
constexpr uint64_t kMask48 = (1ull << 48) - 1;
constexpr uint64_t kWaitLimitNs = 2000000000ull;

enum : uint32_t { kClassA = 0, kClassB = 1, kClassC = 2 };

struct Params {
    const uint8_t *in;
    uint64_t nbytes;
    uint32_t *out;
    uint64_t n;
    uint64_t ntiles;
    uintptr_t base;            // 16-byte aligned address of tile 0
    uint64_t *tdesc;           // per tile: [state|count], [state|gap sum]
    unsigned long long *gacc;  // per group: atomic (contributors << 48 | count), (... | sum)
    uint64_t *gdesc;           // per group: [state|count], [state|gap sum]
    unsigned long long *ctr;   // dynamic tile counter
    uint32_t *status;          // data-error bits
    uint32_t prev;             // x_0 for differential decoding
};

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ uint4 ld_stream16(const void *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_quad(uint32_t *p, uint4 v)
{
    asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// Bit i of the result is 1 iff byte i of w has its high bit clear (a
// terminator).  The multiply moves bits 7, 15, 23, 31 to bits 28..31; the
// other partial products land on distinct lower bits, so nothing carries.
__device__ __forceinline__ uint32_t term4(uint32_t w)
{
    return ((~w & 0x80808080u) * 0x00204081u) >> 28;
}

// Value of an integer of L bytes (1..5) whose terminator byte is x and whose
// preceding four stream bytes are lo4 (byte q-4 in bits 0..7).  The 7-bit
// groups of lo4 are compacted into 28 bits, x is put on top (a 35-bit
// number), and the groups that belong to earlier integers fall off the low
// end with one funnel shift.  For L = 5 the top of x lands above bit 31 and is
// dropped: Algorithm 1's b * 2^28 modulo 2^32.
__device__ __forceinline__ uint32_t assemble(uint32_t lo4, uint32_t x, int L)
{
    const uint32_t t = (lo4 & 0x007F007Fu) | ((lo4 >> 1) & 0x3F803F80u);
    const uint32_t u = (t & 0x00003FFFu) | ((t >> 2) & 0x0FFFC000u);
    return __funnelshift_r(u | (x << 28), x >> 4, 35 - 7 * L);
}

// Volatile 16-byte descriptor access: each 64-bit word is a single-copy
// atomic access with its own state bits, so a reader that sees one word
// published and the other not yet simply waits.
__device__ __forceinline__ void ld_pair(const uint64_t *p, uint64_t &a, uint64_t &b)
{
    asm volatile("ld.volatile.global.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ void st_pair(uint64_t *p, uint64_t a, uint64_t b)
{
    asm volatile("st.volatile.global.v2.u64 [%0], {%1,%2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
    return v;
}

// Lanes 0..k where k is the lowest lane whose bit is set in `incl` (all lanes
// when none is): the descriptors that must be present before summing.
__device__ __forceinline__ unsigned through_first(unsigned incl)
{
    return incl ? (((incl & (0u - incl)) << 1) - 1u) : ~0u;
}

// Inclusive warp scan of x over lanes.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(~0u, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// ------------------------------------------------------------- look-back --
//
// Exclusive prefix (terminator count, gap sum) of a tile, by one warp, with a
// two-level decoupled look-back.  Tiles are grouped kGroup at a time:
//   - each tile publishes its aggregate in its own descriptor (tdesc) and
//     adds it to its group's atomic accumulators; the tile whose addition
//     completes the group publishes the group aggregate (gdesc, state AGG),
//     and once its own prefix is known upgrades it to INCL;
//   - a tile's prefix is the sum of the aggregates of the earlier tiles of
//     its group (one descriptor per lane) plus the prefix of its group, found
//     by looking back over group descriptors 32 at a time until an INCL one.
// The inclusive frontier thus advances 32 * kGroup tiles per L2 round trip.
// Every tile publishes before it waits, and waits only on earlier tiles, so
// every wait ends; each wait is also bounded by the global timer.

struct LbLoads {
    uint64_t ta, tb;   // this lane's intra-group tile descriptor
    uint64_t ga, gb;   // this lane's group descriptor (first window)
};

// Issue the descriptor loads of tile u's look-back early; lb_finish re-polls
// only what was not yet published when these loads returned.
__device__ __forceinline__ LbLoads lb_issue(const Params &p, uint64_t u, int lane)
{
    LbLoads l;
    l.ta = l.tb = l.ga = l.gb = 0;
    const uint64_t g = u / kGroup;
    const uint64_t j = g * kGroup + lane;
    if (j < u) ld_pair(p.tdesc + 2 * j, l.ta, l.tb);
    const long long gi = static_cast<long long>(g) - 1 - lane;
    if (gi >= 0) ld_pair(p.gdesc + 2 * gi, l.ga, l.gb);
    return l;
}

struct Prefix {
    uint64_t cnt;    // values decoded before the tile
    uint32_t sum;    // running x value before the tile's first gap
    uint64_t gcnt;   // values decoded before the tile's group
    uint32_t gsum;   // running x value before the tile's group
};

template <bool kDelta>
__device__ Prefix lb_finish(const Params &p, uint64_t u, LbLoads l, int lane)
{
    const uint64_t g = u / kGroup;
    const uint64_t g0 = g * kGroup;
    uint64_t t_start = 0;
    bool timed_out = false;
    auto expired = [&]() -> bool {
        if (timed_out) return true;
        const uint64_t now = global_ns();
        if (t_start == 0) t_start = now;
        if (now - t_start > kWaitLimitNs) {
            timed_out = true;
            if (lane == 0) atomicOr(p.status, VBYTE_ERR_TIMEOUT);
        }
        return timed_out;
    };

    // earlier tiles of the same group
    const uint64_t j = g0 + lane;
    const bool mine = j < u;
    for (int spin = 0;; ++spin) {
        const bool ready = !mine || ((l.ta >> 62) != 0 && (!kDelta || (l.tb >> 62) != 0));
        if (__all_sync(~0u, ready) || expired()) break;
        if (spin > 8) __nanosleep(100);
        if (mine) ld_pair(p.tdesc + 2 * j, l.ta, l.tb);
    }
    const uint64_t ec = warp_sum64(mine ? (l.ta & kPayload) : 0ull);
    const uint64_t es = warp_sum64(mine ? (l.tb & 0xFFFFFFFFull) : 0ull);

    // earlier groups; the virtual group before group 0 is inclusive (0, prev)
    uint64_t pc = 0, ps = 0;
    bool done_c = false, done_s = !kDelta;
    long long hi = static_cast<long long>(g) - 1;
    uint64_t a = l.ga, b = l.gb;
    for (bool fresh = true; !(done_c && done_s); fresh = false) {
        const long long idx = hi - lane;
        unsigned need_c, need_s, inc_c, inc_s;
        for (int spin = 0;; ++spin) {
            if (!(fresh && spin == 0)) {
                if (idx >= 0) ld_pair(p.gdesc + 2 * idx, a, b);
            }
            if (idx < 0) {
                a = kStateIncl;
                b = kStateIncl | (idx == -1 ? p.prev : 0u);
            }
            inc_c = __ballot_sync(~0u, (a >> 62) == 2u);
            inc_s = __ballot_sync(~0u, (b >> 62) == 2u);
            const unsigned emp_c = __ballot_sync(~0u, (a >> 62) == 0u);
            const unsigned emp_s = __ballot_sync(~0u, (b >> 62) == 0u);
            need_c = done_c ? 0u : through_first(inc_c);
            need_s = done_s ? 0u : through_first(inc_s);
            if ((!(emp_c & need_c) && !(emp_s & need_s)) || expired()) break;
            if (spin > 8) __nanosleep(100);
        }
        pc += warp_sum64(((need_c >> lane) & 1u) ? (a & kPayload) : 0ull);
        ps += warp_sum64(((need_s >> lane) & 1u) ? (b & 0xFFFFFFFFull) : 0ull);
        if (need_c && inc_c) done_c = true;
        if (need_s && inc_s) done_s = true;
        if (timed_out) break;
        hi -= 32;
    }
    Prefix r;
    r.cnt = (pc + ec) & kPayload;
    r.sum = static_cast<uint32_t>(ps + es);
    r.gcnt = pc & kPayload;
    r.gsum = static_cast<uint32_t>(ps);
    return r;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bit j set iff byte va + j lies inside [lo, hi).
__device__ __forceinline__ uint32_t slice_valid(uintptr_t va, uintptr_t lo, uintptr_t hi)
{
    if (va >= lo && va + kBPT <= hi) return 0xFFFFu;
    const long long a = static_cast<long long>(lo) - static_cast<long long>(va);
    const long long z = static_cast<long long>(hi) - static_cast<long long>(va);
    const int first = a > 0 ? (a > kBPT ? kBPT : static_cast<int>(a)) : 0;
    const int last = z > 0 ? (z > kBPT ? kBPT : static_cast<int>(z)) : 0;
    if (last <= first) return 0u;
    return ((1u << last) - 1u) & ~((1u << first) - 1u);
}

// Stage tile t into `bytes`: bytes[16 + 16*tid ..] gets tid's 16-byte slice
// (zero bytes outside the stream), bytes[0..16) the 16 bytes before the tile
// (zero before tile 0, i.e. terminators of earlier, uncounted integers; for
// t > 0 they always lie inside the stream).  Whole slices travel with
// cp.async; the ragged first and last slices of the stream are loaded byte
// by byte.  The caller commits and later waits for the copies.
__device__ __forceinline__ void stage_tile(const Params &p, uint64_t t, int tid, uint8_t *bytes)
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

// ------------------------------------------------------------------ kernel --
//
// Per CTA, iteration k handles two tiles: it decodes tile T (taken from the
// counter in iteration k-1, its bytes copied asynchronously then) and
// publishes T's aggregate, then finishes tile U (decoded in iteration k-1):
// resolves U's prefix -- whose descriptor loads were issued at the top of the
// iteration -- and writes U's values out.  Input bytes rotate through three
// shared-memory buffers (T, U, and the prefetch of the next tile), staged
// values through two (T and U).

constexpr int kByteBuf = kHalo + kTile + 16;
constexpr int kValBuf = 4 + kTile + 16;   // vals[4 + k]: tile rank k

template <bool kDelta>
__global__ void __launch_bounds__(kThreads, 4) decode_kernel(const Params p)
{
    __shared__ __align__(16) uint8_t s_bytes[3][kByteBuf];
    __shared__ __align__(16) uint32_t s_vals[2][kValBuf];
    __shared__ uint32_t s_wcnt[kWarps];
    __shared__ uint32_t s_wflag[kWarps];
    __shared__ uint32_t s_rtot[32];
    __shared__ uint32_t s_off[2][32];
    __shared__ unsigned long long s_R0[2];
    __shared__ uint32_t s_tcnt[2];
    __shared__ uint32_t s_cls[2];
    __shared__ unsigned long long s_next;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);

    if (tid == 0) s_next = atomicAdd(p.ctr, 1ull);
    __syncthreads();
    unsigned long long t = s_next;     // tile decoded this iteration (T)
    unsigned long long u = ~0ull;      // tile finished this iteration (U)
    if (t < p.ntiles) stage_tile(p, t, tid, s_bytes[0]);
    cp_async_commit();
    // warp 0, lane 0: whether U completed its group, and the group aggregate
    bool u_last_c = false, u_last_s = false;
    uint64_t u_gc = 0;
    uint32_t u_gs = 0;
    int rb = 0;   // byte buffer of T; U's is (rb + 2) % 3, the prefetch's (rb + 1) % 3

    for (int k = 0;; ++k) {
        const bool cur = t < p.ntiles;
        const bool fin = u < p.ntiles;
        if (!cur && !fin) break;
        const int vb = k & 1;
        uint32_t *const sw = reinterpret_cast<uint32_t *>(s_bytes[rb]);
        uint32_t *const sv = s_vals[vb] + 4;

        cp_async_wait_all();
        __syncthreads();   // T's bytes are staged; last iteration's readers are done
        LbLoads ll;
        if (warp == 0 && fin) ll = lb_issue(p, u, lane);
        if (cur && tid == 0) s_next = atomicAdd(p.ctr, 1ull);

        // ---- (a) terminator masks, counts, data checks, tile class
        const uintptr_t va = p.base + static_cast<uintptr_t>(t) * kTile + static_cast<uintptr_t>(tid) * kBPT;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        uint32_t tl = 0, t20 = 0, tc = 0, cnt = 0, inc = 0, wprev = 0;
        if (cur) {
            w = *reinterpret_cast<const uint4 *>(s_bytes[rb] + kHalo + tid * kBPT);
            wprev = sw[(kHalo + tid * kBPT) / 4 - 1];
            tl = term4(w.x) | (term4(w.y) << 4) | (term4(w.z) << 8) | (term4(w.w) << 12);
            t20 = term4(wprev) | (tl << 4);   // bits 0..3: the 4 bytes before mine
            const uint32_t valid = slice_valid(va, lo, hi);
            tc = tl & valid;                  // terminators inside the stream
            cnt = __popc(tc);
            const uint32_t c20 = ~t20 & 0xFFFFFu;   // continuation bytes
            if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
                atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
            if (hi - 1 >= va && hi - 1 < va + kBPT && !((tl >> (hi - 1 - va)) & 1u))
                atomicOr(p.status, VBYTE_ERR_TRUNCATED);
            const bool edge = valid != 0xFFFFu;
            const bool notA = edge || (c20 & 0xFFFF8u);
            const bool notB = edge || (c20 & (c20 << 1) & 0xFFFF8u);
            inc = warp_incl_scan(cnt, lane);
            const unsigned fa = __ballot_sync(~0u, notA);
            const unsigned fb = __ballot_sync(~0u, notB);
            if (lane == 31) s_wcnt[warp] = inc;
            if (lane == 0) s_wflag[warp] = (fa ? 1u : 0u) | (fb ? 2u : 0u);
        }
        __syncthreads();

        uint32_t tcnt = 0, cls = kClassC;
        unsigned long long tn = ~0ull;
        if (cur) {
            uint32_t wbase = 0, fl = 0;
#pragma unroll
            for (int q = 0; q < kWarps; ++q) {
                const uint32_t c = s_wcnt[q];
                wbase += (q < warp) ? c : 0u;
                tcnt += c;
                fl |= s_wflag[q];
            }
            cls = (fl & 2u) ? kClassC : ((fl & 1u) ? kClassB : kClassA);
            if (tid == 0) {
                s_tcnt[vb] = tcnt;
                s_cls[vb] = cls;
            }
            const uint32_t mybase = wbase + inc - cnt;

            // prefetch the tile of the next iteration
            tn = s_next;
            if (tn < p.ntiles) stage_tile(p, tn, tid, s_bytes[rb == 2 ? 0 : rb + 1]);

            // ---- (b) value assembly into the staging buffer, at tile rank
            if (cls == kClassC) {
                uint32_t *dst = sv + mybase;
                uint32_t m = tl;
                int prevo = 27 - __clz(t20 & 0xFu);   // last terminator before my bytes (-5: none)
                while (m) {
                    const int o = __ffs(m) - 1;
                    m &= m - 1u;
                    const int L = min(o - prevo, 5);
                    prevo = o;
                    if ((tc >> o) & 1u) {
                        const int q = kHalo + tid * kBPT + o;   // staging byte of the terminator
                        const uint32_t A = sw[(q >> 2) - 1];
                        const uint32_t B = sw[q >> 2];
                        const uint32_t lo4 = __funnelshift_r(A, B, 8 * q);
                        const uint32_t x = (B >> (8 * (q & 3))) & 0xFFu;
                        *dst++ = assemble(lo4, x, L);
                    }
                }
            } else if (cls == kClassB) {
                uint32_t *dst = sv + mybase;
                const uint32_t cur4[4] = {w.x, w.y, w.z, w.w};
                uint32_t wp = wprev;
                int q = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t c = cur4[j];
                    const uint32_t s = __funnelshift_l(wp, c, 8);   // byte i: the byte before byte i
                    const uint32_t cm = prmt(s, 0u, 0xBA98u);        // 0xFF where that byte continues
                    const uint32_t lob = (s & 0x7F7F7F7Fu & cm) | (c & ~cm);
                    const uint32_t hib = c & cm;
                    uint32_t q01 = prmt(lob, hib, 0x5140u);
                    uint32_t q23 = prmt(lob, hib, 0x7362u);
                    q01 -= (q01 & 0xFF00FF00u) >> 1;
                    q23 -= (q23 & 0xFF00FF00u) >> 1;
                    const uint32_t v4[4] = {q01 & 0xFFFFu, q01 >> 16, q23 & 0xFFFFu, q23 >> 16};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if ((tc >> (4 * j + i)) & 1u) dst[q++] = v4[i];
                    wp = c;
                }
            }
        }
        cp_async_commit();
        __syncthreads();

        // ---- (c) delta: scan T's gaps in place, per (round, warp) entry
        if (kDelta && cur) {
            const uint32_t nr1 = (tcnt + kRoundVals - 1) / kRoundVals;
            for (uint32_t r = 0; r < nr1; ++r) {
                const int idx = static_cast<int>(r * kRoundVals) + 4 * tid;
                uint4 v;
                if (cls == kClassA) {
                    const uint32_t x = sw[(kHalo + idx) >> 2];
                    v = make_uint4(prmt(x, 0u, 0x4440u), prmt(x, 0u, 0x4441u), prmt(x, 0u, 0x4442u),
                                   prmt(x, 0u, 0x4443u));
                } else {
                    v = *reinterpret_cast<const uint4 *>(sv + idx);
                }
                if (static_cast<uint32_t>(idx) + 4 > tcnt) {
                    if (static_cast<uint32_t>(idx) + 0 >= tcnt) v.x = 0u;
                    if (static_cast<uint32_t>(idx) + 1 >= tcnt) v.y = 0u;
                    if (static_cast<uint32_t>(idx) + 2 >= tcnt) v.z = 0u;
                    if (static_cast<uint32_t>(idx) + 3 >= tcnt) v.w = 0u;
                }
                v.y += v.x;
                v.z += v.y;
                v.w += v.z;
                const uint32_t ws = warp_incl_scan(v.w, lane);
                const uint32_t ex = ws - v.w;
                v.x += ex;
                v.y += ex;
                v.z += ex;
                v.w += ex;
                *reinterpret_cast<uint4 *>(sv + idx) = v;
                if (lane == 31) s_rtot[r * kWarps + warp] = ws;
            }
        }
        if (kDelta) __syncthreads();

        // ---- warp 0: publish T's aggregate, then resolve U's prefix
        if (warp == 0) {
            unsigned long long oc = 0, os = 0;
            uint64_t gt = 0, gsize = 0;
            uint32_t tsum = 0;
            if (cur) {
                if (kDelta) {
                    const uint32_t ne = ((tcnt + kRoundVals - 1) / kRoundVals) * kWarps;
                    const uint32_t e = static_cast<uint32_t>(lane) < ne ? s_rtot[lane] : 0u;
                    const uint32_t ie = warp_incl_scan(e, lane);
                    tsum = __shfl_sync(~0u, ie, 31);
                    s_off[vb][lane] = ie - e;   // tile-local; T's prefix is added next iteration
                }
                gt = t / kGroup;
                const uint64_t g0t = gt * kGroup;
                gsize = (p.ntiles - g0t < kGroup) ? (p.ntiles - g0t) : static_cast<uint64_t>(kGroup);
                if (lane == 0) {
                    st_pair(p.tdesc + 2 * t, kStateAgg | tcnt, kStateAgg | tsum);
                    oc = atomicAdd(p.gacc + 2 * gt, (1ull << 48) | tcnt);
                    if (kDelta) os = atomicAdd(p.gacc + 2 * gt + 1, (1ull << 48) | tsum);
                }
            }
            if (fin) {
                const Prefix pre = lb_finish<kDelta>(p, u, ll, lane);
                if (kDelta) s_off[vb ^ 1][lane] += pre.sum;
                if (lane == 0) {
                    s_R0[vb ^ 1] = pre.cnt;
                    const uint64_t gu = u / kGroup;
                    if (u_last_c) st_relaxed(p.gdesc + 2 * gu, kStateIncl | ((pre.gcnt + u_gc) & kPayload));
                    if (kDelta && u_last_s)
                        st_relaxed(p.gdesc + 2 * gu + 1, kStateIncl | static_cast<uint32_t>(pre.gsum + u_gs));
                    if (u == p.ntiles - 1 && pre.cnt + s_tcnt[vb ^ 1] != p.n)
                        atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
                }
            }
            if (lane == 0) {
                u_last_c = false;
                u_last_s = false;
                if (cur) {
                    u_last_c = (oc >> 48) + 1 == gsize;
                    u_gc = (oc + tcnt) & kMask48;
                    if (u_last_c) st_relaxed(p.gdesc + 2 * gt, kStateAgg | u_gc);
                    if (kDelta) {
                        u_last_s = (os >> 48) + 1 == gsize;
                        u_gs = static_cast<uint32_t>(os + tsum);
                        if (u_last_s) st_relaxed(p.gdesc + 2 * gt + 1, kStateAgg | u_gs);
                    }
                }
            }
        }
        __syncthreads();

        // ---- copy-out of U: 16-byte aligned output quads, alignment fixed by
        // a one-lane shuffle of the staged quads
        if (fin) {
            const uint32_t *const pw = reinterpret_cast<const uint32_t *>(s_bytes[rb == 0 ? 2 : rb - 1]);
            const uint32_t *const pv = s_vals[vb ^ 1] + 4;
            const uint32_t ucnt = s_tcnt[vb ^ 1];
            const uint32_t ucls = s_cls[vb ^ 1];
            const unsigned long long R0 = s_R0[vb ^ 1];
            auto rank_quad = [&](int idx) -> uint4 {   // idx >= -4
                if (!kDelta && ucls == kClassA) {
                    const uint32_t x = pw[(kHalo + idx) >> 2];
                    return make_uint4(prmt(x, 0u, 0x4440u), prmt(x, 0u, 0x4441u), prmt(x, 0u, 0x4442u),
                                      prmt(x, 0u, 0x4443u));
                }
                uint4 v = *reinterpret_cast<const uint4 *>(pv + idx);
                if (kDelta) {
                    const uint32_t off = s_off[vb ^ 1][min(max(idx, 0) / 128, 31)];
                    v.x += off;
                    v.y += off;
                    v.z += off;
                    v.w += off;
                }
                return v;
            };
            const uint32_t sh = (out_word + static_cast<uint32_t>(R0)) & 3u;
            const long long rho0 = static_cast<long long>(R0) - sh;   // output rank of quad 0
            const uint32_t nr2 = (ucnt + sh + kRoundVals - 1) / kRoundVals;
            for (uint32_t r = 0; r < nr2; ++r) {
                const int idx = static_cast<int>(r * kRoundVals) + 4 * tid;
                const int ridx = min(idx, kTile);   // keep reads inside the buffers
                const uint4 qc = rank_quad(ridx);
                uint4 qp;
                qp.x = __shfl_up_sync(~0u, qc.x, 1);
                qp.y = __shfl_up_sync(~0u, qc.y, 1);
                qp.z = __shfl_up_sync(~0u, qc.z, 1);
                qp.w = __shfl_up_sync(~0u, qc.w, 1);
                if (lane == 0 && sh != 0u) qp = rank_quad(ridx - 4);
                uint4 o;
                switch (sh) {
                case 0: o = qc; break;
                case 1: o = make_uint4(qp.w, qc.x, qc.y, qc.z); break;
                case 2: o = make_uint4(qp.z, qp.w, qc.x, qc.y); break;
                default: o = make_uint4(qp.y, qp.z, qp.w, qc.x); break;
                }
                const int k0 = idx - static_cast<int>(sh);   // tile rank of o.x
                const long long g0 = rho0 + idx;             // output rank of o.x
                if (k0 >= 0 && k0 + 4 <= static_cast<int>(ucnt) && g0 + 4 <= static_cast<long long>(p.n)) {
                    st_quad(p.out + g0, o);
                } else if (k0 + 4 > 0 && k0 < static_cast<int>(ucnt)) {
                    const uint32_t e4[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (k0 + j >= 0 && k0 + j < static_cast<int>(ucnt) &&
                            g0 + j < static_cast<long long>(p.n))
                            p.out[g0 + j] = e4[j];
                }
            }
        }

        u = cur ? t : ~0ull;
        t = cur ? tn : ~0ull;
        rb = rb == 2 ? 0 : rb + 1;
    }
    cp_async_wait_all();
}

__global__ void set_status_kernel(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// ------------------------------------------------------------- workspace --

// Workspace layout: [0,4) status word, [256,264) tile counter, [512, ...)
// tile descriptors (16 bytes per tile), group accumulators (16 bytes per
// group), group descriptors (16 bytes per group).  Everything past the status
// word is cleared before each launch.
constexpr size_t kWsCounter = 256;
constexpr size_t kWsDesc = 512;

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

struct DeviceInfo {
    int sms = 0;
    int occ[2] = {0, 0};
};

std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, Workspace> g_ws;
std::map<std::pair<int, uintptr_t>, HostBuffers> g_hb;
std::map<int, DeviceInfo> g_dev;

uint64_t num_groups(uint64_t ntiles) { return (ntiles + kGroup - 1) / kGroup; }

size_t ws_bytes(uint64_t ntiles)
{
    return kWsDesc + 16 * static_cast<size_t>(ntiles) + 32 * static_cast<size_t>(num_groups(ntiles));
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

int device_info(DeviceInfo *di)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo &d = g_dev[dev];
    if (d.sms == 0) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return VBYTE_ECUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[0], decode_kernel<false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[1], decode_kernel<true>, kThreads, 0);
        for (int &o : d.occ) o = std::max(o, 1);
    }
    *di = d;
    return VBYTE_OK;
}

int launch_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta,
                  uint32_t prev, cudaStream_t s)
{
    if (nbytes == 0 && n == 0) return VBYTE_OK;
    if ((nbytes && !in) || (n && !out)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(out) & 3u) return VBYTE_EINVAL;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    const uint64_t ntiles = nbytes ? ((a & 15u) + nbytes + kTile - 1) / kTile : 0;
    Workspace *w = nullptr;
    int rc = get_workspace(s, ws_bytes(ntiles), &w);
    if (rc != VBYTE_OK) return rc;
    uint32_t *status = reinterpret_cast<uint32_t *>(w->ptr);
    if (nbytes == 0) {  // n > 0 values expected from an empty stream
        set_status_kernel<<<1, 1, 0, s>>>(status, VBYTE_ERR_COUNT_MISMATCH);
        return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
    }
    DeviceInfo di;
    rc = device_info(&di);
    if (rc != VBYTE_OK) return rc;
    if (cudaMemsetAsync(w->ptr + kWsCounter, 0, ws_bytes(ntiles) - kWsCounter, s) != cudaSuccess)
        return VBYTE_ECUDA;
    Params p;
    p.in = in;
    p.nbytes = nbytes;
    p.out = out;
    p.n = n;
    p.ntiles = ntiles;
    p.base = a & ~static_cast<uintptr_t>(15);
    p.ctr = reinterpret_cast<unsigned long long *>(w->ptr + kWsCounter);
    p.tdesc = reinterpret_cast<uint64_t *>(w->ptr + kWsDesc);
    p.gacc = reinterpret_cast<unsigned long long *>(p.tdesc + 2 * ntiles);
    p.gdesc = reinterpret_cast<uint64_t *>(p.gacc + 2 * num_groups(ntiles));
    p.status = status;
    p.prev = prev;
    const uint64_t grid = std::min<uint64_t>(ntiles, static_cast<uint64_t>(di.sms) * di.occ[delta]);
    if (delta)
        decode_kernel<true><<<static_cast<unsigned>(grid), kThreads, 0, s>>>(p);
    else
        decode_kernel<false><<<static_cast<unsigned>(grid), kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace vbk

extern "C" {

int vbyte_decode(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, false, 0u, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n,
                       uint32_t prev, void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, true, prev, static_cast<cudaStream_t>(stream));
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
    if (n && cudaMemcpyAsync(h_out, hb->d_out, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess)
        return VBYTE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int vbyte_get_status(void *stream, uint32_t *status_out)
{
    if (!status_out) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vbk::Workspace *w = nullptr;
    int rc = vbk::get_workspace(s, vbk::kWsDesc, &w);
    if (rc != VBYTE_OK) return rc;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, w->ptr, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VBYTE_ECUDA;
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
    default: return "unknown vbyte error code";
    }
}

size_t vbyte_workspace_size(size_t nbytes)
{
    const uint64_t ntiles = (15 + nbytes + vbk::kTile - 1) / vbk::kTile;
    return vbk::ws_bytes(ntiles);
}

}  // extern "C"
