// libvbyte: single-pass GPU decoder for VByte-coded uint32 streams (sm_103a).
//
// Operation (arXiv 1503.07387): the result of Algorithm 1 (Sec. 2) on the
// byte stream -- seven data bits per byte, least significant group first,
// high bit set on every byte of an integer except its last (Sec. 1, Table 1)
// -- optionally followed by the prefix sum that undoes differential coding
// (Sec. 1 "Differential coding", Sec. 4 "Differential Coding").
//
// GPU design (one kernel, one pass over the input, persistent CTAs):
//   (a) terminator mask + slot assignment.  A tile is 4 KiB of input aligned
//       to 16 bytes in absolute address space.  Each thread loads 16 bytes
//       with one vector load, forms a 16-bit mask of terminator bytes (high
//       bit clear -- the GPU counterpart of pmovmskb in Sec. 3/4) and counts
//       them.  A block scan gives every thread its first slot inside the
//       tile; a decoupled look-back over per-tile descriptors gives the
//       tile's first global slot.  A tile owns exactly the integers whose
//       terminator byte lies inside it; the 16 bytes before the tile are
//       staged too, so an integer that starts in the previous tile (at most
//       four bytes earlier) is assembled by the tile holding its terminator.
//   (b) value assembly.  Integers are assembled branch-free from the (up to)
//       five bytes ending at their terminator.  The work is split by the
//       longest code in the tile, the GPU counterpart of the paper's case
//       split on the 12-bit mask (Sec. 4): class A (every byte a
//       terminator: values are the bytes themselves), class B (codes of at
//       most two bytes: a SWAR byte-pair merge over 4-byte words) and class
//       C (any length: per-terminator assembly from shared memory).
//       Values are staged in shared memory at their tile rank, shifted so
//       that every output quad is 16-byte aligned in global memory.
//   (c) fused delta prefix sum.  Staged gaps are scanned in registers (four
//       consecutive values per thread, then a warp scan, then a block scan of
//       warp totals) and the tile's carry-in comes from a second decoupled
//       look-back on gap sums, seeded with `prev` (uint32 wrap-around).
//   Output quads leave with 16-byte stores, clamped to [0, n).
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
constexpr int kMaxRounds = (kTile + 3 + kRoundVals - 1) / kRoundVals;
constexpr int kValStage = kTile + 16;         // staged values (+ alignment shift)

constexpr uint64_t kStateAgg = 1ull << 62;    // descriptor holds the tile aggregate
constexpr uint64_t kStateIncl = 2ull << 62;   // descriptor holds the inclusive prefix
constexpr uint64_t kPayload = (1ull << 62) - 1;
constexpr uint64_t kWaitLimitNs = 2000000000ull;

enum : uint32_t { kClassA = 0, kClassB = 1, kClassC = 2 };

struct Params {
    const uint8_t *in;
    uint64_t nbytes;
    uint32_t *out;
    uint64_t n;
    uint64_t ntiles;
    uintptr_t base;            // 16-byte aligned address of tile 0
    uint64_t *dcnt;            // per-tile terminator-count descriptors
    uint64_t *dsum;            // per-tile gap-sum descriptors (delta mode)
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

// Decoupled look-back (one warp).  Lane i inspects descriptor t-1-i; the warp
// waits until every descriptor up to the nearest inclusive one has been
// published, adds their payloads and repeats 32 tiles further back if none
// of them was inclusive.  Descriptors before tile 0 count as inclusive zero.
__device__ uint64_t lookback(const uint64_t *desc, unsigned long long t, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    uint64_t acc = 0;
    long long hi = static_cast<long long>(t) - 1;
    uint64_t t0 = 0;
    bool timed_out = false;
    for (;;) {
        const long long idx = hi - lane;
        uint64_t w;
        unsigned incl, need;
        for (;;) {
            w = idx >= 0 ? ld_relaxed(desc + idx) : kStateIncl;
            const unsigned st = static_cast<unsigned>(w >> 62);
            incl = __ballot_sync(~0u, st == 2u);
            const unsigned empty = __ballot_sync(~0u, st == 0u);
            need = incl ? (((incl & (0u - incl)) << 1) - 1u) : ~0u;
            if (!(empty & need) || timed_out) break;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > kWaitLimitNs) {
                timed_out = true;
                if (lane == 0) atomicOr(status, VBYTE_ERR_TIMEOUT);
            }
            __nanosleep(32);
        }
        uint64_t v = ((need >> lane) & 1u) ? (w & kPayload) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
        acc += v;
        if (incl || timed_out) break;
        hi -= 32;
    }
    return acc;
}

// Exclusive warp scan helper: returns the inclusive scan of x over lanes.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(~0u, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// ------------------------------------------------------------------ kernel --

template <bool kDelta>
__global__ void __launch_bounds__(kThreads) decode_kernel(const Params p)
{
    __shared__ __align__(16) uint8_t s_bytes[kHalo + kTile + 16];
    __shared__ __align__(16) uint32_t s_vals[kValStage];
    __shared__ uint32_t s_wcnt[kWarps];
    __shared__ uint32_t s_wflag[kWarps];
    __shared__ uint32_t s_woff[kWarps];
    __shared__ uint32_t s_rtot[64];
    __shared__ unsigned long long s_tile;
    __shared__ unsigned long long s_R0;
    __shared__ uint32_t s_tcnt;
    __shared__ uint32_t s_class;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.in);
    const uintptr_t hi = lo + p.nbytes;
    const uint32_t out_word = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p.out) >> 2);
    uint32_t *const sw = reinterpret_cast<uint32_t *>(s_bytes);

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(p.ctr, 1ull);
        __syncthreads();
        const unsigned long long t = s_tile;
        if (t >= p.ntiles) break;
        const uintptr_t tstart = p.base + static_cast<uintptr_t>(t) * kTile;
        const uintptr_t va = tstart + static_cast<uintptr_t>(tid) * kBPT;

        // ---- stage the tile (and the 16 bytes before it) in shared memory
        uint4 w;
        uint32_t valid;
        if (va >= lo && va + kBPT <= hi) {
            w = ld_stream16(reinterpret_cast<const void *>(va));
            valid = 0xFFFFu;
        } else {
            uint32_t wb[4] = {0u, 0u, 0u, 0u};
            valid = 0u;
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                const uintptr_t ad = va + j;
                if (ad >= lo && ad < hi) {
                    wb[j >> 2] |= static_cast<uint32_t>(*reinterpret_cast<const uint8_t *>(ad))
                                  << (8 * (j & 3));
                    valid |= 1u << j;
                }
            }
            w = make_uint4(wb[0], wb[1], wb[2], wb[3]);
        }
        *reinterpret_cast<uint4 *>(s_bytes + kHalo + tid * kBPT) = w;
        if (tid == 0) {
            // The 16 bytes before tile t > 0 always lie inside the stream; before
            // tile 0 they read as zero bytes, i.e. as terminators of earlier,
            // uncounted integers.
            uint4 h = make_uint4(0u, 0u, 0u, 0u);
            if (t > 0) h = ld_stream16(reinterpret_cast<const void *>(tstart - 16));
            *reinterpret_cast<uint4 *>(s_bytes) = h;
        }
        if (tid == kThreads - 1)
            *reinterpret_cast<uint4 *>(s_bytes + kHalo + kTile) = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();

        // ---- (a) terminator masks, counts, data checks, tile class
        const uint32_t wprev = sw[(kHalo + tid * kBPT) / 4 - 1];
        const uint32_t tl = term4(w.x) | (term4(w.y) << 4) | (term4(w.z) << 8) | (term4(w.w) << 12);
        const uint32_t t20 = term4(wprev) | (tl << 4);   // bits 0..3: the 4 bytes before mine
        const uint32_t tc = tl & valid;                   // terminators inside the stream
        const uint32_t cnt = __popc(tc);
        const uint32_t c20 = ~t20 & 0xFFFFFu;             // continuation bytes
        if (c20 & (c20 << 1) & (c20 << 2) & (c20 << 3) & (c20 << 4) & 0xFFFF0u)
            atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
        if (hi - 1 >= va && hi - 1 < va + kBPT && !((tl >> (hi - 1 - va)) & 1u))
            atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        const bool edge = valid != 0xFFFFu;
        const bool notA = edge || (c20 & 0xFFFF8u);
        const bool notB = edge || (c20 & (c20 << 1) & 0xFFFF8u);

        const uint32_t inc = warp_incl_scan(cnt, lane);
        const unsigned fa = __ballot_sync(~0u, notA);
        const unsigned fb = __ballot_sync(~0u, notB);
        if (lane == 31) s_wcnt[warp] = inc;
        if (lane == 0) s_wflag[warp] = (fa ? 1u : 0u) | (fb ? 2u : 0u);
        __syncthreads();

        if (warp == 0) {
            const uint32_t wc = lane < kWarps ? s_wcnt[lane] : 0u;
            uint32_t wi = wc;
#pragma unroll
            for (int o = 1; o < kWarps; o <<= 1) {
                const uint32_t y = __shfl_up_sync(~0u, wi, o);
                if (lane >= o) wi += y;
            }
            const uint32_t tcnt = __shfl_sync(~0u, wi, kWarps - 1);
            const uint32_t fl = __reduce_or_sync(~0u, lane < kWarps ? s_wflag[lane] : 0u);
            if (lane < kWarps) s_woff[lane] = wi - wc;
            uint64_t excl = 0;
            if (t == 0) {
                if (lane == 0) st_relaxed(p.dcnt, kStateIncl | tcnt);
            } else {
                if (lane == 0) st_relaxed(p.dcnt + t, kStateAgg | tcnt);
                excl = lookback(p.dcnt, t, p.status);
                if (lane == 0) st_relaxed(p.dcnt + t, kStateIncl | ((excl + tcnt) & kPayload));
            }
            if (lane == 0) {
                s_R0 = excl;
                s_tcnt = tcnt;
                s_class = (fl & 2u) ? kClassC : ((fl & 1u) ? kClassB : kClassA);
                if (t == p.ntiles - 1 && excl + tcnt != p.n)
                    atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
            }
        }
        __syncthreads();

        const unsigned long long R0 = s_R0;
        const uint32_t tcnt = s_tcnt;
        const uint32_t cls = s_class;
        // staging index sh holds tile rank 0; it is chosen so that staging index
        // 4k maps to a 16-byte aligned output address
        const uint32_t sh = (out_word + static_cast<uint32_t>(R0)) & 3u;
        const uint32_t mybase = s_woff[warp] + inc - cnt;

        // ---- (b) value assembly into the staging buffer
        if (cls == kClassC) {
            uint32_t *dst = s_vals + sh + mybase;
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
            uint32_t *dst = s_vals + sh + mybase;
            const uint32_t cur4[4] = {w.x, w.y, w.z, w.w};
            uint32_t wp = wprev;
            int k = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t cur = cur4[j];
                const uint32_t s = __funnelshift_l(wp, cur, 8);  // byte i: the byte before byte i
                const uint32_t cm = prmt(s, 0u, 0xBA98u);         // 0xFF where that byte continues
                const uint32_t lob = (s & 0x7F7F7F7Fu & cm) | (cur & ~cm);
                const uint32_t hib = cur & cm;
                uint32_t q01 = prmt(lob, hib, 0x5140u);
                uint32_t q23 = prmt(lob, hib, 0x7362u);
                q01 -= (q01 & 0xFF00FF00u) >> 1;
                q23 -= (q23 & 0xFF00FF00u) >> 1;
                const uint32_t v4[4] = {q01 & 0xFFFFu, q01 >> 16, q23 & 0xFFFFu, q23 >> 16};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if ((tc >> (4 * j + i)) & 1u) dst[k++] = v4[i];
                wp = cur;
            }
        }
        __syncthreads();

        // ---- copy-out (c: with the fused prefix sum in delta mode)
        const uint32_t lim = sh + tcnt;                        // staged indices [sh, lim)
        const long long gb = static_cast<long long>(R0) - sh;  // global rank of index 0
        const uint32_t nr = (lim + kRoundVals - 1) / kRoundVals;

        auto load_quad = [&](uint32_t idx) -> uint4 {
            if (cls == kClassA) {
                // every byte is a one-byte integer: tile rank k is tile byte k
                const int q0 = kHalo + static_cast<int>(idx) - static_cast<int>(sh);
                const uint32_t x = __funnelshift_r(sw[q0 >> 2], sw[(q0 >> 2) + 1], 8 * q0);
                return make_uint4(prmt(x, 0u, 0x4440u), prmt(x, 0u, 0x4441u),
                                  prmt(x, 0u, 0x4442u), prmt(x, 0u, 0x4443u));
            }
            return *reinterpret_cast<const uint4 *>(s_vals + idx);
        };
        auto store_quad = [&](uint32_t idx, uint4 v) {
            const long long g0 = gb + idx;
            if (idx >= sh && idx + 4 <= lim && g0 + 4 <= static_cast<long long>(p.n)) {
                st_quad(p.out + g0, v);
            } else {
                const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (idx + j >= sh && idx + j < lim && g0 + j < static_cast<long long>(p.n))
                        p.out[g0 + j] = e[j];
            }
        };

        if (!kDelta) {
            for (uint32_t r = 0; r < nr; ++r) {
                const uint32_t idx = r * kRoundVals + 4 * tid;
                if (idx < lim) store_quad(idx, load_quad(idx));
            }
        } else {
            uint4 vv[kMaxRounds];
#pragma unroll
            for (int r = 0; r < kMaxRounds; ++r) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (r < static_cast<int>(nr)) {
                    const uint32_t idx = r * kRoundVals + 4 * tid;
                    if (idx < lim) {
                        v = load_quad(idx);
                        if (idx < sh || idx + 4 > lim) {
                            if (idx + 0 < sh || idx + 0 >= lim) v.x = 0u;
                            if (idx + 1 < sh || idx + 1 >= lim) v.y = 0u;
                            if (idx + 2 < sh || idx + 2 >= lim) v.z = 0u;
                            if (idx + 3 < sh || idx + 3 >= lim) v.w = 0u;
                        }
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
                    if (lane == 31) s_rtot[r * kWarps + warp] = ws;
                }
                vv[r] = v;
            }
            __syncthreads();
            if (warp == 0) {
                const uint32_t ne = nr * kWarps;
                const uint32_t e0 = static_cast<uint32_t>(lane) < ne ? s_rtot[lane] : 0u;
                const uint32_t e1 = static_cast<uint32_t>(lane) + 32 < ne ? s_rtot[lane + 32] : 0u;
                const uint32_t i0 = warp_incl_scan(e0, lane);
                const uint32_t c0 = __shfl_sync(~0u, i0, 31);
                const uint32_t i1 = warp_incl_scan(e1, lane);
                const uint32_t tsum = c0 + __shfl_sync(~0u, i1, 31);
                uint32_t excl;
                if (t == 0) {
                    excl = p.prev;
                    if (lane == 0) st_relaxed(p.dsum, kStateIncl | static_cast<uint32_t>(excl + tsum));
                } else {
                    if (lane == 0) st_relaxed(p.dsum + t, kStateAgg | tsum);
                    excl = static_cast<uint32_t>(lookback(p.dsum, t, p.status));
                    if (lane == 0)
                        st_relaxed(p.dsum + t, kStateIncl | static_cast<uint32_t>(excl + tsum));
                }
                s_rtot[lane] = excl + i0 - e0;
                s_rtot[lane + 32] = excl + c0 + i1 - e1;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kMaxRounds; ++r) {
                if (r < static_cast<int>(nr)) {
                    const uint32_t idx = r * kRoundVals + 4 * tid;
                    if (idx < lim) {
                        const uint32_t off = s_rtot[r * kWarps + warp];
                        uint4 v = vv[r];
                        v.x += off;
                        v.y += off;
                        v.z += off;
                        v.w += off;
                        store_quad(idx, v);
                    }
                }
            }
        }
    }
}

__global__ void set_status_kernel(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// ------------------------------------------------------------- workspace --

// Workspace layout: [0,4) status word, [256,264) tile counter, [512, ...)
// count descriptors (8 bytes per tile) then sum descriptors (8 bytes per tile).
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

size_t ws_bytes(uint64_t ntiles) { return kWsDesc + 16 * static_cast<size_t>(ntiles); }

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
    p.dcnt = reinterpret_cast<uint64_t *>(w->ptr + kWsDesc);
    p.dsum = p.dcnt + ntiles;
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
