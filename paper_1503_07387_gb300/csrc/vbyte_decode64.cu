// 64-bit VByte decoding (vbyte_decode64, vbyte_decode_delta64).
//
// Operation (arXiv 1503.07387): Sec. 1 notes that the VByte format covers
// 64-bit integers as well as the 32-bit ones the paper works with.  Read for
// uint64: seven data bits per byte, least significant group first, the high
// bit set on every byte of an integer but the last, so up to ten bytes; an
// integer ends at a byte whose high bit is clear, and Algorithm 1 (Sec. 2)
// run for ten steps rebuilds it, the tenth byte multiplied by 2^63 modulo
// 2^64.  In delta mode the integers are gaps and the output is their running
// sum from prev, modulo 2^64 (Sec. 1, "Differential coding").
//
// Design: three launches and no waits between CTAs.
//   count64:  per 4 KiB tile of the input, the number of integers that end
//             in it and, in delta mode, their sum; also the data-error
//             checks (a run of ten or more high-bit bytes; a last byte with
//             the high bit set);
//   scan64:   one CTA turns the per-tile counts and sums into the values
//             before each tile and prev plus the sum of every integer before
//             it (1024 tiles per round, a carry between rounds), and checks
//             the total count against n;
//   decode64: per tile, every integer that ends in it, assembled from its own
//             bytes (at most nine before its terminator; the 16 bytes staged
//             ahead of the tile cover them): codes of at most two bytes by
//             byte pairs, longer ones from the eight bytes ending at the
//             terminator compacted into 56 bits with SWAR steps; placed by a
//             block scan of the per-thread counts into shared memory (one
//             padding slot every 16, so that a warp's stores do not share
//             banks), prefix-summed there in delta mode, and written out with
//             coalesced 8-byte stores.
// Tiles start at the input address rounded down to 16 bytes, so every
// staged chunk is one aligned 16-byte load; bytes of a chunk outside the
// input are staged as zero and never counted.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "vbyte.h"
#include "vbyte64.h"
#include "vbyte_device.cuh"
#include "vbyte_internal.h"

namespace vbk {
namespace d64 {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 4096;                 // input bytes per tile
constexpr int kSlice = kTile / kThreads;    // bytes per thread
constexpr int kHalo = 16;                   // bytes staged before the tile
constexpr int kMaxLen = 10;                 // bytes of the longest uint64 code
constexpr int kScanThreads = 1024;
constexpr size_t kHead = 256;               // workspace: status word, then the tile arrays
static_assert(kSlice == 16, "one 16-byte chunk per thread");
static_assert(kHalo >= kMaxLen - 1, "an integer's earlier bytes lie in the halo");

struct Params {
    const uint8_t *base;   // the input rounded down to 16 bytes
    int64_t lo, hi;        // the input is [lo, hi) from base (lo < 16)
    uint64_t ntiles;
    uint64_t *out;
    uint64_t n;
    uint64_t prev;
    uint64_t *tcnt;        // per tile: integers ending in it; after scan64, integers before it
    uint64_t *tsum;        // per tile (delta): their sum; after scan64, prev + the sum before it
    uint32_t *status;
};

struct CountShared {
    alignas(16) uint8_t bytes[kHalo + kTile];
    unsigned long long wsum[kWarps];
    uint32_t wcnt[kWarps];
};

// The tile's integers in order, one padding slot after every 16: a thread's
// run of 16 consecutive ranks then starts 17 slots after its neighbour's, so
// the 32 lanes of a warp touch 32 different 8-byte bank pairs.
constexpr int kPadded = kTile + kTile / 16;
__device__ __forceinline__ uint32_t slot(uint32_t j) { return j + (j >> 4); }

struct DecodeShared {
    alignas(16) uint8_t bytes[kHalo + kTile];
    alignas(16) unsigned long long vals[kPadded];
    unsigned long long wsum[kWarps];
    uint32_t wcnt[kWarps];
};

// Zero the bytes of the chunk at q0 that lie outside [lo, hi).
__device__ __forceinline__ uint4 clip_chunk(uint4 v, int64_t q0, int64_t lo, int64_t hi)
{
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t q = q0 + 4 * k + j;
            if (q < lo || q >= hi) w[k] &= ~(0xFFu << (8 * j));
        }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Stage tile t and the 16 bytes before it: chunk c in [-1, kTile/16) goes to
// bytes[kHalo + 16c].  A chunk is loaded only if it holds an input byte; it
// is then one aligned 16-byte load that stays inside the input's 16-byte
// blocks.
__device__ __forceinline__ void stage(const Params &p, uint64_t t, uint8_t *bytes)
{
    const int64_t t0 = static_cast<int64_t>(t) * kTile;
    for (int c = static_cast<int>(threadIdx.x) - 1; c < kTile / 16; c += kThreads) {
        const int64_t q0 = t0 + 16ll * c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (q0 + 16 > p.lo && q0 < p.hi) {   // then q0 >= 0: q0 is a multiple of 16 above -16
            v = __ldg(reinterpret_cast<const uint4 *>(p.base + q0));
            if (q0 < p.lo || q0 + 16 > p.hi) v = clip_chunk(v, q0, p.lo, p.hi);
        }
        *reinterpret_cast<uint4 *>(bytes + kHalo + 16 * c) = v;
    }
}

// Four 7-bit payloads (the bytes of x) compacted into 28 bits, byte i at bit
// 7 i (the fields are disjoint, so they are added).
__device__ __forceinline__ uint32_t compact28(uint32_t x)
{
    const uint32_t t = (x & 0x007F007Fu) + ((x >> 1) & 0x3F803F80u);
    return (t & 0x00003FFFu) + ((t >> 2) & 0x0FFFC000u);
}

// The integers that end in this thread's slice, tile bytes [16 tid, 16 tid +
// 16), at tile positions in [a, b), in order: f(v) for each (kValues).  They
// come from a 32-byte window (the 16 bytes before the slice, possibly the
// halo, and the slice) held in registers and masks: codes of at most two
// bytes by byte pairs, any others one terminator at a time from the eight
// bytes that end at it (and at most two more).  Returns whether the slice
// holds a byte that makes a run of ten or more high-bit bytes.
template <bool kValues, class F>
__device__ __forceinline__ bool values64(const uint8_t *bytes, int tid, int a, int b, F &&f)
{
    const uint8_t *const wb = bytes + kHalo + kSlice * tid - 16;
    const uint32_t *const ww = reinterpret_cast<const uint32_t *>(wb);
    const uint4 pq = reinterpret_cast<const uint4 *>(wb)[0];
    const uint4 q = reinterpret_cast<const uint4 *>(wb)[1];
    const uint32_t W[8] = {pq.x, pq.y, pq.z, pq.w, q.x, q.y, q.z, q.w};
    uint32_t T = 0;   // bit i: window byte i has the high bit clear
#pragma unroll
    for (int k = 0; k < 8; ++k) T |= term4(W[k]) << (4 * k);
    const uint32_t Cn = ~T;   // bit i: window byte i continues
    // a run of ten continuation bytes ending in the slice (window bytes 16..31)
    const uint32_t r2 = Cn & (Cn << 1), r4 = r2 & (r2 << 2), r8 = r4 & (r4 << 4);
    const bool bad = (r8 & (r2 << 8) & 0xFFFF0000u) != 0;
    if (!kValues) return bad;
    const int s0 = kSlice * tid;
    uint32_t tc = T >> 16;   // the slice's terminators inside the input
    if (s0 < a || s0 + kSlice > b) {
#pragma unroll
        for (int j = 0; j < kSlice; ++j)
            if (s0 + j < a || s0 + j >= b) tc &= ~(1u << j);
    }
    if (!(r2 & 0xFFFF8000u)) {   // codes of at most two bytes
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const Pairs pr = pairs_le2(W[3 + j], W[4 + j]);
            uint32_t q01 = prmt(pr.lob, pr.hib, 0x5140u);
            uint32_t q23 = prmt(pr.lob, pr.hib, 0x7362u);
            q01 -= (q01 & 0xFF00FF00u) >> 1;
            q23 -= (q23 & 0xFF00FF00u) >> 1;
            const uint32_t v4[4] = {q01 & 0xFFFFu, q01 >> 16, q23 & 0xFFFFu, q23 >> 16};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((tc >> (4 * j + i)) & 1u) f(static_cast<uint64_t>(v4[i]));
        }
        return bad;
    }
    uint32_t m = tc;
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        const int Q = 16 + j;   // the terminator's window byte
        const uint32_t below = T & ((1u << Q) - 1u);
        const int L = below ? Q - (31 - __clz(below)) : Q + 1;   // over ten: malformed, the value unspecified
        const int st = Q - 7;                                    // the first of the eight bytes ending at Q
        const int w0 = st >> 2, sh = 8 * (st & 3);
        const uint32_t A = ww[w0], B = ww[w0 + 1];
        const uint32_t lo = __funnelshift_r(A, B, sh);
        const uint32_t hi = sh ? __funnelshift_r(B, ww[w0 + 2], sh) : B;
        // the eight payloads as 56 bits: group g is byte Q - 7 + g
        const uint64_t c56 = compact28(lo) | (static_cast<uint64_t>(compact28(hi)) << 28);
        uint64_t v;
        if (L <= 8) {
            v = c56 >> (7 * (8 - L));
        } else {   // nine or ten bytes: the tenth group's top bits fall off (x 2^63 modulo 2^64)
            v = (c56 << 7) | (wb[Q - 8] & 0x7Fu);
            if (L >= 10) v = (v << 7) | (wb[Q - 9] & 0x7Fu);
        }
        f(v);
    }
    return bad;
}

// Bytes with the high bit clear at tile positions [a, b) of this thread's slice.
__device__ __forceinline__ uint32_t slice_count(const uint8_t *bytes, int tid, int a, int b)
{
    const uint4 q = *reinterpret_cast<const uint4 *>(bytes + kHalo + kSlice * tid);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
    const int s0 = kSlice * tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t m = ~w[k] & 0x80808080u;
        if (s0 < a || s0 + kSlice > b) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int pos = s0 + 4 * k + j;
                if (pos < a || pos >= b) m &= ~(0x80u << (8 * j));
            }
        }
        cnt += __popc(m);
    }
    return cnt;
}

__device__ __forceinline__ uint32_t warp_sum32(uint32_t x)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, d);
    return x;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t x)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, d);
    return x;
}

template <class T>
__device__ __forceinline__ T warp_incl(T x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// Exclusive block scan over kThreads threads (wt: kWarps words of shared
// memory, free since the last barrier); *total gets the block's sum.
template <class T>
__device__ __forceinline__ T block_excl(T x, T *wt, T *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T inc = warp_incl(x, lane);
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    T before = 0, all = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
        const T v = wt[k];
        if (k < warp) before += v;
        all += v;
    }
    *total = all;
    return before + inc - x;
}

// Tile positions [a, b) of tile t that hold input bytes.
__device__ __forceinline__ void tile_range(const Params &p, uint64_t t, int *a, int *b)
{
    const int64_t t0 = static_cast<int64_t>(t) * kTile;
    *a = static_cast<int>(p.lo > t0 ? p.lo - t0 : 0);
    *b = static_cast<int>(p.hi - t0 < kTile ? p.hi - t0 : kTile);
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads) count64_kernel(Params p)
{
    __shared__ CountShared S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint64_t t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
        stage(p, t, S.bytes);
        __syncthreads();
        int a, b;
        tile_range(p, t, &a, &b);
        uint32_t cnt = 0;
        uint64_t sum = 0;
        cnt = slice_count(S.bytes, tid, a, b);
        const bool bad = values64<kDelta>(S.bytes, tid, a, b, [&](uint64_t v) { sum += v; });
        if (bad) atomicOr(p.status, VBYTE_ERR_MALFORMED_LONG);
        if (t + 1 == p.ntiles && b - 1 >= kSlice * tid && b - 1 < kSlice * (tid + 1) &&
            (S.bytes[kHalo + b - 1] & 0x80u))
            atomicOr(p.status, VBYTE_ERR_TRUNCATED);
        cnt = warp_sum32(cnt);
        if (kDelta) sum = warp_sum64(sum);
        if (lane == 0) {
            S.wcnt[warp] = cnt;
            S.wsum[warp] = sum;
        }
        __syncthreads();   // also: every slice of this tile is read before the next stage
        if (tid == 0) {
            uint64_t c = 0, s = 0;
#pragma unroll
            for (int k = 0; k < kWarps; ++k) {
                c += S.wcnt[k];
                s += S.wsum[k];
            }
            p.tcnt[t] = c;
            if (kDelta) p.tsum[t] = s;
        }
    }
}

// One CTA, 1024 tiles per round (coalesced), a carry between rounds.
template <bool kDelta>
__global__ void __launch_bounds__(kScanThreads) scan64_kernel(Params p)
{
    __shared__ unsigned long long wc[kScanThreads / 32], ws[kScanThreads / 32];
    __shared__ unsigned long long carry_c, carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry_c = 0;
        carry_s = p.prev;
    }
    __syncthreads();
    for (uint64_t b0 = 0; b0 < p.ntiles; b0 += kScanThreads) {
        const uint64_t i = b0 + tid;
        const uint64_t c = i < p.ntiles ? p.tcnt[i] : 0u;
        const uint64_t s = (kDelta && i < p.ntiles) ? p.tsum[i] : 0u;
        const uint64_t ci = warp_incl<uint64_t>(c, lane);
        const uint64_t si = kDelta ? warp_incl<uint64_t>(s, lane) : 0u;
        if (lane == 31) {
            wc[warp] = ci;
            ws[warp] = si;
        }
        __syncthreads();
        uint64_t cb = carry_c, sb = carry_s, tc = 0, ts = 0;
        for (int k = 0; k < kScanThreads / 32; ++k) {
            if (k < warp) {
                cb += wc[k];
                sb += ws[k];
            }
            tc += wc[k];
            ts += ws[k];
        }
        if (i < p.ntiles) {
            p.tcnt[i] = cb + ci - c;
            if (kDelta) p.tsum[i] = sb + si - s;
        }
        __syncthreads();
        if (tid == 0) {
            carry_c += tc;
            carry_s += ts;
        }
        __syncthreads();
    }
    if (tid == 0 && carry_c != p.n) atomicOr(p.status, VBYTE_ERR_COUNT_MISMATCH);
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads) decode64_kernel(Params p)
{
    __shared__ DecodeShared S;
    const int tid = threadIdx.x;
    for (uint64_t t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
        stage(p, t, S.bytes);
        __syncthreads();
        int a, b;
        tile_range(p, t, &a, &b);
        uint32_t C = 0;
        uint32_t rank = block_excl<uint32_t>(slice_count(S.bytes, tid, a, b), S.wcnt, &C);
        values64<true>(S.bytes, tid, a, b, [&](uint64_t v) { S.vals[slot(rank++)] = v; });
        __syncthreads();
        if (kDelta) {
            // running sums of the tile's integers from prev + everything before it
            const uint32_t j0 = kSlice * tid, j1 = min(j0 + kSlice, C);
            uint64_t run = 0;
            for (uint32_t j = j0; j < j1; ++j) run += S.vals[slot(j)];
            unsigned long long tot;
            uint64_t x = p.tsum[t] + block_excl<unsigned long long>(run, S.wsum, &tot);
            for (uint32_t j = j0; j < j1; ++j) {
                x += S.vals[slot(j)];
                S.vals[slot(j)] = x;
            }
            __syncthreads();
        }
        const uint64_t r0 = p.tcnt[t];
        for (uint32_t j = tid; j < C; j += kThreads) {
            const uint64_t g = r0 + j;
            if (g < p.n) p.out[g] = S.vals[slot(j)];
        }
        __syncthreads();   // the next stage and scan reuse S
    }
}

namespace {

int occupancy_grid(const void *kernel, int smem, uint64_t ntiles, int *grid)
{
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem) != cudaSuccess)
        return VBYTE_ECUDA;
    *grid = static_cast<int>(std::min<uint64_t>(ntiles, static_cast<uint64_t>(sms) * std::max(occ, 1)));
    return VBYTE_OK;
}

template <bool kDelta>
int enqueue(const Params &p, cudaStream_t s)
{
    int gc = 0, gd = 0;
    int rc = occupancy_grid(reinterpret_cast<const void *>(count64_kernel<kDelta>), 0, p.ntiles, &gc);
    if (rc == VBYTE_OK) rc = occupancy_grid(reinterpret_cast<const void *>(decode64_kernel<kDelta>), 0, p.ntiles, &gd);
    if (rc != VBYTE_OK) return rc;
    count64_kernel<kDelta><<<gc, kThreads, 0, s>>>(p);
    scan64_kernel<kDelta><<<1, kScanThreads, 0, s>>>(p);
    decode64_kernel<kDelta><<<gd, kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int launch(const uint8_t *in, size_t nbytes, uint64_t *out, size_t n, bool delta, uint64_t prev, cudaStream_t s)
{
    if (nbytes == 0 && n == 0) return VBYTE_OK;
    if ((nbytes && !in) || (n && !out)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(out) & 7u) return VBYTE_EINVAL;
    const uintptr_t ia = reinterpret_cast<uintptr_t>(in);
    const uint64_t lo = ia & 15u;
    const uint64_t ntiles = (lo + nbytes + kTile - 1) / kTile;
    uint8_t *ws = nullptr;
    const int rc = stream_workspace(s, kHead + 16 * ntiles, &ws);
    if (rc != VBYTE_OK) return rc;
    uint32_t *status = reinterpret_cast<uint32_t *>(ws);
    if (nbytes == 0) return set_status_async(status, VBYTE_ERR_COUNT_MISMATCH, s);   // n > 0 from no bytes
    Params p = {};
    p.base = reinterpret_cast<const uint8_t *>(ia - lo);
    p.lo = static_cast<int64_t>(lo);
    p.hi = static_cast<int64_t>(lo + nbytes);
    p.ntiles = ntiles;
    p.out = out;
    p.n = n;
    p.prev = prev;
    p.tcnt = reinterpret_cast<uint64_t *>(ws + kHead);
    p.tsum = p.tcnt + ntiles;
    p.status = status;
    return delta ? enqueue<true>(p, s) : enqueue<false>(p, s);
}

}  // namespace
}  // namespace d64
}  // namespace vbk

extern "C" {

int vbyte_decode64(const uint8_t *d_in, size_t nbytes, uint64_t *d_out, size_t n, void *stream)
{
    return vbk::d64::launch(d_in, nbytes, d_out, n, false, 0u, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta64(const uint8_t *d_in, size_t nbytes, uint64_t *d_out, size_t n, uint64_t prev,
                         void *stream)
{
    return vbk::d64::launch(d_in, nbytes, d_out, n, true, prev, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
