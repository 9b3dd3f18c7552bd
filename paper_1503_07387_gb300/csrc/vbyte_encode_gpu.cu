// Device encoder (vbyte_encode_device, vbyte_encode_delta_device).
//
// Operation (arXiv 1503.07387): the VByte format of Sec. 1 (Table 1): each
// uint32 is written least significant 7-bit group first, one group per
// byte, the high bit set on every byte but the last; its length is
// 1 + [v >= 2^7] + [v >= 2^14] + [v >= 2^21] + [v >= 2^28].  In delta mode
// the values written are the gaps x_i - x_{i-1} (mod 2^32) with
// x_{-1} = prev (Sec. 1, "Differential coding"); in the variant for lists
// without repeated values (kM1, named in the same paragraph) every gap after
// the first is one less.
//
// Design: one pass over the input with a decoupled look-back over tiles of
// 6144 values.  Persistent CTAs take tiles in ticket order; a CTA loads its
// tile, computes every value's length, publishes the tile's byte count,
// looks back over the words of earlier tiles for its byte offset, publishes
// its inclusive offset, encodes the tile into shared memory and writes it
// out with aligned 4-byte stores.  The published words carry their own
// state in their low two bits (1: the tile's count, 2: the count of every
// tile up to it) and are read and written with single 64-bit relaxed
// accesses after the workspace is cleared, so no step takes a fence.  Every
// wait is on a CTA holding an earlier ticket and is bounded by the global
// timer (VBYTE_ERR_TIMEOUT).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "vbyte.h"
#include "vbyte_device.cuh"
#include "vbyte_internal.h"

namespace vbk {
namespace enc {

constexpr int kLanes = 32;
constexpr int kThreads = 256;
constexpr int kVPT = 24;                             // values per thread
constexpr int kTileVals = kThreads * kVPT;           // 6144 values per tile
constexpr int kTileBytesMax = 5 * kTileVals;         // encoded bytes of a tile, at most
constexpr int kBuf = kTileBytesMax + 16;
static_assert(kVPT % 4 == 0, "vector loads of four values");

struct Params {
    const uint32_t *in;
    uint64_t n;
    uint8_t *out;
    uint64_t *nbytes;          // total encoded bytes (written by the last tile)
    uint64_t ntiles;
    uint64_t *tword;           // per tile: look-back word
    unsigned int *ctr;         // tickets
    uint32_t *status;
    uint32_t prev;             // x_{-1} in delta mode
    bool vec;                  // in is 16-byte aligned: vector loads
};

struct Shared {
    alignas(16) uint8_t bytes[kBuf];   // the tile, encoded
    uint32_t wsum[kThreads / 32];      // per-warp byte counts
    unsigned long long off;            // the tile's byte offset
    uint32_t tile;
};

__device__ __forceinline__ uint32_t vlen(uint32_t v)
{
    return 1u + (v >= (1u << 7)) + (v >= (1u << 14)) + (v >= (1u << 21)) + (v >= (1u << 28));
}

// Warp 0: the exclusive byte offset of tile t from the words of tiles t - 1,
// t - 2, ... (the nearest inclusive word ends the walk).  On a timeout the
// status word has VBYTE_ERR_TIMEOUT and the offset is 0.
__device__ uint64_t look_back(const Params &p, uint64_t t, int lane)
{
    uint64_t acc = 0;
    long long base = static_cast<long long>(t) - 1;
    while (base >= 0) {
        const long long j = base - lane;
        uint64_t w = 2u;   // before tile 0: an inclusive count of 0
        if (j >= 0) {
            w = ld_relaxed_u64(p.tword + j);
            if (!(w & 3u)) w = wait_bits(p.tword + j, 3u, p.status);
        }
        const unsigned incl = __ballot_sync(~0u, (w & 3u) == 2u);
        const int stop = incl ? __ffs(incl) - 1 : kLanes;   // nearest inclusive word in the window
        uint64_t v = lane <= stop ? (w >> 2) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
        acc += v;
        if (incl) break;
        base -= kLanes;
    }
    return acc;
}

template <bool kDelta, bool kM1 = false>
__global__ void __launch_bounds__(kThreads) encode_kernel(const Params p)
{
    __shared__ Shared S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) S.tile = atomicAdd(p.ctr, 1u);
        __syncthreads();
        const uint64_t t = S.tile;
        if (t >= p.ntiles) break;
        const uint64_t v0 = t * kTileVals + static_cast<uint64_t>(tid) * kVPT;   // my first value
        // my values (zeros past n: they are not written)
        uint32_t x[kVPT];
        if (p.vec && v0 + kVPT <= p.n) {
#pragma unroll
            for (int i = 0; i < kVPT; i += 4) {
                const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p.in + v0 + i));
                x[i] = a.x;
                x[i + 1] = a.y;
                x[i + 2] = a.z;
                x[i + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kVPT; ++i) x[i] = v0 + i < p.n ? __ldg(p.in + v0 + i) : 0u;
        }
        const int cnt = v0 >= p.n ? 0 : (p.n - v0 >= kVPT ? kVPT : static_cast<int>(p.n - v0));
        if (kDelta) {
            // the value before my first: the previous thread's last, or the
            // value before the tile
            uint32_t before = __shfl_up_sync(~0u, x[kVPT - 1], 1);
            if (lane == 0)
                before = v0 == 0 ? p.prev : (v0 - 1 < p.n ? __ldg(p.in + v0 - 1) : 0u);
#pragma unroll
            for (int i = kVPT - 1; i > 0; --i) x[i] -= x[i - 1] + (kM1 ? 1u : 0u);
            x[0] -= before + ((kM1 && v0 > 0) ? 1u : 0u);
        }
        uint32_t len = 0;
#pragma unroll
        for (int i = 0; i < kVPT; ++i) len += i < cnt ? vlen(x[i]) : 0u;
        // byte offsets within the tile
        const uint32_t inc = warp_incl_scan(len, lane);
        if (lane == 31) S.wsum[warp] = inc;
        __syncthreads();
        uint32_t wb = 0, tot = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            wb += q < warp ? S.wsum[q] : 0u;
            tot += S.wsum[q];
        }
        if (warp == 0) {
            uint64_t off = 0;
            if (t == 0) {
                if (lane == 0) st_relaxed_u64(p.tword, (static_cast<uint64_t>(tot) << 2) | 2u);
            } else {
                if (lane == 0) st_relaxed_u64(p.tword + t, (static_cast<uint64_t>(tot) << 2) | 1u);
                off = look_back(p, t, lane);
                if (lane == 0) st_relaxed_u64(p.tword + t, ((off + tot) << 2) | 2u);
            }
            if (lane == 0) {
                S.off = off;
                if (t == p.ntiles - 1) *p.nbytes = off + tot;
            }
        }
        // encode my values into the staged tile: byte k of a value of length
        // L is its k-th 7-bit group, with the high bit set while k < L - 1
        // (the first four groups spread to the four bytes of one word)
        uint32_t o = wb + inc - len;
#pragma unroll
        for (int i = 0; i < kVPT; ++i) {
            if (i < cnt) {
                const uint32_t v = x[i];
                const uint32_t L = vlen(v);
                const uint32_t g = (v & 0x7Fu) | ((v << 1) & 0x7F00u) | ((v << 2) & 0x7F0000u) | ((v << 3) & 0x7F000000u);
                const uint32_t w = g | static_cast<uint32_t>(0x80808080ull >> (8 * (5 - L)));
                S.bytes[o] = static_cast<uint8_t>(w);
                if (L > 1) S.bytes[o + 1] = static_cast<uint8_t>(w >> 8);
                if (L > 2) S.bytes[o + 2] = static_cast<uint8_t>(w >> 16);
                if (L > 3) S.bytes[o + 3] = static_cast<uint8_t>(w >> 24);
                if (L > 4) S.bytes[o + 4] = static_cast<uint8_t>(v >> 28);
                o += L;
            }
        }
        __syncthreads();
        // the tile's bytes [0, tot) to out + off: aligned 4-byte words in the
        // middle, single bytes at the two ends
        const uint64_t off = S.off;
        uint8_t *const dst = p.out + off;
        const uint32_t head = static_cast<uint32_t>((4u - (reinterpret_cast<uintptr_t>(dst) & 3u)) & 3u);
        const uint32_t h = min(head, tot);
        if (static_cast<uint32_t>(tid) < h) dst[tid] = S.bytes[tid];
        const uint32_t nw = (tot - h) >> 2;   // whole words after the head
        uint32_t *const dw = reinterpret_cast<uint32_t *>(dst + h);
        const uint32_t *const sw = reinterpret_cast<const uint32_t *>(S.bytes);
        const uint32_t sh = 8u * (h & 3u);   // staged word alignment of byte h
        for (uint32_t w = tid; w < nw; w += kThreads) {
            const uint32_t b = h + 4u * w;        // first staged byte of this word
            const uint32_t lo = sw[b >> 2], hi = sw[(b >> 2) + 1];
            dw[w] = sh ? __funnelshift_r(lo, hi, sh) : lo;
        }
        const uint32_t tail0 = h + 4u * nw;
        if (static_cast<uint32_t>(tid) < tot - tail0) dst[tail0 + tid] = S.bytes[tail0 + tid];
        __syncthreads();   // S.bytes and S.tile are reused by the next tile
    }
}

}  // namespace enc

namespace {

int launch_encode(const uint32_t *in, size_t n, bool delta, uint32_t prev, uint8_t *out, uint64_t *d_nbytes,
                  cudaStream_t s, bool m1 = false)
{
    if ((n && (!in || !out)) || !d_nbytes) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(in) & 3u) return VBYTE_EINVAL;
    if (n == 0) return cudaMemsetAsync(d_nbytes, 0, sizeof(uint64_t), s) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
    const uint64_t ntiles = (n + enc::kTileVals - 1) / enc::kTileVals;
    if (ntiles >= (1ull << 31)) return VBYTE_EINVAL;
    // workspace: the status head, a ticket counter, one word per tile
    constexpr size_t kCtr = 256, kWords = 272;
    const size_t need = kWords + 8 * ntiles;
    uint8_t *ws = nullptr;
    int rc = stream_workspace(s, need, &ws);
    if (rc != VBYTE_OK) return rc;
    if (cudaMemsetAsync(ws + kCtr, 0, need - kCtr, s) != cudaSuccess) return VBYTE_ECUDA;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return VBYTE_ECUDA;
    if (m1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, enc::encode_kernel<true, true>, enc::kThreads, 0);
    else if (delta)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, enc::encode_kernel<true>, enc::kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, enc::encode_kernel<false>, enc::kThreads, 0);
    enc::Params p = {};
    p.in = in;
    p.n = n;
    p.out = out;
    p.nbytes = d_nbytes;
    p.ntiles = ntiles;
    p.tword = reinterpret_cast<uint64_t *>(ws + kWords);
    p.ctr = reinterpret_cast<unsigned int *>(ws + kCtr);
    p.status = reinterpret_cast<uint32_t *>(ws);
    p.prev = prev;
    p.vec = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
    const uint64_t grid = std::min<uint64_t>(ntiles, static_cast<uint64_t>(sms) * std::max(occ, 1));
    if (m1)
        enc::encode_kernel<true, true><<<static_cast<unsigned>(grid), enc::kThreads, 0, s>>>(p);
    else if (delta)
        enc::encode_kernel<true><<<static_cast<unsigned>(grid), enc::kThreads, 0, s>>>(p);
    else
        enc::encode_kernel<false><<<static_cast<unsigned>(grid), enc::kThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace
}  // namespace vbk

extern "C" {

int vbyte_encode_device(const uint32_t *d_in, size_t n, uint8_t *d_out, uint64_t *d_nbytes, void *stream)
{
    return vbk::launch_encode(d_in, n, false, 0u, d_out, d_nbytes, static_cast<cudaStream_t>(stream));
}

int vbyte_encode_delta_device(const uint32_t *d_in, size_t n, uint32_t prev, uint8_t *d_out, uint64_t *d_nbytes,
                              void *stream)
{
    return vbk::launch_encode(d_in, n, true, prev, d_out, d_nbytes, static_cast<cudaStream_t>(stream));
}

int vbyte_encode_delta_m1_device(const uint32_t *d_in, size_t n, uint32_t prev, uint8_t *d_out,
                                 uint64_t *d_nbytes, void *stream)
{
    return vbk::launch_encode(d_in, n, true, prev, d_out, d_nbytes, static_cast<cudaStream_t>(stream), true);
}

}  // extern "C"
