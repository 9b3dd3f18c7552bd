// Copy-out of a warp's decoded values: from the warp's value buffer (values
// at warp rank r in vals[4 + r]) or, for a warp of one-byte integers only,
// straight from its staged bytes, to the output with coalesced 16-byte
// stores realigned to the output's 16-byte boundaries.  Shared by the
// decoders of vbyte_stream.cu and vbyte_split.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vbyte_device.cuh"

namespace vbk {

constexpr int kEmitLanes = 32;

// Output quad q of a warp holds its ranks 4q - SH .. 4q - SH + 3, staged at
// vals[4q + 4 - SH ..]: the tail of U = vals[4q..] and the head of
// V = vals[4q+4..].
template <int SH>
__device__ __forceinline__ uint4 staged_quad(const uint32_t *vals, int q)
{
    const uint4 V = *reinterpret_cast<const uint4 *>(vals + 4 * q + 4);
    if (SH == 0) return V;
    const uint4 U = *reinterpret_cast<const uint4 *>(vals + 4 * q);
    if (SH == 1) return make_uint4(U.w, V.x, V.y, V.z);
    if (SH == 2) return make_uint4(U.z, U.w, V.x, V.y);
    return make_uint4(U.y, U.z, U.w, V.x);
}

// A warp's staged values to the output, SH = (output word of rank 0) mod 4.
// Output quad q holds ranks 4q - SH .. 4q - SH + 3, staged at
// vals[4q + 4 - SH ..]; quads [qa, qb) are whole (inside the warp's ranks and
// below `room`, the ranks the output still holds); the ranks outside them
// are written one per lane.  `add` goes to every rank; with kRank the rank
// itself too, counted from rb (the gaps-minus-one variant).
template <int SH, bool kRank>
__device__ __forceinline__ void emit_staged(uint32_t *oq, const uint32_t *vals, int wc, uint32_t add, uint32_t rb,
                                            long long room, int lane)
{
    constexpr int qa = SH ? 1 : 0;
    const int lim = room < wc ? (room > 0 ? static_cast<int>(room) : 0) : wc;   // ranks [0, lim) are written
    const int qb = (lim + SH) >> 2;
#pragma unroll 2
    for (int q = qa + lane; q < qb; q += kEmitLanes) {
        uint4 e = staged_quad<SH>(vals, q);
        const uint32_t a0 = add + (kRank ? rb + static_cast<uint32_t>(4 * q - SH) : 0u);
        e.x += a0;
        e.y += a0 + (kRank ? 1u : 0u);
        e.z += a0 + (kRank ? 2u : 0u);
        e.w += a0 + (kRank ? 3u : 0u);
        st_quad(oq + 4 * q, e);
    }
    const bool whole = qb > qa;
    const int hb = whole ? min(4 * qa - SH, lim) : lim;   // ranks [0, hb)
    const int tb = whole ? 4 * qb - SH : lim;             // ranks [tb, lim)
    for (int r = lane; r < hb; r += kEmitLanes)
        oq[SH + r] = vals[4 + r] + add + (kRank ? rb + static_cast<uint32_t>(r) : 0u);
    for (int r = tb + lane; r < lim; r += kEmitLanes)
        oq[SH + r] = vals[4 + r] + add + (kRank ? rb + static_cast<uint32_t>(r) : 0u);
}

template <bool kRank>
__device__ __forceinline__ void emit_staged(uint32_t *oq, const uint32_t *vals, int wc, uint32_t add, uint32_t rb,
                                            long long room, int lane, int sh)
{
    switch (sh) {   // warp-uniform
    case 0: emit_staged<0, kRank>(oq, vals, wc, add, rb, room, lane); break;
    case 1: emit_staged<1, kRank>(oq, vals, wc, add, rb, room, lane); break;
    case 2: emit_staged<2, kRank>(oq, vals, wc, add, rb, room, lane); break;
    default: emit_staged<3, kRank>(oq, vals, wc, add, rb, room, lane); break;
    }
}

// Component k of v (k in 0..3).
__device__ __forceinline__ uint32_t pick4(uint4 v, uint32_t k)
{
    return (k & 2u) ? ((k & 1u) ? v.w : v.z) : ((k & 1u) ? v.y : v.x);
}

// The same copy-out with an addend per output word position within its
// 16-byte quad (add4.x for the words on 16-byte boundaries, add4.y for the
// next ones, ...): in the blocked-difference variant that position fixes a
// value's class (its rank modulo 4).
template <int SH>
__device__ __forceinline__ void emit_staged4(uint32_t *oq, const uint32_t *vals, int wc, uint4 add4, long long room,
                                             int lane)
{
    constexpr int qa = SH ? 1 : 0;
    const int lim = room < wc ? (room > 0 ? static_cast<int>(room) : 0) : wc;
    const int qb = (lim + SH) >> 2;
    for (int q = qa + lane; q < qb; q += kEmitLanes) {
        uint4 e = staged_quad<SH>(vals, q);
        e.x += add4.x;
        e.y += add4.y;
        e.z += add4.z;
        e.w += add4.w;
        st_quad(oq + 4 * q, e);
    }
    const bool whole = qb > qa;
    const int hb = whole ? min(4 * qa - SH, lim) : lim;
    const int tb = whole ? 4 * qb - SH : lim;
    for (int r = lane; r < hb; r += kEmitLanes) oq[SH + r] = vals[4 + r] + pick4(add4, (SH + r) & 3);
    for (int r = tb + lane; r < lim; r += kEmitLanes) oq[SH + r] = vals[4 + r] + pick4(add4, (SH + r) & 3);
}

__device__ __forceinline__ void emit_staged4(uint32_t *oq, const uint32_t *vals, int wc, uint4 add4, long long room,
                                             int lane, int sh)
{
    switch (sh) {   // warp-uniform
    case 0: emit_staged4<0>(oq, vals, wc, add4, room, lane); break;
    case 1: emit_staged4<1>(oq, vals, wc, add4, room, lane); break;
    case 2: emit_staged4<2>(oq, vals, wc, add4, room, lane); break;
    default: emit_staged4<3>(oq, vals, wc, add4, room, lane); break;
    }
}

// The copy-out of a one-byte warp from its staged bytes (wb: its first byte;
// the 4 bytes before and after it are staged too).  Output quad Q = 32m + l,
// taken by lane l, holds ranks 4Q - SH .. 4Q - SH + 3, whose bytes start at
// wb + 4Q - SH.  In delta mode the sums before each quad come from two
// packed warp scans (a quad's sum is at most 4 * 127, so 16 bits hold a
// warp's prefix).  Quad 0 skips the SH ranks before the warp; lane 31 writes
// the last SH ranks after quad 127.  With kRank each value also gets its
// rank, counted from rb.
template <int SH, bool kDelta, bool kRank>
__device__ __forceinline__ void emit_bytes_a(uint32_t *oq, const uint8_t *wb, uint32_t add, uint32_t rb, int lane)
{
    const uint32_t *ww = reinterpret_cast<const uint32_t *>(wb);
    uint32_t x[4], qs[4], P[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int k = 32 * m + lane;
        x[m] = SH == 0 ? ww[k] : __funnelshift_r(ww[k - 1], ww[k], 8 * (4 - SH));
    }
    if (SH > 0 && lane == 0) x[0] &= 0xFFFFFFFFu << (8 * SH);   // ranks before the warp
    if (kDelta) {
#pragma unroll
        for (int m = 0; m < 4; ++m) qs[m] = __dp4a(x[m], 0x01010101u, 0u);
        const uint32_t o01 = qs[0] | (qs[1] << 16), o23 = qs[2] | (qs[3] << 16);
        const uint32_t s01 = warp_incl_scan(o01, lane), s23 = warp_incl_scan(o23, lane);
        const uint32_t t01 = __shfl_sync(~0u, s01, 31), t23 = __shfl_sync(~0u, s23, 31);
        const uint32_t e01 = s01 - o01, e23 = s23 - o23;
        P[0] = e01 & 0xFFFFu;
        P[1] = (t01 & 0xFFFFu) + (e01 >> 16);
        P[2] = (t01 & 0xFFFFu) + (t01 >> 16) + (e23 & 0xFFFFu);
        P[3] = (t01 & 0xFFFFu) + (t01 >> 16) + (t23 & 0xFFFFu) + (e23 >> 16);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        uint32_t e[4];
        uint32_t run = kDelta ? add + P[m] : add;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t b = (x[m] >> (8 * j)) & 0xFFu;
            if (kDelta) {
                run += b;
                e[j] = run;
            } else {
                e[j] = b + add;
            }
        }
        if (kRank) {
            const uint32_t r0 = rb + static_cast<uint32_t>(4 * (32 * m + lane) - SH);
#pragma unroll
            for (int j = 0; j < 4; ++j) e[j] += r0 + j;
        }
        uint32_t *const o = oq + 4 * (32 * m + lane);
        if (SH == 0 || m > 0 || lane > 0) {
            st_quad(o, make_uint4(e[0], e[1], e[2], e[3]));
        } else {
#pragma unroll
            for (int j = SH; j < 4; ++j) o[j] = e[j];
        }
    }
    if (SH > 0 && lane == kEmitLanes - 1) {   // quad 128: ranks 512 - SH .. 511
        const uint32_t xt = __funnelshift_r(ww[127], ww[128], 8 * (4 - SH));
        uint32_t run = kDelta ? add + P[3] + qs[3] : add;
#pragma unroll
        for (int j = 0; j < SH; ++j) {
            const uint32_t b = (xt >> (8 * j)) & 0xFFu;
            const uint32_t rk = kRank ? rb + static_cast<uint32_t>(4 * 128 + j - SH) : 0u;
            if (kDelta) {
                run += b;
                oq[4 * 128 + j] = run + rk;
            } else {
                oq[4 * 128 + j] = b + add + rk;
            }
        }
    }
}

}  // namespace vbk
