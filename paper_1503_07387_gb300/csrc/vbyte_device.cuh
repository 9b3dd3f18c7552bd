// Device helpers shared by the decode kernels: inline PTX wrappers, the
// terminator mask, value assembly, warp scans and the per-slice count/sum of
// a staged tile (a halo of 16 bytes, then 16 bytes per thread or lane).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vbyte.h"

namespace vbk {

constexpr int kBPT = 16;                          // input bytes per thread (one slice)
constexpr int kHalo = 16;                         // bytes staged before a tile
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bound of every spin-wait

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ void st_quad(uint32_t *p, uint4 v)
{
    asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N committed groups of this thread are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait_prior()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Words published between CTAs carry their own validity: bit 0 is set in
// every written value and the workspace is cleared before each launch, so a
// reader needs no fence -- one 64-bit relaxed access is the whole protocol.
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One thread waits until *p has one of the bits of `mask` set, bounded by
// the global timer (limit_ns); on expiry, or once another wait of the launch
// has expired, the status word has VBYTE_ERR_TIMEOUT and 0 is returned.
__device__ __forceinline__ uint64_t wait_bits(const uint64_t *p, uint64_t mask, uint32_t *status,
                                              uint64_t limit_ns = kWaitLimitNs)
{
    uint64_t t0 = 0;
    for (int spin = 0;; ++spin) {
        const uint64_t v = ld_relaxed_u64(p);
        if (v & mask) return v;
        const uint64_t now = global_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > limit_ns) {
            atomicOr(status, VBYTE_ERR_TIMEOUT);
            return 0u;
        }
        if (spin > 4) {
            if (*reinterpret_cast<volatile uint32_t *>(status) & VBYTE_ERR_TIMEOUT) return 0u;
            __nanosleep(200);
        }
    }
}

// The same for bit 0 (a published word).
__device__ __forceinline__ uint64_t wait_word(const uint64_t *p, uint32_t *status, uint64_t limit_ns = kWaitLimitNs)
{
    return wait_bits(p, 1u, status, limit_ns);
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
// The compaction runs scaled by 8 (each step moves the lower field up rather
// than the upper one down), so that its joins are multiply-adds, which run on
// the multiply-add pipe while the masks and shifts use the integer ALU pipe
// that bounds the decoders: 2t = 2 (lo4 & 0x007F007F) + (lo4 & 0x7F007F00),
// 8u = 4 (2t & 0x7FFE) + (2t & 0x7FFE0000) with u the 28-bit compaction, and
// the 38-bit number 8 (u + x 2^28) is split into its low word
// 8u + (x & 1) 2^31 (8u < 2^31) and its high word x >> 1.
__device__ __forceinline__ uint32_t assemble(uint32_t lo4, uint32_t x, int L)
{
    const uint32_t t2 = (lo4 & 0x007F007Fu) * 2u + (lo4 & 0x7F007F00u);
    const uint32_t u8 = (t2 & 0x00007FFEu) * 4u + (t2 & 0x7FFE0000u);
    return __funnelshift_r(u8 + x * 0x80000000u, x >> 1, 38 - 7 * L);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(~0u, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ uint32_t byte_sum4(uint4 w)
{
    return __dp4a(w.x, 0x01010101u, __dp4a(w.y, 0x01010101u, __dp4a(w.z, 0x01010101u,
                                                                      __dp4a(w.w, 0x01010101u, 0u))));
}

__device__ __forceinline__ uint4 bytes_as_values(uint32_t x)
{
    return make_uint4(prmt(x, 0u, 0x4440u), prmt(x, 0u, 0x4441u), prmt(x, 0u, 0x4442u),
                      prmt(x, 0u, 0x4443u));
}

// 0xFF in byte i of the result iff bit i of the nibble m is set.
__device__ __forceinline__ uint32_t nibble_to_bytes(uint32_t m)
{
    return ((m * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// Codes of at most two bytes (SWAR over one 4-byte word c, wp the word before
// it): lob holds each integer's low 7-bit group and hib its high byte, at the
// position of the integer's terminator.
struct Pairs {
    uint32_t lob, hib;
};

__device__ __forceinline__ Pairs pairs_le2(uint32_t wp, uint32_t c)
{
    const uint32_t s = __funnelshift_l(wp, c, 8);   // byte i: the byte before byte i
    const uint32_t cm = prmt(s, 0u, 0xBA98u);        // 0xFF where that byte continues
    Pairs r;
    r.lob = (s & 0x7F7F7F7Fu & cm) | (c & ~cm);
    r.hib = c & cm;
    return r;
}

// Sum of the values whose terminators are marked in tc, for a thread whose
// codes are all at most two bytes long.
__device__ __forceinline__ uint32_t sum_le2(uint4 w, uint32_t wprev, uint32_t tc)
{
    const uint32_t c4[4] = {w.x, w.y, w.z, w.w};
    uint32_t wp = wprev, s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const Pairs pr = pairs_le2(wp, c4[j]);
        const uint32_t tm = nibble_to_bytes((tc >> (4 * j)) & 0xFu);
        s += __dp4a(pr.lob & tm, 0x01010101u, 0u) + (__dp4a(pr.hib & tm, 0x01010101u, 0u) << 7);
        wp = c4[j];
    }
    return s;
}

// Per-terminator assembly for codes of any length.  Calls emit(value) for each
// terminator marked in tc, in order.  t20 bits 0..3 describe the four bytes
// before the thread's slice, bits 4..19 the slice; sw is the staged tile.
template <typename F>
__device__ __forceinline__ void assemble_all(const uint32_t *sw, int tid, uint32_t tl, uint32_t t20,
                                             uint32_t tc, F emit)
{
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
            emit(assemble(lo4, x, L));
        }
    }
}

// The same from registers: wp is the word before the slice, w the slice.  The
// word pair holding a terminator's four preceding bytes and itself is picked
// by selects (no shared-memory loads, so no bank conflicts between lanes
// whose slices lie 16 bytes apart).
template <typename F>
__device__ __forceinline__ void assemble_regs(uint32_t wp, uint4 w, uint32_t tl, uint32_t t20, uint32_t tc, F emit)
{
    uint32_t m = tl & tc;
    int prevo = 27 - __clz(t20 & 0xFu);   // last terminator before my bytes (-5: none)
    uint32_t all = tl;                     // every terminator, for the code lengths
    while (m) {
        const int o = __ffs(m) - 1;
        m &= m - 1u;
        const uint32_t below = all & ((1u << o) - 1u);   // terminators of the slice before o
        const int po = below ? 31 - __clz(below) : prevo;
        const int L = min(o - po, 5);
        const int k = o >> 2;
        const uint32_t A = (k & 2) ? ((k & 1) ? w.z : w.y) : ((k & 1) ? w.x : wp);
        const uint32_t B = (k & 2) ? ((k & 1) ? w.w : w.z) : ((k & 1) ? w.y : w.x);
        const uint32_t lo4 = __funnelshift_r(A, B, 8 * (o & 3));
        const uint32_t x = prmt(B, 0u, 0x4440u | static_cast<uint32_t>(o & 3));
        emit(assemble(lo4, x, L));
    }
}

// 1 in each byte of w that has its high bit set (a continuation byte).
__device__ __forceinline__ uint32_t cont_flags(uint32_t w) { return (w >> 7) & 0x01010101u; }

// Sum of the values whose terminators lie in a thread's slice, without
// assembling them, for codes of any length (every byte inside the stream):
// each byte's 7-bit payload p times 128^k, k = its place within its integer
// (the number of continuation bytes right before it, at most four), summed
// over the bytes of those values -- from the first byte after the last
// terminator before the slice through the slice's last terminator.  With
// a_i = the sum of p over those bytes with k >= i, the sum is
// a_0 + 127 (a_1 + 128 (a_2 + 128 (a_3 + 128 a_4))) modulo 2^32, since
// 128^k = 1 + 127 (1 + 128 + ... + 128^(k-1)); a_1 + 128 a_2 and
// a_3 + 128 a_4 are one byte dot product each (weights 0, 1 or 129, see
// place_sums).  The bytes before the four before the slice count as
// terminators, which holds in a well-formed stream whenever it matters (a
// run of five continuation bytes is malformed).
__device__ __forceinline__ uint32_t sum_any_fast(uint4 w, uint32_t wp, uint32_t tl, uint32_t t20)
{
    if (!tl) return 0u;
    const uint32_t lt = 31u - __clz(tl);                    // last terminator of the slice
    const uint32_t low = t20 & 0xFu;
    const uint32_t st = low ? 32u - __clz(low) : 0u;        // first byte of the first value (t20 bits)
    const uint32_t mem = ((2u << (lt + 4u)) - 1u) & (~0u << st);
    const uint32_t W[5] = {wp, w.x, w.y, w.z, w.w};
    uint32_t a0 = 0, a12 = 0, a34 = 0;
    uint32_t cpv = 0u;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint32_t P = W[i] & 0x7F7F7F7Fu & nibble_to_bytes((mem >> (4 * i)) & 0xFu);
        const uint32_t cc = cont_flags(W[i]);
        // 1 in byte b iff byte b-1 (b-1 and b-2, ..., b-1 .. b-4) continues
        const uint32_t m1 = __funnelshift_l(cpv, cc, 8);
        const uint32_t m2 = m1 & __funnelshift_l(cpv, cc, 16);
        const uint32_t m3 = m2 & __funnelshift_l(cpv, cc, 24);
        const uint32_t m4 = m3 & cpv;
        a0 = __dp4a(P, 0x01010101u, a0);
        a12 = __dp4a(P, m2 * 128u + m1, a12);
        a34 = __dp4a(P, m4 * 128u + m3, a34);
        cpv = cc;
    }
    return a0 + 127u * (a12 + 16384u * a34);
}

// One word c of a stream (cpv = cont_flags of the word before it): adds the
// 7-bit payloads p of the bytes marked 0xFF in keep to a[0], p [k >= 1] +
// 128 p [k >= 2] to a[1] and p [k >= 3] + 128 p [k >= 4] to a[2], k the
// byte's place within its integer (the continuation bytes right before it,
// at most four); returns cont_flags(c) for the next word.  Summed over the
// bytes of some integers, a[0] + 127 (a[1] + 16384 a[2]) is the sum of their
// values modulo 2^32, since each payload p at place k then counts
// p (1 + 127 (1 + 128 + ... + 128^(k-1))) = p 128^k.  The place flags are
// 0 or 1 per byte, so each pair of places is one byte dot product with
// weights 0, 1 or 129 (place k >= 2 implies k >= 1), and the weight words
// are multiply-adds.
__device__ __forceinline__ uint32_t place_sums(uint32_t cpv, uint32_t c, uint32_t keep, uint32_t (&a)[3])
{
    const uint32_t cc = cont_flags(c);
    // 1 in byte b iff byte b-1 (b-1 and b-2, ..., b-1 .. b-4) continues
    const uint32_t m1 = __funnelshift_l(cpv, cc, 8);
    const uint32_t m2 = m1 & __funnelshift_l(cpv, cc, 16);
    const uint32_t m3 = m2 & __funnelshift_l(cpv, cc, 24);
    const uint32_t m4 = m3 & cpv;
    const uint32_t P = c & keep & 0x7F7F7F7Fu;
    a[0] = __dp4a(P, 0x01010101u, a[0]);
    a[1] = __dp4a(P, m2 * 128u + m1, a[1]);
    a[2] = __dp4a(P, m4 * 128u + m3, a[2]);
    return cc;
}

// Nonzero iff some 4-byte word of the slice holds two or more terminators
// (tl: one bit per byte, four per word).
__device__ __forceinline__ uint32_t dense_words(uint32_t tl)
{
    return ((tl & (tl >> 1)) & 0x7777u) | ((tl & (tl >> 2)) & 0x3333u) | ((tl & (tl >> 3)) & 0x1111u);
}

// Values of a slice whose words each hold at most one terminator
// (dense_words(tl) == 0) and lie inside the stream, all four words at once
// and without branches: v[j] is the value ending in word j when bit j of the
// result is set.  A value's length follows from the terminator of the word
// before it (the last one, for the word before the slice): none there means
// five bytes -- or more, which is malformed and reported by the count pass.
__device__ __forceinline__ uint32_t words4(uint32_t wp, uint4 w, uint32_t tl, uint32_t t20, uint32_t (&v)[4])
{
    const uint32_t W[5] = {wp, w.x, w.y, w.z, w.w};
    int prev = 31 - __clz(t20 & 0xFu);   // last terminator of the word before (-1: none)
    uint32_t nz = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t nib = (tl >> (4 * j)) & 0xFu;
        const int o4 = 31 - __clz(nib);   // the word's terminator (-1: none)
        const int L = min(4 + o4 - prev, 5);
        // (a word with no terminator, o4 = -1, yields a value that is not used)
        const uint32_t sh = static_cast<uint32_t>(o4);
        v[j] = assemble(__funnelshift_r(W[j], W[j + 1], 8 * sh), prmt(W[j + 1], 0u, 0x4440u | sh), L);
        nz |= (nib ? 1u : 0u) << j;
        prev = o4;
    }
    return nz;
}

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

// Terminator masks of tid's 16-byte slice of a staged tile.
struct SliceMasks {
    uint4 w;          // the slice
    uint32_t wprev;   // the 4 bytes before it
    uint32_t tl;      // terminator bits of the slice
    uint32_t t20;     // bits 0..3: the 4 bytes before, 4..19: the slice
    uint32_t tc;      // terminators inside the stream
};

__device__ __forceinline__ SliceMasks slice_masks(const uint8_t *bt, int tid, bool interior, uintptr_t va,
                                                  uintptr_t lo, uintptr_t hi)
{
    SliceMasks m;
    m.w = *reinterpret_cast<const uint4 *>(bt + kHalo + tid * kBPT);
    m.wprev = reinterpret_cast<const uint32_t *>(bt)[(kHalo + tid * kBPT) / 4 - 1];
    m.tl = term4(m.w.x) | (term4(m.w.y) << 4) | (term4(m.w.z) << 8) | (term4(m.w.w) << 12);
    m.t20 = term4(m.wprev) | (m.tl << 4);
    m.tc = interior ? m.tl : (m.tl & slice_valid(va, lo, hi));
    return m;
}

// Sum of the values whose terminators lie in a thread's slice, for a thread
// whose codes are at most two bytes (every continuation byte is followed by
// its terminator): the 7-bit payloads of the bytes of those values plus 127
// times each two-byte value's high byte.  The byte before the slice belongs
// to my first value when it is a continuation byte; my last byte belongs to
// the next slice's first value when it is one.
__device__ __forceinline__ uint32_t sum_le2_fast(uint4 w, uint32_t wprev)
{
    const uint32_t c4[4] = {w.x, w.y, w.z, w.w};
    uint32_t s = 0, hi = 0, wp = wprev;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t c = c4[j];
        s = __dp4a(c & 0x7F7F7F7Fu, 0x01010101u, s);
        const uint32_t sh = __funnelshift_l(wp, c, 8);      // byte i: the byte before byte i
        hi = __dp4a(c & prmt(sh, 0u, 0xBA98u), 0x01010101u, hi);
        wp = c;
    }
    if (wprev & 0x80000000u) s += (wprev >> 24) & 0x7Fu;   // my first value started earlier
    if (w.w & 0x80000000u) s -= (w.w >> 24) & 0x7Fu;       // my last byte starts the next value
    return s + 127u * hi;
}

// ---- list heads (batched decoding) ---------------------------------------
constexpr int kHeadTile = 4096;                          // tile bytes of the decoders using these
constexpr int kHeadBack = 8;                             // window start before a tile or slice
constexpr int kHeadWords = (kHalo + kHeadTile) / 32 + 2; // head bitmap of a staged tile
// ---- segmented sums (batched differential decoding) ----------------------
// A list head restarts the running value at that list's x_0.  A slice of
// integers acts on the running value x as: f ? s : x + s, where f says that a
// head was crossed and s is the sum since the last head (including its x_0).
struct Seg {
    uint32_t f, s;
};

__device__ __forceinline__ Seg seg_op(Seg a, Seg b)
{
    Seg r;
    r.f = a.f | b.f;
    r.s = b.f ? b.s : a.s + b.s;
    return r;
}

__device__ __forceinline__ uint32_t seg_apply(uint32_t x, Seg a) { return a.f ? a.s : x + a.s; }

__device__ __forceinline__ Seg warp_seg_incl(Seg x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ys = __shfl_up_sync(~0u, x.s, o);
        const uint32_t yf = __shfl_up_sync(~0u, x.f, o);
        if (lane >= o) {
            if (!x.f) x.s += ys;
            x.f |= yf;
        }
    }
    return x;
}

// The list heads of a tile in shared memory: a bitmap of their first bytes
// over the staged window (bit i: staging byte i, the 16 halo bytes first)
// and, for the first kMaxHeadList lists of the tile's range [ha, he), each
// list's staging index, x_0 and value offset, so that lookups stay on chip.
constexpr int kMaxHeadList = 256;
struct HeadTab {
    int pos[kMaxHeadList];
    uint32_t prv[kMaxHeadList];
    unsigned long long vo[kMaxHeadList];
    uint32_t bits[kHeadWords];
};

// Where the list heads come from: byte offsets, value offsets and x_0 of
// every list (prevs may be null: x_0 = 0).
struct HeadSrc {
    const uint64_t *bo;
    const uint64_t *vo;
    const uint32_t *prevs;
};

// Fill T for the tile starting at stream offset trel (threads of a CTA of
// nthreads take part; the caller syncs before and after as documented).
__device__ __forceinline__ void fill_heads(const HeadSrc &p, long long trel, uint64_t ha, uint64_t he, HeadTab &T,
                                           bool want_prev, bool want_vo, int nthreads)
{
    const int tid = threadIdx.x;
    const long long w0 = trel - kHalo;
    const uint64_t nh = he - ha;
    for (uint64_t i = tid; i < nh; i += nthreads) {
        const uint64_t j = ha + i;
        const long long d = static_cast<long long>(p.bo[j]) - w0;
        if (d >= 0 && d < kHalo + kHeadTile) atomicOr(T.bits + (d >> 5), 1u << (d & 31));
        if (i < static_cast<uint64_t>(kMaxHeadList)) {
            T.pos[i] = d < 0 ? -1 : (d > (1 << 30) ? (1 << 30) : static_cast<int>(d));
            if (want_prev) T.prv[i] = p.prevs ? p.prevs[j] : 0u;
            if (want_vo) T.vo[i] = p.vo[j];
        }
    }
}

// Index of the last table entry whose staging index is <= q (-1 if none).
__device__ __forceinline__ int tab_last_le(const HeadTab &T, int n, int q)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T.pos[mid] <= q)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo - 1;
}

// The 24 staged bytes ending with tid's slice: terminator bits (t24) and head
// bits (h24); bit i is staging byte kHalo + 16*tid - kHeadBack + i.
struct HeadWin {
    uint32_t t24, h24;
};

__device__ __forceinline__ HeadWin head_window(const uint32_t *sw, const uint32_t *bits, int tid, uint32_t tl)
{
    HeadWin h;
    const int q = (kHalo + tid * kBPT) / 4;
    h.t24 = term4(sw[q - 2]) | (term4(sw[q - 1]) << 4) | (tl << 8);
    const int b0 = kHalo + tid * kBPT - kHeadBack;   // a multiple of 8
    h.h24 = __funnelshift_r(bits[b0 >> 5], bits[(b0 >> 5) + 1], b0 & 31) & 0xFFFFFFu;
    return h;
}

// Terminators (slice bits) that end the first integer of a list: the integer
// starting at a head bit h ends at the first terminator at or after h.  Adding
// h to the non-terminator mask carries from h through the continuation bytes
// into exactly that terminator.
__device__ __forceinline__ uint32_t head_terms(const HeadWin &h, uint32_t tc)
{
    const uint32_t r = ~h.t24 & 0xFFFFFFu;
    return (((r + h.h24) & h.t24) >> kHeadBack) & tc;
}

// Index of the last list in [ha, he) whose byte offset is pos (a head bit was
// set from one of them); ha - 1 if none.
__device__ __forceinline__ long long last_list_at(const HeadSrc &p, uint64_t ha, uint64_t he, long long pos)
{
    uint64_t lo = ha, hi = he;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (static_cast<long long>(p.bo[mid]) <= pos)
            lo = mid + 1;
        else
            hi = mid;
    }
    return static_cast<long long>(lo) - 1;
}

// x_0 of the list whose first integer ends at slice bit o (a head_terms bit):
// that integer starts after the previous terminator; the head bit in between
// names the list.  srel: stream offset of the slice's first byte.
__device__ __forceinline__ uint32_t head_prev(const HeadSrc &p, const HeadTab &T, const HeadWin &h, int o, int tid,
                                              long long srel, uint64_t ha, uint64_t he)
{
    const int P = o + kHeadBack;
    const uint32_t below = h.t24 & ((1u << P) - 1u);
    const int q = below ? 31 - __clz(below) : -1;          // previous terminator
    const uint32_t above_q = q >= 0 ? ~((2u << q) - 1u) : ~0u;
    const uint32_t hb = h.h24 & ((2u << P) - 1u) & above_q;   // heads in (q, P]
    if (!hb) return 0u;
    const int k = 31 - __clz(hb);
    if (he - ha <= static_cast<uint64_t>(kMaxHeadList)) {
        const int qs = kHalo + tid * kBPT - kHeadBack + k;   // staging index of the head
        const int i = tab_last_le(T, static_cast<int>(he - ha), qs);
        return (i >= 0 && T.pos[i] == qs) ? T.prv[i] : 0u;
    }
    const long long j = last_list_at(p, ha, he, srel - kHeadBack + k);
    if (j < static_cast<long long>(ha) || p.prevs == nullptr) return 0u;
    return p.prevs[j];
}

// Per-terminator assembly as assemble_all, also passing each terminator's
// slice bit to emit(o, value).
template <typename F>
__device__ __forceinline__ void assemble_all_o(const uint32_t *sw, int tid, uint32_t tl, uint32_t t20, uint32_t tc,
                                               F emit)
{
    uint32_t m = tl;
    int prevo = 27 - __clz(t20 & 0xFu);
    while (m) {
        const int o = __ffs(m) - 1;
        m &= m - 1u;
        const int L = min(o - prevo, 5);
        prevo = o;
        if ((tc >> o) & 1u) {
            const int q = kHalo + tid * kBPT + o;
            const uint32_t A = sw[(q >> 2) - 1];
            const uint32_t B = sw[q >> 2];
            const uint32_t lo4 = __funnelshift_r(A, B, 8 * q);
            const uint32_t x = (B >> (8 * (q & 3))) & 0xFFu;
            emit(o, assemble(lo4, x, L));
        }
    }
}

// Segmented sum of a slice that holds list heads (ht != 0): the sum since the
// last head, starting from that list's x_0.
__device__ __forceinline__ uint32_t slice_seg_sum(const HeadSrc &p, const HeadTab &T, const uint32_t *sw, int tid,
                                                  uint32_t tl, uint32_t t20, uint32_t tc, const HeadWin &h,
                                                  uint32_t ht, long long srel, uint64_t ha, uint64_t he)
{
    uint32_t s = 0;
    assemble_all_o(sw, tid, tl, t20, tc, [&](int o, uint32_t v) {
        if ((ht >> o) & 1u)
            s = head_prev(p, T, h, o, tid, srel, ha, he) + v;
        else
            s += v;
    });
    return s;
}

}  // namespace vbk
