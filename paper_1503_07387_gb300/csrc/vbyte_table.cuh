// The table-driven decoding step of Masked VByte (Sec. 4 of arXiv 1503.07387),
// restated for the GPU: a 12-bit mask of the high bits of the next 12 bytes
// picks, from a 2^12-entry table, how many bytes to consume and one of 170
// cases; the case fixes the lengths of the integers the step decodes.
//
//   * mask 0: twelve one-byte integers as they are (no table lookup needed);
//   * cases 0..63: the next six integers each take one or two bytes
//     (2^6 length patterns);
//   * cases 64..144: else the next four take at most three bytes each (3^4);
//   * cases 145..169: else the next two take at most five bytes each (5^2);
//   * anything else (an integer of more than five bytes) is malformed: no
//     case, nothing consumed.
//
// The same functions build the table on the host (tests and the library's
// pins) and in each CTA's shared memory on the device, so both use one
// definition.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define VBK_HD __host__ __device__ __forceinline__
#else
#define VBK_HD inline
#endif

namespace vbk {
namespace tab {

constexpr int kCases = 170;          // 64 + 81 + 25
constexpr uint32_t kTwelve = 255;    // the case id of mask 0 (twelve one-byte integers)

// A case: how many integers it decodes, their lengths, the bytes they take.
//   bits 0..2: k (6, 4 or 2; 0 for none), bits 3 + 3t .. 5 + 3t: the t-th
//   length (t < 6), bits 24..27: bytes consumed.
VBK_HD uint32_t case_k(uint32_t d) { return d & 7u; }
VBK_HD uint32_t case_len(uint32_t d, int t) { return (d >> (3 + 3 * t)) & 7u; }
VBK_HD uint32_t case_consumed(uint32_t d) { return (d >> 24) & 15u; }

// The descriptor of case `id` (0 .. 169).
VBK_HD uint32_t case_desc(uint32_t id)
{
    uint32_t k, len[6] = {0, 0, 0, 0, 0, 0};
    if (id < 64) {
        k = 6;
        for (int t = 0; t < 6; ++t) len[t] = 1 + ((id >> t) & 1u);
    } else if (id < 145) {
        k = 4;
        uint32_t r = id - 64;
        for (int t = 0; t < 4; ++t) {
            len[t] = 1 + r % 3;
            r /= 3;
        }
    } else {
        k = 2;
        len[0] = 1 + (id - 145) % 5;
        len[1] = 1 + (id - 145) / 5;
    }
    uint32_t d = k, used = 0;
    for (int t = 0; t < 6; ++t) {
        d |= len[t] << (3 + 3 * t);
        used += len[t];
    }
    return d | (used << 24);
}

// Table entry of a 12-bit mask (bit b set: byte b has its high bit set):
// bytes consumed (bits 0..3, 0 if malformed) and the case id (bits 4..11).
VBK_HD uint32_t table_entry(uint32_t mask)
{
    mask &= 0xFFFu;
    if (mask == 0) return 12u | (kTwelve << 4);
    // the lengths of the integers that end within the 12 bytes
    uint32_t len[12];
    int nint = 0;
    uint32_t start = 0;
    for (uint32_t b = 0; b < 12; ++b) {
        if (!((mask >> b) & 1u)) {
            len[nint++] = b + 1 - start;
            start = b + 1;
        }
    }
    bool ok = nint >= 6;
    for (int t = 0; ok && t < 6; ++t) ok = len[t] <= 2;
    if (ok) {
        uint32_t id = 0, used = 0;
        for (int t = 0; t < 6; ++t) {
            id |= (len[t] - 1) << t;
            used += len[t];
        }
        return used | (id << 4);
    }
    ok = nint >= 4;
    for (int t = 0; ok && t < 4; ++t) ok = len[t] <= 3;
    if (ok) {
        uint32_t id = 0, used = 0, w = 1;
        for (int t = 0; t < 4; ++t) {
            id += (len[t] - 1) * w;
            w *= 3;
            used += len[t];
        }
        return used | ((64u + id) << 4);
    }
    ok = nint >= 2 && len[0] <= 5 && len[1] <= 5;
    if (ok) return (len[0] + len[1]) | ((145u + (len[0] - 1) + 5 * (len[1] - 1)) << 4);
    return 0u;
}

}  // namespace tab
}  // namespace vbk
