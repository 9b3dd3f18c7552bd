// Host side of the table-driven decoding step (vbyte_table.cuh): the table
// and its case descriptors for inspection, and a host decoder that follows
// the step from the start of a byte stream, for the pins that tie the table
// to Algorithm 1.
#include <stddef.h>
#include <stdint.h>

#include "vbyte.h"
#include "vbyte_table.cuh"

extern "C" {

int vbyte_table(uint16_t *h_entries, uint32_t *h_cases)
{
    if (!h_entries || !h_cases) return VBYTE_EINVAL;
    for (uint32_t m = 0; m < 4096; ++m) h_entries[m] = static_cast<uint16_t>(vbk::tab::table_entry(m));
    for (uint32_t i = 0; i < static_cast<uint32_t>(vbk::tab::kCases); ++i) h_cases[i] = vbk::tab::case_desc(i);
    return VBYTE_OK;
}

size_t vbyte_table_decode(const uint8_t *h_in, size_t nbytes, uint32_t *h_out, size_t cap)
{
    if (nbytes && !h_in) return 0;
    size_t p = 0, w = 0;
    auto emit = [&](uint32_t v) {
        if (w < cap) h_out[w] = v;
        ++w;
    };
    // whole 12-byte windows: one table step each
    while (p + 12 <= nbytes) {
        uint32_t mask = 0;
        for (uint32_t b = 0; b < 12; ++b) mask |= static_cast<uint32_t>(h_in[p + b] >> 7) << b;
        const uint32_t e = vbk::tab::table_entry(mask);
        const uint32_t consumed = e & 15u, id = e >> 4;
        if (!consumed) break;   // an integer of more than five bytes: the steps below
        if (id == vbk::tab::kTwelve) {
            for (uint32_t b = 0; b < 12; ++b) emit(h_in[p + b]);
        } else {
            const uint32_t d = vbk::tab::case_desc(id);
            uint32_t o = 0;
            for (uint32_t t = 0; t < vbk::tab::case_k(d); ++t) {
                const uint32_t L = vbk::tab::case_len(d, static_cast<int>(t));
                uint32_t v = 0;
                for (uint32_t i = 0; i < L; ++i) v |= static_cast<uint32_t>(h_in[p + o + i] & 0x7Fu) << (7 * i);
                emit(v);
                o += L;
            }
        }
        p += consumed;
    }
    // the rest one integer at a time: up to five bytes, the fifth taken whole
    while (p < nbytes) {
        uint32_t v = 0;
        int i = 0;
        for (;; ++i) {
            if (p + i >= nbytes) return w;   // ends inside an integer
            const uint32_t b = h_in[p + i];
            if (i == 4) {
                v += b << 28;
                break;
            }
            v |= (b & 0x7Fu) << (7 * i);
            if (b < 128) break;
        }
        emit(v);
        p += i + 1;
    }
    return w;
}

}  // extern "C"
