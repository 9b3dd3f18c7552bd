// Host-side VByte encoder for uint64 (input generation for vbyte_decode64).
//
// Format (Sec. 1 of arXiv 1503.07387, which notes that VByte covers 64-bit
// integers too): seven data bits per byte, least significant group first,
// the high bit set on every byte of an integer but the last.  The length is
// taken from the position of the value's highest set bit, ceil(bits / 7)
// with at least one byte, and the bytes are written for that length.
#include "vbyte64.h"

namespace {

inline size_t code_length(uint64_t v)
{
    const int bits = v ? 64 - __builtin_clzll(v) : 1;
    return static_cast<size_t>((bits + 6) / 7);
}

inline size_t put_value(uint64_t v, uint8_t *o)
{
    const size_t len = code_length(v);
    for (size_t k = 0; k + 1 < len; ++k) o[k] = static_cast<uint8_t>(0x80u | ((v >> (7 * k)) & 0x7Fu));
    o[len - 1] = static_cast<uint8_t>(v >> (7 * (len - 1)));
    return len;
}

}  // namespace

extern "C" {

size_t vbyte_max_encoded_size64(size_t n) { return 10 * n; }

size_t vbyte_encode64(const uint64_t *h_in, size_t n, uint8_t *h_out)
{
    if (n == 0 || !h_in || !h_out) return 0;
    uint8_t *o = h_out;
    for (size_t i = 0; i < n; ++i) o += put_value(h_in[i], o);
    return static_cast<size_t>(o - h_out);
}

size_t vbyte_encode_delta64(const uint64_t *h_in, size_t n, uint64_t prev, uint8_t *h_out)
{
    if (n == 0 || !h_in || !h_out) return 0;
    uint8_t *o = h_out;
    for (size_t i = 0; i < n; ++i) {
        o += put_value(h_in[i] - prev, o);   // modulo 2^64
        prev = h_in[i];
    }
    return static_cast<size_t>(o - h_out);
}

}  // extern "C"
