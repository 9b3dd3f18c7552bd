// Host-side VByte encoder of libvbyte (input generation for the GPU decoder).
//
// Format (Sec. 1, Table 1 of arXiv 1503.07387): seven data bits per byte,
// least significant group first, high bit set on every byte of an integer but
// the last.  The code length is chosen from the value's range
// ([0,2^7) -> 1 byte, [2^7,2^14) -> 2, ... [2^28,2^32) -> 5) and the bytes are
// written straight-line for that length.
#include "vbyte.h"

namespace {

inline size_t put_value(uint32_t v, uint8_t *o)
{
    if (v < (1u << 7)) {
        o[0] = static_cast<uint8_t>(v);
        return 1;
    }
    if (v < (1u << 14)) {
        o[0] = static_cast<uint8_t>(0x80u | (v & 0x7Fu));
        o[1] = static_cast<uint8_t>(v >> 7);
        return 2;
    }
    if (v < (1u << 21)) {
        o[0] = static_cast<uint8_t>(0x80u | (v & 0x7Fu));
        o[1] = static_cast<uint8_t>(0x80u | ((v >> 7) & 0x7Fu));
        o[2] = static_cast<uint8_t>(v >> 14);
        return 3;
    }
    if (v < (1u << 28)) {
        o[0] = static_cast<uint8_t>(0x80u | (v & 0x7Fu));
        o[1] = static_cast<uint8_t>(0x80u | ((v >> 7) & 0x7Fu));
        o[2] = static_cast<uint8_t>(0x80u | ((v >> 14) & 0x7Fu));
        o[3] = static_cast<uint8_t>(v >> 21);
        return 4;
    }
    o[0] = static_cast<uint8_t>(0x80u | (v & 0x7Fu));
    o[1] = static_cast<uint8_t>(0x80u | ((v >> 7) & 0x7Fu));
    o[2] = static_cast<uint8_t>(0x80u | ((v >> 14) & 0x7Fu));
    o[3] = static_cast<uint8_t>(0x80u | ((v >> 21) & 0x7Fu));
    o[4] = static_cast<uint8_t>(v >> 28);
    return 5;
}

size_t encode_plain(const uint32_t *in, size_t n, uint8_t *out)
{
    uint8_t *o = out;
    for (size_t i = 0; i < n; ++i) o += put_value(in[i], o);
    return static_cast<size_t>(o - out);
}

// Gaps x_i - x_{i-1} from x_{-1} = prev; with minus_one every gap after the
// first is one less (the variant for lists without repeated values).
size_t encode_gaps(const uint32_t *in, size_t n, uint32_t prev, uint8_t *out, bool minus_one = false)
{
    uint8_t *o = out;
    for (size_t i = 0; i < n; ++i) {
        const uint32_t x = in[i];
        o += put_value(x - prev - ((minus_one && i > 0) ? 1u : 0u), o);  // modulo 2^32
        prev = x;
    }
    return static_cast<size_t>(o - out);
}

// Blocked differences x_i - x_{i-4}, with x_{-4..-1} = prev4[0..3].
size_t encode_blocks(const uint32_t *in, size_t n, const uint32_t *prev4, uint8_t *out)
{
    uint8_t *o = out;
    for (size_t i = 0; i < n; ++i) {
        const uint32_t before = i >= 4 ? in[i - 4] : (prev4 ? prev4[i] : 0u);
        o += put_value(in[i] - before, o);   // modulo 2^32
    }
    return static_cast<size_t>(o - out);
}

}  // namespace

extern "C" {

size_t vbyte_max_encoded_size(size_t n) { return 5 * n; }

size_t vbyte_encode(const uint32_t *h_in, size_t n, uint8_t *h_out)
{
    if (n == 0) return 0;
    if (!h_in || !h_out) return 0;
    return encode_plain(h_in, n, h_out);
}

size_t vbyte_encode_delta(const uint32_t *h_in, size_t n, uint32_t prev,
                          uint8_t *h_out)
{
    if (n == 0) return 0;
    if (!h_in || !h_out) return 0;
    return encode_gaps(h_in, n, prev, h_out);
}

size_t vbyte_encode_delta_m1(const uint32_t *h_in, size_t n, uint32_t prev, uint8_t *h_out)
{
    if (n == 0) return 0;
    if (!h_in || !h_out) return 0;
    return encode_gaps(h_in, n, prev, h_out, true);
}

size_t vbyte_encode_delta4(const uint32_t *h_in, size_t n, const uint32_t *h_prev4, uint8_t *h_out)
{
    if (n == 0) return 0;
    if (!h_in || !h_out) return 0;
    return encode_blocks(h_in, n, h_prev4, h_out);
}

size_t vbyte_encode_batched(const uint32_t *h_in, const uint64_t *h_val_off,
                            size_t num_lists, int delta, const uint32_t *h_prev,
                            uint8_t *h_out, uint64_t *h_byte_off)
{
    if (!h_val_off || !h_byte_off) return 0;
    size_t w = 0;
    h_byte_off[0] = 0;
    for (size_t j = 0; j < num_lists; ++j) {
        const size_t v0 = static_cast<size_t>(h_val_off[j]);
        const size_t nv = static_cast<size_t>(h_val_off[j + 1] - h_val_off[j]);
        if (delta)
            w += encode_gaps(h_in + v0, nv, h_prev ? h_prev[j] : 0u, h_out + w);
        else
            w += encode_plain(h_in + v0, nv, h_out + w);
        h_byte_off[j + 1] = w;
    }
    return w;
}

}  // extern "C"
