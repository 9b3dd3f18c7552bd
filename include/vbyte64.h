/*
 * libvbyte, 64-bit integers: C ABI.
 *
 * Sec. 1 of "Vectorized VByte Decoding" (Plaisance, Kurz, Lemire; arXiv
 * 1503.07387) notes that the VByte format applies to 64-bit integers as well
 * as to the 32-bit ones the paper works with.  These calls read it for
 * uint64:
 *   - format: seven data bits per byte, least significant group first, the
 *     high bit set on every byte of an integer except the last (Sec. 1,
 *     Table 1), so an integer takes 1 + [v >= 2^7] + ... + [v >= 2^63]
 *     bytes, at most ten;
 *   - decoding: Algorithm 1 (Sec. 2) with ten steps instead of five; the
 *     tenth byte of an integer is taken without testing its high bit and
 *     multiplied by 2^63 modulo 2^64;
 *   - differential coding (Sec. 1 "Differential coding"): the stream holds
 *     gaps x_i - x_{i-1} with x_0 = prev, and decoding returns the prefix
 *     sums x_i modulo 2^64.
 *
 * The conventions of vbyte.h hold: "d_" pointers are caller-owned device
 * memory, "h_" pointers caller-owned host memory; `stream` is a cudaStream_t
 * passed as void* (NULL = the legacy default stream) and the calls return
 * without synchronising; the return codes are VBYTE_OK ... ; data errors are
 * OR-ed into the same per-stream status word and read with
 * vbyte_get_status().  For uint64 streams the data-error bits mean:
 *   VBYTE_ERR_MALFORMED_LONG  a run of ten or more consecutive bytes with the
 *                             high bit set;
 *   VBYTE_ERR_TRUNCATED       the last byte has the high bit set;
 *   VBYTE_ERR_COUNT_MISMATCH  the number of bytes with the high bit clear
 *                             differs from n.
 * Output writes are clamped to [0, n); when a data error is recorded, output
 * slots the stream does not define are unspecified.
 */
#ifndef VBYTE64_H
#define VBYTE64_H

#include <stddef.h>
#include <stdint.h>

#include "vbyte.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Upper bound on the encoded size of n uint64 values: 10*n bytes (Sec. 1). */
size_t vbyte_max_encoded_size64(size_t n);

/* Encode n uint64 values (Sec. 1) into h_out, which must hold
 * vbyte_max_encoded_size64(n) bytes.  Returns the number of bytes written
 * (0 for n == 0 or a null pointer).  Host memory only; no CUDA call. */
size_t vbyte_encode64(const uint64_t *h_in, size_t n, uint8_t *h_out);

/* Encode the gaps h_in[i] - h_in[i-1] (mod 2^64), h_in[-1] = prev, as
 * vbyte_encode64 does. */
size_t vbyte_encode_delta64(const uint64_t *h_in, size_t n, uint64_t prev, uint8_t *h_out);

/* Decode the nbytes bytes at d_in into n uint64 at d_out (Algorithm 1 read
 * for uint64).  d_out must be 8-byte aligned; d_in has no alignment rule.
 * Uses the stream's workspace (16 bytes per 4 KiB of input plus a fixed
 * head), grown as vbyte.h describes.  Returns VBYTE_EINVAL for a null
 * pointer with a nonzero size or a misaligned d_out, VBYTE_ENOMEM if the
 * workspace cannot grow, VBYTE_ECUDA if a launch fails. */
int vbyte_decode64(const uint8_t *d_in, size_t nbytes, uint64_t *d_out, size_t n, void *stream);

/* As vbyte_decode64, returning the running sums from prev of the decoded
 * gaps, modulo 2^64 (Sec. 1 and Sec. 2, differential coding). */
int vbyte_decode_delta64(const uint8_t *d_in, size_t nbytes, uint64_t *d_out, size_t n, uint64_t prev,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VBYTE64_H */
