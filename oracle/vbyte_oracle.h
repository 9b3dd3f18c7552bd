/*
 * Plain scalar CPU oracle for VByte coding of uint32 (arXiv 1503.07387).
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the library's product path.
 */
#ifndef VBYTE_ORACLE_H
#define VBYTE_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Data-error bits of the validation contract.  The numeric values are part
 * of the documented library contract, so the tests can compare status words
 * from both sides bit for bit. */
#define ORACLE_ERR_MALFORMED_LONG 1u
#define ORACLE_ERR_TRUNCATED 2u
#define ORACLE_ERR_COUNT_MISMATCH 4u

size_t oracle_encode_one(uint32_t v, uint8_t *out);
size_t oracle_encode(const uint32_t *in, size_t n, uint8_t *out);
size_t oracle_encode_delta(const uint32_t *in, size_t n, uint32_t prev,
                           uint8_t *out);

size_t oracle_encode_delta_m1(const uint32_t *in, size_t n, uint32_t prev,
                              uint8_t *out);

size_t oracle_decode(const uint8_t *in, size_t nbytes, uint32_t *out,
                     size_t cap);
size_t oracle_decode_delta_m1(const uint8_t *in, size_t nbytes, uint32_t *out,
                              size_t cap, uint32_t prev);
size_t oracle_decode_delta(const uint8_t *in, size_t nbytes, uint32_t *out,
                           size_t cap, uint32_t prev);
uint32_t oracle_validate(const uint8_t *in, size_t nbytes, size_t n);

size_t oracle_encode_delta4(const uint32_t *in, size_t n, const uint32_t *prev4, uint8_t *out);
size_t oracle_decode_delta4(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                            const uint32_t *prev4);

size_t oracle_encode64_one(uint64_t v, uint8_t *out);
size_t oracle_encode64(const uint64_t *in, size_t n, uint8_t *out);
size_t oracle_encode_delta64(const uint64_t *in, size_t n, uint64_t prev, uint8_t *out);
size_t oracle_decode64(const uint8_t *in, size_t nbytes, uint64_t *out, size_t cap);
size_t oracle_decode_delta64(const uint8_t *in, size_t nbytes, uint64_t *out, size_t cap,
                             uint64_t prev);
uint32_t oracle_validate64(const uint8_t *in, size_t nbytes, size_t n);

uint32_t oracle_decode_batched(const uint8_t *in, const uint64_t *byte_off,
                               const uint64_t *val_off, size_t num_lists,
                               int delta, const uint32_t *prev, uint32_t *out);
size_t oracle_encode_batched(const uint32_t *in, const uint64_t *val_off,
                             size_t num_lists, int delta, const uint32_t *prev,
                             uint8_t *out, uint64_t *byte_off);
int oracle_decode_batched_mt(const uint8_t *in, const uint64_t *byte_off,
                             const uint64_t *val_off, size_t num_lists,
                             int delta, const uint32_t *prev, uint32_t *out,
                             int threads);

#ifdef __cplusplus
}
#endif

#endif
