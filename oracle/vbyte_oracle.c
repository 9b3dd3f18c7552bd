/*
 * Plain scalar CPU oracle for VByte coding of uint32 (Plaisance, Kurz, Lemire,
 * "Vectorized VByte Decoding", arXiv 1503.07387).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What it follows:
 *   - format: seven data bits per byte, least significant group first, the
 *     high bit set on every byte of an integer except the last (Sec. 1 and
 *     Table 1);
 *   - decoding: Algorithm 1 (Sec. 2), executed one byte at a time with uint32
 *     arithmetic, the fifth byte of an integer taken without testing its high
 *     bit;
 *   - differential coding: gaps x_i - x_{i-1} with x_0 = prev (0 by default),
 *     undone by keeping the last decoded value and adding it to each gap
 *     (Sec. 1 "Differential coding" and Sec. 2); and the variant for lists
 *     without repeated values that Sec. 1 also names, which stores the first
 *     gap as is and every later one minus one (x_1 - x_0, x_2 - x_1 - 1, ...),
 *     undone by adding one more for every value after the first;
 *     The blocked variant Sec. 1 names as well (x_1..x_4, then x_i - x_{i-4})
 *     is undone by adding, to each decoded difference, the value four
 *     places before it;
 *   - 64-bit integers, which Sec. 1 says the format also covers: the same
 *     rules read for uint64 (up to ten bytes, Algorithm 1 with ten steps,
 *     the tenth byte taken without testing its high bit);
 *   - validation: a separate pass that states the data-error contract
 *     (a run of five or more bytes with the high bit set; a final byte with
 *     the high bit set; a terminator count that differs from the expected
 *     count).  The paper defines no error handling; this contract is the
 *     reading adopted for malformed input.
 *
 * Every function is single-threaded except the *_mt batched decoders, which
 * split whole lists across POSIX threads for the CPU baseline timing.
 */
#include "vbyte_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- encode -- */

/* Sec. 1: write the integer seven bits at a time from the least significant
 * end; every byte but the last carries the continuation flag 0x80. */
size_t oracle_encode_one(uint32_t v, uint8_t *out)
{
    size_t k = 0;
    while (v >= 128u) {
        out[k++] = (uint8_t)((v & 127u) | 128u);
        v >>= 7;
    }
    out[k++] = (uint8_t)v;
    return k;
}

size_t oracle_encode(const uint32_t *in, size_t n, uint8_t *out)
{
    size_t w = 0;
    for (size_t i = 0; i < n; ++i) w += oracle_encode_one(in[i], out + w);
    return w;
}

/* Sec. 1 "Differential coding": store x_1 - x_0, x_2 - x_1, ... with x_0 =
 * prev; differences are taken modulo 2^32. */
size_t oracle_encode_delta(const uint32_t *in, size_t n, uint32_t prev,
                           uint8_t *out)
{
    size_t w = 0;
    for (size_t i = 0; i < n; ++i) {
        uint32_t gap = in[i] - prev;
        prev = in[i];
        w += oracle_encode_one(gap, out + w);
    }
    return w;
}

/* Sec. 1 "Differential coding", the variant for lists without repeated
 * values: store x_1 - x_0, then x_i - x_{i-1} - 1; x_0 = prev. */
size_t oracle_encode_delta_m1(const uint32_t *in, size_t n, uint32_t prev,
                              uint8_t *out)
{
    size_t w = 0;
    for (size_t i = 0; i < n; ++i) {
        uint32_t gap = in[i] - prev - (i > 0 ? 1u : 0u);
        prev = in[i];
        w += oracle_encode_one(gap, out + w);
    }
    return w;
}

/* ---------------------------------------------------------------- decode -- */

/* Algorithm 1, step by step.  Returns the number of integers Algorithm 1
 * appends; values beyond `cap` are counted but not stored.  If the input ends
 * inside an integer (readByte has nothing left to return), the partial
 * integer is dropped.  With delta != 0 the running value p starts at prev and
 * each decoded gap is added to it (Sec. 2, last paragraph before Alg. 1);
 * with delta == 2 (gaps minus one) every value after the first adds one
 * more. */
static size_t algorithm1(const uint8_t *in, size_t nbytes, uint32_t *y,
                         size_t cap, int delta, uint32_t prev)
{
    size_t pos = 0, count = 0;
    uint32_t p = prev;
#define READ_BYTE(dst)                  \
    do {                                \
        if (pos >= nbytes) goto done;   \
        (dst) = in[pos++];              \
    } while (0)
#define APPEND(val)                                  \
    do {                                             \
        uint32_t v_ = (uint32_t)(val);               \
        if (delta) {                                 \
            p = p + v_ + (delta == 2 && count > 0);  \
            v_ = p;                                  \
        }                                            \
        if (count < cap) y[count] = v_;              \
        ++count;                                     \
    } while (0)
    while (pos < nbytes) {
        uint32_t b, c;
        READ_BYTE(b);
        if (b < 128u) { APPEND(b); continue; }
        c = b % 128u;
        READ_BYTE(b);
        if (b < 128u) { APPEND(c + b * 128u); continue; }
        c = c + (b % 128u) * 128u;
        READ_BYTE(b);
        if (b < 128u) { APPEND(c + b * 16384u); continue; }
        c = c + (b % 128u) * 16384u;
        READ_BYTE(b);
        if (b < 128u) { APPEND(c + b * 2097152u); continue; }
        c = c + (b % 128u) * 2097152u;
        READ_BYTE(b);
        APPEND(c + b * 268435456u); /* b * 2^28, taken modulo 2^32 */
    }
done:
#undef READ_BYTE
#undef APPEND
    return count;
}

size_t oracle_decode(const uint8_t *in, size_t nbytes, uint32_t *out,
                     size_t cap)
{
    return algorithm1(in, nbytes, out, cap, 0, 0u);
}

size_t oracle_decode_delta(const uint8_t *in, size_t nbytes, uint32_t *out,
                           size_t cap, uint32_t prev)
{
    return algorithm1(in, nbytes, out, cap, 1, prev);
}

size_t oracle_decode_delta_m1(const uint8_t *in, size_t nbytes, uint32_t *out,
                              size_t cap, uint32_t prev)
{
    return algorithm1(in, nbytes, out, cap, 2, prev);
}

/* -------------------------------------------------------------- validate -- */

/* The data-error contract, stated on the bytes themselves:
 *   MALFORMED_LONG  some five consecutive bytes all have the high bit set;
 *   TRUNCATED       the last byte has the high bit set;
 *   COUNT_MISMATCH  the number of bytes with the high bit clear differs from
 *                   the expected count n. */
uint32_t oracle_validate(const uint8_t *in, size_t nbytes, size_t n)
{
    uint32_t st = 0;
    size_t run = 0, terminators = 0;
    for (size_t i = 0; i < nbytes; ++i) {
        if (in[i] & 128u) {
            if (++run >= 5) st |= ORACLE_ERR_MALFORMED_LONG;
        } else {
            run = 0;
            ++terminators;
        }
    }
    if (nbytes > 0 && (in[nbytes - 1] & 128u)) st |= ORACLE_ERR_TRUNCATED;
    if (terminators != n) st |= ORACLE_ERR_COUNT_MISMATCH;
    return st;
}

/* ------------------------------------------------ blocked differences -- */

/* Sec. 1 "Differential coding" also names differences taken across blocks
 * of four for speed: x_1, x_2, x_3, x_4, x_5 - x_1, x_6 - x_2, ...  Written
 * with a seed: value i (from 0) is stored as x_i - x_{i-4} modulo 2^32,
 * where x_{-4}, x_{-3}, x_{-2}, x_{-1} are prev4[0..3] (all zero when prev4
 * is NULL, which gives the paper's list). */
size_t oracle_encode_delta4(const uint32_t *in, size_t n, const uint32_t *prev4, uint8_t *out)
{
    size_t w = 0;
    for (size_t i = 0; i < n; ++i) {
        const uint32_t before = i >= 4 ? in[i - 4] : (prev4 ? prev4[i] : 0u);
        w += oracle_encode_one(in[i] - before, out + w);
    }
    return w;
}

/* Algorithm 1 gives the stored differences g_i; then x_i = g_i + x_{i-4}
 * modulo 2^32, in order, with the same seed.  Returns Algorithm 1's count;
 * values beyond cap are not stored (and not needed: x_i depends only on
 * earlier values). */
size_t oracle_decode_delta4(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                            const uint32_t *prev4)
{
    const size_t count = algorithm1(in, nbytes, out, cap, 0, 0u);
    const size_t m = count < cap ? count : cap;
    for (size_t i = 0; i < m; ++i) {
        const uint32_t before = i >= 4 ? out[i - 4] : (prev4 ? prev4[i] : 0u);
        out[i] = out[i] + before;
    }
    return count;
}

/* ---------------------------------------------------------------- 64-bit -- */

/* Sec. 1 notes that the format applies to 64-bit integers as well.  The same
 * rules, read for uint64: seven bits per byte from the least significant
 * end, so a value takes 1 + [v >= 2^7] + ... + [v >= 2^63] bytes (at most
 * ten); the decoder follows Algorithm 1 with ten steps instead of five, the
 * tenth byte taken without testing its high bit and multiplied by 2^63
 * modulo 2^64; a run of ten or more bytes with the high bit set is
 * malformed. */
size_t oracle_encode64_one(uint64_t v, uint8_t *out)
{
    size_t k = 0;
    while (v >= 128u) {
        out[k++] = (uint8_t)((v & 127u) | 128u);
        v >>= 7;
    }
    out[k++] = (uint8_t)v;
    return k;
}

size_t oracle_encode64(const uint64_t *in, size_t n, uint8_t *out)
{
    size_t w = 0;
    for (size_t i = 0; i < n; ++i) w += oracle_encode64_one(in[i], out + w);
    return w;
}

size_t oracle_encode_delta64(const uint64_t *in, size_t n, uint64_t prev, uint8_t *out)
{
    size_t w = 0;
    for (size_t i = 0; i < n; ++i) {
        w += oracle_encode64_one(in[i] - prev, out + w);
        prev = in[i];
    }
    return w;
}

/* Algorithm 1 for uint64: read a byte; while its high bit is set and fewer
 * than ten bytes of this integer were read, add its seven bits at the next
 * position and read another; the last byte read goes in whole (the tenth:
 * b * 2^63 modulo 2^64).  delta != 0: running sum from prev.  A partial
 * integer at the end is dropped. */
static size_t algorithm1_64(const uint8_t *in, size_t nbytes, uint64_t *y, size_t cap, int delta,
                            uint64_t prev)
{
    size_t pos = 0, count = 0;
    uint64_t p = prev;
    while (pos < nbytes) {
        uint64_t c = 0;
        int k = 0;
        int complete = 0;
        while (pos < nbytes) {
            const uint64_t b = in[pos++];
            if (b < 128u || k == 9) {
                c += b << (7 * k);
                complete = 1;
                break;
            }
            c += (b & 127u) << (7 * k);
            ++k;
        }
        if (!complete) break;
        if (delta) {
            p += c;
            c = p;
        }
        if (count < cap) y[count] = c;
        ++count;
    }
    return count;
}

size_t oracle_decode64(const uint8_t *in, size_t nbytes, uint64_t *out, size_t cap)
{
    return algorithm1_64(in, nbytes, out, cap, 0, 0u);
}

size_t oracle_decode_delta64(const uint8_t *in, size_t nbytes, uint64_t *out, size_t cap, uint64_t prev)
{
    return algorithm1_64(in, nbytes, out, cap, 1, prev);
}

uint32_t oracle_validate64(const uint8_t *in, size_t nbytes, size_t n)
{
    uint32_t st = 0;
    size_t run = 0, terminators = 0;
    for (size_t i = 0; i < nbytes; ++i) {
        if (in[i] & 128u) {
            if (++run >= 10) st |= ORACLE_ERR_MALFORMED_LONG;
        } else {
            run = 0;
            ++terminators;
        }
    }
    if (nbytes > 0 && (in[nbytes - 1] & 128u)) st |= ORACLE_ERR_TRUNCATED;
    if (terminators != n) st |= ORACLE_ERR_COUNT_MISMATCH;
    return st;
}

/* --------------------------------------------------------------- batched -- */

/* A batch is a list of independent streams laid end to end: list j owns bytes
 * [byte_off[j], byte_off[j+1]) and values [val_off[j], val_off[j+1]).  Each list
 * is decoded on its own with Algorithm 1; in delta mode the running value
 * restarts at prev[j] (0 when prev is NULL) at the head of every list.  The
 * status is the OR of the per-list validation against the list's own count. */
uint32_t oracle_decode_batched(const uint8_t *in, const uint64_t *byte_off,
                               const uint64_t *val_off, size_t num_lists,
                               int delta, const uint32_t *prev, uint32_t *out)
{
    uint32_t st = 0;
    for (size_t j = 0; j < num_lists; ++j) {
        const uint8_t *b = in + byte_off[j];
        size_t nb = (size_t)(byte_off[j + 1] - byte_off[j]);
        size_t nv = (size_t)(val_off[j + 1] - val_off[j]);
        uint32_t p0 = prev ? prev[j] : 0u;
        algorithm1(b, nb, out + val_off[j], nv, delta, p0);
        st |= oracle_validate(b, nb, nv);
    }
    return st;
}

size_t oracle_encode_batched(const uint32_t *in, const uint64_t *val_off,
                             size_t num_lists, int delta, const uint32_t *prev,
                             uint8_t *out, uint64_t *byte_off)
{
    size_t w = 0;
    byte_off[0] = 0;
    for (size_t j = 0; j < num_lists; ++j) {
        const uint32_t *v = in + val_off[j];
        size_t nv = (size_t)(val_off[j + 1] - val_off[j]);
        if (delta)
            w += oracle_encode_delta(v, nv, prev ? prev[j] : 0u, out + w);
        else
            w += oracle_encode(v, nv, out + w);
        byte_off[j + 1] = w;
    }
    return w;
}

/* Multi-threaded batched decode for the CPU baseline: lists are dealt out in
 * contiguous ranges of roughly equal byte volume, one range per thread.  Each
 * thread runs the same single-threaded Algorithm 1 per list. */
typedef struct {
    const uint8_t *in;
    const uint64_t *byte_off, *val_off;
    size_t j0, j1;
    int delta;
    const uint32_t *prev;
    uint32_t *out;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *jb = (batch_job *)arg;
    for (size_t j = jb->j0; j < jb->j1; ++j) {
        size_t nb = (size_t)(jb->byte_off[j + 1] - jb->byte_off[j]);
        size_t nv = (size_t)(jb->val_off[j + 1] - jb->val_off[j]);
        algorithm1(jb->in + jb->byte_off[j], nb, jb->out + jb->val_off[j], nv,
                   jb->delta, jb->prev ? jb->prev[j] : 0u);
    }
    return NULL;
}

int oracle_decode_batched_mt(const uint8_t *in, const uint64_t *byte_off,
                             const uint64_t *val_off, size_t num_lists,
                             int delta, const uint32_t *prev, uint32_t *out,
                             int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    batch_job jobs[256];
    uint64_t total = byte_off[num_lists] - byte_off[0];
    size_t j = 0;
    int used = 0;
    for (int t = 0; t < threads && j < num_lists; ++t) {
        uint64_t target = byte_off[0] + total * (uint64_t)(t + 1) / threads;
        size_t j1 = j;
        while (j1 < num_lists && (byte_off[j1 + 1] <= target || j1 == j)) ++j1;
        if (t == threads - 1) j1 = num_lists;
        jobs[used] = (batch_job){in, byte_off, val_off, j, j1, delta, prev, out};
        if (pthread_create(&tid[used], NULL, batch_worker, &jobs[used]) != 0) {
            batch_worker(&jobs[used]);
            tid[used] = 0;
        }
        ++used;
        j = j1;
    }
    for (int t = 0; t < used; ++t)
        if (tid[t]) pthread_join(tid[t], NULL);
    return used;
}
