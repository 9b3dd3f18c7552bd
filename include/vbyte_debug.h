/*
 * libvbyte -- fault injection for tests of the bounded waits.
 *
 * The paper has no counterpart: its decoder is one sequential loop.  The GPU
 * decoders pass tile counts and running sums between CTAs through published
 * words, and every wait for such a word is bounded by the global timer; when
 * a bound runs out the launch records VBYTE_ERR_TIMEOUT in the status word,
 * writes nothing outside [0, n) and returns.  This call makes that happen on
 * purpose, with no GPU fault: a chosen tile's count is simply never
 * published, so the wait for it runs out.  Not for production use.
 */
#ifndef VBYTE_DEBUG_H
#define VBYTE_DEBUG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Process-wide, for the single-stream and batched decode launches queued
 * after the call (vbyte_decode*, vbyte_decode_noalloc, the batched calls and
 * plans created afterwards; a plan keeps the setting it was captured with):
 *   skip_tile      index of the 4 KiB input tile (tile 0 starts at the input
 *                  rounded down to 16 bytes) whose count descriptor is never
 *                  published; < 0 for none (the default);
 *   wait_limit_ns  bound of every wait between CTAs, in nanoseconds; 0 for
 *                  the default of two seconds.
 * Returns VBYTE_OK, or VBYTE_EINVAL for a limit above the default.  The
 * output of a launch that timed out is unspecified within [0, n); read and
 * clear the status word (vbyte_get_status) before the next call on that
 * stream, since a recorded timeout makes every later wait give up at once. */
int vbyte_debug_inject(long long skip_tile, uint64_t wait_limit_ns);

/* Which single-stream kernel vbyte_decode, vbyte_decode_delta and
 * vbyte_decode_delta_m1 use from now on (process-wide): 1 = single pass (each
 * tile resolves its output position and running sum by looking back over
 * earlier tiles' published counts and sums), 2 = count then decode in one
 * launch (a count pass runs a fixed number of tiles ahead of the decode
 * pass), 3 = split (separate count, scan and decode launches; no CTA waits
 * on another), 4 = split with the decode launch following the table-driven
 * steps of Sec. 4 (vbyte_table) in place of per-terminator assembly (the
 * gaps-minus-one variant keeps assembly), 0 = the library's choice (the
 * default).  All give identical
 * results; this exists so that tests can check each and benchmarks can
 * compare them.  Returns VBYTE_OK, or VBYTE_EINVAL for another value. */
int vbyte_debug_force_passes(int passes);

/* The choice vbyte_plan_create makes from now on (process-wide), in place of
 * its defaults or its timing: kernel 0 (the segmented stream kernel), 1
 * (list items of chunk_bytes, a multiple of 16 of at least 4096, with
 * threads_per_block 128 or 256) or 2 (the same, decoding by the table-driven
 * steps of Sec. 4); kernel -1 restores the usual choice.
 * Exists so that tests can check every candidate.  Returns VBYTE_OK, or
 * VBYTE_EINVAL for another value. */
int vbyte_debug_force_plan(int kernel, uint64_t chunk_bytes, int threads_per_block);

/* The kernel (1 to 4, as above) that a single-stream call on an
 * nbytes-byte input holding n values would use now. */
int vbyte_debug_passes_for(size_t nbytes, size_t n, int delta);

#ifdef __cplusplus
}
#endif

#endif /* VBYTE_DEBUG_H */
