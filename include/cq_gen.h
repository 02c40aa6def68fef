/* cq_gen.h -- device-side generator of the synthetic per-row columns of the
 * nested (lexicographically sorted) table, library libcqgen.so.
 *
 * Input infrastructure, not part of the query method: it only draws values
 * and bit-packs them, so that tables of billions of rows can be produced in
 * device memory.  Every value is a pure function of (seed, column, row)
 * through SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014):
 *
 *   h(seed, col, i) = mix((seed XOR col << 56) + (i + 1) * 0x9E3779B97F4A7C15)
 *   mix(z): z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9;
 *           z = (z ^ z >> 27) * 0x94D049BB133111EB;  return z ^ z >> 31
 *
 * (all mod 2^64), the same definition the host-side generator evaluates for
 * any sampled row.  Packed output is LSB-first in little-endian uint32 words
 * (field r occupies bits r*w .. r*w+w-1 of the stream), the layout
 * cq_column_create_bitpacked / cq_column_create_dict take; words past the
 * last field are written as zero.
 *
 * All pointers are device pointers the caller owns; `cuda_stream` may be
 * NULL (legacy default stream).  The calls are asynchronous on the stream and
 * return 0, or -1 for a bad argument, or -2 when the launch fails. */
#ifndef CQ_GEN_H
#define CQ_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* words[0 .. n_words) <- the packed fields (h(seed, col, r) mod 2^bit_width)
 * for r < n_rows, 1 <= bit_width <= 32, n_words >= ceil(n_rows*bit_width/32). */
int cqgen_hash_fields(uint32_t* words, uint64_t n_words, uint64_t n_rows, uint32_t bit_width,
                      uint64_t seed, uint32_t col, void* cuda_stream);

/* words[0 .. n_words) <- 4-bit codes of the nested table's c4: row r in the
 * c3 run [s, e) (run j, exclusive ends c3_ends[0 .. n_runs), the last equal
 * to n_rows) gets #{k in 0..14 : h(seed, 4, 15 j + k) mod (e - s) <= r - s},
 * a code in 0..15 that never decreases along a run. */
int cqgen_nested_codes4(uint32_t* words, uint64_t n_words, const int64_t* c3_ends, uint64_t n_runs,
                        uint64_t n_rows, uint64_t seed, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif
