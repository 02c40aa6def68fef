/*
 * cq_oracle.h -- plain, slow CPU oracle for filter / group-by / aggregate
 * queries over lightweight-compressed columns.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library: it decompresses every
 * referenced column to flat int64 rows with its own decoders and evaluates
 * the query row by row, which is the plain definition of what the
 * compressed-domain method computes exactly (Sections 6-7 of the paper:
 * selection, grouping, aggregation; Appendix A.2 worked example).
 *
 * Column encodings (Section 3, "Basic Encodings"):
 *   RLE    run values + exclusive run ends (row r is in run i iff
 *          ends[i-1] <= r < ends[i]); ends strictly increasing, last == n_rows.
 *   INDEX  sorted unique positions + values; unlisted rows hold a default.
 *   DICT   bytewise-sorted unique strings; per-row codes bit-packed LSB-first.
 *   PACKED per-row unsigned offsets bit-packed LSB-first; value = base + offset.
 *   PLAIN  one value per row.
 * All integer inputs are passed as int64 (the test wrapper widens them).
 */
#ifndef CQ_ORACLE_H
#define CQ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ORC_RLE_INDEX: the RLE + Index composite (Section 3.2): runs
 * [run_starts[i], run_ends[i]) hold run_values[i] (starts and exclusive
 * ends, sorted, disjoint), rows positions[k] hold idx_values[k]; runs and
 * positions together cover every row exactly once. */
/* ORC_PACKED_INDEX: the Plain + Index composite (Section 3.2, outlier
 * patching): a narrow bit-packed part (the PACKED fields: words, bit_width,
 * base) holds one field per row, and the rows positions[k] (sorted, unique)
 * hold idx_values[k] instead; the packed fields at those rows are never read. */
enum { ORC_RLE = 1, ORC_DICT = 2, ORC_INDEX = 3, ORC_PACKED = 4, ORC_PLAIN = 5, ORC_RLE_INDEX = 6,
       ORC_PACKED_INDEX = 7 };
enum { ORC_LT = 0, ORC_LE, ORC_GT, ORC_GE, ORC_EQ, ORC_NE, ORC_BETWEEN, ORC_IN };
enum { ORC_SUM = 0, ORC_COUNT, ORC_MIN, ORC_MAX, ORC_AVG,
       /* Section 7: STD and VAR from COUNT, SUM and the sum of squares; the
          exact rational value rounded once to double (STD: the square root of
          that double); population (n) or sample (n - 1) denominator, 0 when
          the denominator is 0 */
       ORC_VAR_POP, ORC_VAR_SAMP, ORC_STD_POP, ORC_STD_SAMP };
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OVERFLOW = -6 };

typedef struct {
  int32_t enc;
  uint64_t n_rows;
  /* RLE */
  const int64_t* run_values;
  const int64_t* run_ends;
  uint64_t n_runs;
  /* PACKED and DICT codes */
  const uint32_t* words;
  uint64_t n_words;
  uint32_t bit_width;
  int64_t base;
  /* INDEX */
  const int64_t* idx_values;
  const int64_t* positions;
  uint64_t nnz;
  int64_t default_value;
  /* PLAIN */
  const int64_t* values;
  /* DICT strings: entry i is dict_bytes[dict_offsets[i] .. dict_offsets[i+1]) */
  const uint8_t* dict_bytes;
  const uint64_t* dict_offsets;
  uint32_t n_entries;
  /* RLE_INDEX: run starts (with run_values, run_ends, n_runs and the INDEX
     fields idx_values, positions, nnz) */
  const int64_t* run_starts;
} orc_column;

typedef struct {
  uint32_t col;
  int32_t op;
  int64_t lo, hi;                 /* integer literals; BETWEEN is inclusive */
  const int64_t* in_ints;         /* IN list on an integer column */
  uint32_t n_in;
  const uint8_t* const* strs;     /* string literals on a DICT column */
  const uint32_t* str_lens;
  uint32_t n_strs;
  uint32_t or_group;              /* 0: a conjunct of its own; g > 0: OR-ed with every other
                                     predicate of group g, the group being one conjunct */
  uint32_t negate;                /* nonzero: the predicate is replaced by its complement (NOT) */
} orc_pred;

/* A boolean filter over the predicates as a postfix program (Section 5:
 * logical AND, OR, NOT of mask columns).  PRED pushes predicate `arg`'s
 * truth (its negate flag applied); AND / OR pop `arg` >= 1 values and push
 * their conjunction / disjunction; NOT replaces the top value by its
 * complement.  The program must leave exactly one value. */
enum { ORC_NODE_PRED = 0, ORC_NODE_AND = 1, ORC_NODE_OR = 2, ORC_NODE_NOT = 3 };
typedef struct {
  int32_t kind;
  uint32_t arg;
} orc_node;

/* An aggregate's input is column `col`, or, with an expression, the
 * position-wise result `col` (expr) `col2` of two columns (Section 6:
 * arithmetic on aligned columns, e.g. c1 + c2 after alignment): computed
 * exactly per row; a row whose result leaves the int64 range makes the
 * query fail with ORC_ERR_OVERFLOW.  Expressions take SUM, MIN, MAX and
 * AVG over non-dictionary columns. */
enum { ORC_EXPR_NONE = 0, ORC_EXPR_ADD = 1, ORC_EXPR_SUB = 2, ORC_EXPR_MUL = 3 };
typedef struct {
  int32_t op;
  uint32_t col;                   /* ignored for COUNT(*) */
  int32_t expr;                   /* ORC_EXPR_* */
  uint32_t col2;                  /* second operand of an expression */
} orc_agg;

typedef struct orc_result orc_result;

/* Decode rows [row_begin, row_end) of one column to int64 (DICT: codes). */
int orc_decode(const orc_column* c, uint64_t row_begin, uint64_t row_end, int64_t* out);

/* Evaluate the query.  Without a filter program (n_filter == 0) a row
 * passes when every conjunct holds: each predicate with or_group 0, and for
 * every group g > 0 at least one of its predicates.  With one, a row passes
 * when the program yields true (or_group must then be 0 everywhere).
 * row_ranges (optional, n_ranges pairs [b,e) in row order) restricts the
 * scan to those rows; n_threads >= 1 splits the scan into fixed 1M-row
 * chunks whose per-chunk maps are merged exactly. */
int orc_query(const orc_column* cols, uint32_t n_cols, uint64_t n_rows,
              const orc_pred* preds, uint32_t n_preds,
              const orc_node* filter, uint32_t n_filter,
              const uint32_t* group_by, uint32_t n_group_by,
              const orc_agg* aggs, uint32_t n_aggs,
              const uint64_t* row_ranges, uint32_t n_ranges,
              uint32_t n_threads, orc_result** out);

int orc_result_status(const orc_result* r);
uint64_t orc_result_num_groups(const orc_result* r);
/* key column k of every group, groups in ascending lexicographic key order */
void orc_result_keys(const orc_result* r, uint32_t k, int64_t* out);
/* aggregate a: SUM/MIN/MAX as int64, COUNT as uint64 bits, AVG / VAR / STD as double */
void orc_result_agg(const orc_result* r, uint32_t a, void* out);
/* exact 128-bit SUM of aggregate a (lo, hi words) for every group */
void orc_result_sum128(const orc_result* r, uint32_t a, uint64_t* lo, int64_t* hi);
void orc_result_free(orc_result* r);

/* n / d rounded once to the nearest double (ties to even), n given as four
 * 64-bit limbs (least significant first), d as two; the rounding step of
 * VAR / STD, exported for its own tests.  0 when d is 0. */
double orc_div_round(const uint64_t* n4, const uint64_t* d2);

/* Common refinement of k RLE columns' run boundaries (Section 6 Alignment):
 * the sorted distinct union of all exclusive run ends, and for each segment
 * and column the index of the run covering it.  Call once with seg_ends and
 * ridx NULL to get the count, then again with buffers of that size
 * (ridx is column-major: ridx[j * S + s]). */
int orc_align(uint32_t k, const int64_t* const* run_ends, const uint64_t* n_runs,
              uint64_t n_rows, uint64_t* n_segments, int64_t* seg_ends, int64_t* ridx);

/* Get Join Index (the paper's Join Operations section): every pair (i, j) of
 * rows with left[i] == right[j] (values as decoded; dictionary columns by
 * code), in ascending (i, j) order.  The paper's Join Index tensors hold the
 * same pairs in whatever order the hash join yields them.  Call once with
 * left_rows and right_rows NULL to get the count, then with buffers of that
 * size. */
int orc_join_index(const orc_column* left, const orc_column* right, uint64_t* n_pairs, int64_t* left_rows,
                   int64_t* right_rows);

/* Apply Join Index: out[k] = the value of column c at row rows[k] (rows in
 * any order, with repeats). */
int orc_apply_join_index(const orc_column* c, const int64_t* rows, uint64_t n, int64_t* out);

#ifdef __cplusplus
}
#endif
#endif
