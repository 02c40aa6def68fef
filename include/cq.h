/*
 * cq.h -- C ABI of the compressed-column query library (GB300, sm_103a).
 *
 * The library runs SQL filter -> group-by -> aggregate queries directly on
 * lightweight-compressed columns without decompressing them, the method of
 * "GPU Acceleration of SQL Analytics on Compressed Data" (arXiv 2506.10092):
 * encodings of Section 3, alignment of run boundaries of Section 6 (the
 * common refinement of several RLE columns' runs), selection of Section 6
 * and grouping / aggregation of Section 7 (SUM = value x run length,
 * COUNT = run length, MIN / MAX on values, AVG = SUM / COUNT).
 *
 * Conventions for every entry point:
 *  - Every call returns a cq_status; CQ_OK is 0, errors are negative.  A
 *    human-readable message for the last error of the calling thread is
 *    available from cq_last_error().  No C++ exception crosses the ABI.
 *  - Handles are created by *_create / cq_table_bind / cq_query_run* and
 *    released by the matching *_destroy; all handles belong to the caller.
 *  - "Device" pointers are CUDA device addresses on the context's device;
 *    "host" pointers are ordinary (pageable or pinned) host memory.
 *  - Integer results are exact.  SUM is accumulated in 128 bits and
 *    reported as int64; a group whose SUM does not fit int64 makes the query
 *    fail with CQ_ERR_OVERFLOW.  AVG is the exact 128-bit SUM rounded once to
 *    double (nearest even) divided by the COUNT converted to double.
 *  - The library never falls back to the CPU: with no usable CUDA device the
 *    context cannot be created (CQ_ERR_CUDA).
 */
#ifndef CQ_H
#define CQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cq_ctx cq_ctx;
typedef struct cq_column cq_column;
typedef struct cq_table cq_table;
typedef struct cq_result cq_result;

typedef enum {
  CQ_OK = 0,
  CQ_ERR_INVALID_ARG = -1,   /* malformed argument, plan or column buffer */
  CQ_ERR_UNSORTED = -2,      /* run ends / positions not strictly increasing */
  CQ_ERR_SIZE_MISMATCH = -3, /* lengths disagree (run ends vs n_rows, table rows) */
  CQ_ERR_OOM = -4,           /* device or host allocation failed */
  CQ_ERR_CUDA = -5,          /* a CUDA runtime call failed */
  CQ_ERR_OVERFLOW = -6,      /* a SUM result does not fit int64 */
  CQ_ERR_UNSUPPORTED = -7,   /* valid request outside what this build supports */
  CQ_ERR_TABLE_FULL = -8,    /* group table capacity exceeded (device flag) */
  CQ_ERR_TIMEOUT = -9,       /* a bounded device wait gave up (device flag) */
  CQ_ERR_NOT_READY = -10,    /* cq_result_wait: still running when the timeout expired */
  CQ_ERR_BUSY = -11          /* serving loop: admission refused, over the memory budget */
} cq_status;

typedef enum { CQ_I32 = 1, CQ_I64 = 2 } cq_dtype;

/* mem_flags of the column constructors */
enum {
  CQ_MEM_HOST_COPY = 0,      /* buffers are host memory; the library copies them to the device */
  CQ_MEM_DEVICE_BORROW = 1   /* buffers are device memory the caller keeps alive and unmodified
                                until cq_column_destroy; each must be 16-byte aligned and readable
                                up to the next 16-byte multiple of its length */
};

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  `cuda_stream` (a cudaStream_t,
 * may be NULL for the legacy default stream) is the stream used by calls that
 * are not given one.  The context owns a stream-ordered memory pool from which
 * all per-query scratch and result buffers are taken. */
int cq_ctx_create(int device, void* cuda_stream, cq_ctx** out);
int cq_ctx_destroy(cq_ctx* ctx);

/* Number of streaming multiprocessors of the context's device. */
int cq_ctx_num_sms(cq_ctx* ctx, uint32_t* out);

/* Message describing the last failed call of the calling thread ("" if none).
 * The pointer stays valid until the thread's next cq_* call. */
const char* cq_last_error(void);

/* ------------------------------------------------------------------ columns
 * Section 3 ("Basic Encodings") of the paper.  All constructors validate the
 * buffers (on the device for borrowed buffers) and record the column's value
 * range, which the planner uses for dense group keys and exactness bounds.
 * Creation is synchronous.  A column may be bound into several tables; it is
 * released when the last table holding it and the caller have destroyed it. */

/* RLE (Section 3.1): run i holds run_values[i] on rows
 * [run_ends[i-1], run_ends[i]) (run_ends[-1] = 0).  run_ends are EXCLUSIVE
 * ends -- the paper's inclusive end is run_ends[i] - 1 -- strictly
 * increasing, and the last equals n_rows (a base-table column has no gaps).
 * Adjacent runs may hold equal values.  val_t / end_t: CQ_I32 or CQ_I64.
 * Errors: CQ_ERR_UNSORTED (ends not strictly increasing),
 * CQ_ERR_SIZE_MISMATCH (last end != n_rows, n_runs == 0 with n_rows > 0). */
int cq_column_create_rle(cq_ctx* ctx, cq_dtype val_t, const void* run_values,
                         cq_dtype end_t, const void* run_ends, uint64_t n_runs,
                         uint64_t n_rows, uint32_t mem_flags, cq_column** out);

/* RLE + Index composite (Section 3.2 Composite Encodings): RLE runs for the
 * column's pure stretches, Index entries for its scattered rows.  Run i holds
 * run_values[i] on rows [run_starts[i], run_ends[i]) (exclusive ends); row
 * positions[k] holds values[k].  Runs are sorted and disjoint, positions
 * sorted and unique, and runs and positions together cover rows 0 ..
 * n_rows - 1 exactly once.  All buffers are HOST memory (copied); val_t for
 * run_values and values, pos_t for starts, ends and positions (CQ_I32 /
 * CQ_I64).  The library merges the two parts in row order into one RLE
 * column whose unit runs are the listed rows (cq_column_encoding reports 1,
 * RLE): an RLE run here is a value and an end, a listed row a value
 * and a position, so the merged column is as large as the composite.
 * Errors: CQ_ERR_SIZE_MISMATCH (a row neither started by the next run nor
 * the next listed row -- a gap, an overlap or unsorted input -- or coverage
 * other than n_rows), CQ_ERR_UNSORTED (an empty run), CQ_ERR_INVALID_ARG. */
int cq_column_create_rle_index(cq_ctx* ctx, cq_dtype val_t, cq_dtype pos_t, const void* run_values,
                               const void* run_starts, const void* run_ends, uint64_t n_runs,
                               const void* values, const void* positions, uint64_t nnz, uint64_t n_rows,
                               cq_column** out);

/* Dictionary-encoded strings (Section 2.1: strings are value- and
 * dictionary-encoded to numeric codes).  The dictionary -- always HOST memory
 * -- holds n_entries strings, entry i being dict_bytes[dict_offsets[i] ..
 * dict_offsets[i+1]); entries must be sorted bytewise (unsigned lexicographic,
 * a proper prefix sorts first) and unique, so code order is string order.
 * Row r's code is field r of the LSB-first bit stream in packed_codes
 * (n_words little-endian uint32; field r occupies stream bits
 * [r*bit_width, (r+1)*bit_width), stream bit b is bit b%32 of word b/32).
 * 1 <= bit_width <= 32; n_words >= ceil(n_rows*bit_width/32) rounded up to a
 * multiple of 4 (borrowed buffers; copies are padded by the library).
 * Errors: CQ_ERR_INVALID_ARG (bit width, short buffer, a code >= n_entries,
 * dictionary not sorted / not unique). */
int cq_column_create_dict(cq_ctx* ctx, const char* dict_bytes, const uint64_t* dict_offsets,
                          uint32_t n_entries, const uint32_t* packed_codes, uint64_t n_words,
                          uint32_t bit_width, uint64_t n_rows, uint32_t mem_flags,
                          cq_column** out);

/* Index encoding for sparse data (Section 3.1 Index; unlisted rows hold
 * default_value, which makes it the Plain + Index composite of Section 3.2
 * with a constant plain part): row positions[k] holds values[k]; positions
 * are sorted, unique and < n_rows.  nnz may be 0 or n_rows.
 * Errors: CQ_ERR_UNSORTED, CQ_ERR_INVALID_ARG (position out of range). */
int cq_column_create_index(cq_ctx* ctx, cq_dtype val_t, const void* values,
                           cq_dtype pos_t, const void* positions, uint64_t nnz,
                           int64_t default_value, uint64_t n_rows, uint32_t mem_flags,
                           cq_column** out);

/* Bit-width reduction (Section 3.2, "centering"; here frame of reference with
 * base = the minimum): row r holds base + field r of the LSB-first bit stream
 * in words (layout as for dictionary codes), computed modulo 2^64.
 * 1 <= bit_width <= 64.  logical_t is the column's declared type.
 * Errors: CQ_ERR_INVALID_ARG (bit width, short buffer). */
int cq_column_create_bitpacked(cq_ctx* ctx, cq_dtype logical_t, const uint32_t* words,
                               uint64_t n_words, uint32_t bit_width, int64_t base,
                               uint64_t n_rows, uint32_t mem_flags, cq_column** out);

/* Plain (Section 3.1): one value per row. */
int cq_column_create_plain(cq_ctx* ctx, cq_dtype t, const void* values, uint64_t n_rows,
                           uint32_t mem_flags, cq_column** out);

int cq_column_destroy(cq_column* col);

/* Encoding of a column: 1 RLE, 2 dictionary, 3 index, 4 bit-packed, 5 plain. */
int cq_column_encoding(const cq_column* col, uint32_t* enc);

/* Bytes of the column's compressed device representation (strings excluded). */
int cq_column_device_bytes(const cq_column* col, uint64_t* bytes);

/* ------------------------------------------------------------------ tables */

/* Bind n_cols columns (all with the same n_rows) into a table; column i of
 * the table is cols[i].  The table holds a reference to each column.
 * Errors: CQ_ERR_SIZE_MISMATCH (row counts differ), CQ_ERR_INVALID_ARG. */
int cq_table_bind(cq_ctx* ctx, cq_column* const* cols, uint32_t n_cols, cq_table** out);
int cq_table_destroy(cq_table* table);
int cq_table_num_rows(const cq_table* table, uint64_t* n_rows);

/* ------------------------------------------------------------------ plans
 * A plan is a filter over predicates, each on one column, then GROUP BY the
 * listed columns and the listed aggregates (Sections 6-7).  Predicates on a
 * dictionary column take string literals (strs); predicates on every other
 * column take integer literals compared with the row's logical value.
 * Literals absent from a dictionary simply match nothing.
 *
 * The filter combines the predicates with the logical operators of
 * Section 5 (AND, OR, NOT of masks) in one of two forms:
 *  - conjunctive (filter == NULL): a row passes when every conjunct holds.
 *    A predicate with or_group 0 is a conjunct of its own; the predicates
 *    sharing an or_group g > 0 form one conjunct, their OR.  A predicate
 *    with negate != 0 stands for its complement (NOT), taken before the OR.
 *    All predicates with or_group 0 and negate 0 is the plain AND.
 *  - a program (n_filter > 0): an expression tree over the predicates in
 *    postfix order (below); or_group must then be 0 on every predicate,
 *    negate still complements a predicate where it appears.  The library
 *    rewrites it to the conjunctive form (NOT moved to the predicates by
 *    De Morgan's laws, AND distributed over OR, repeated literals, clauses
 *    that always hold and clauses that contain another clause dropped);
 *    predicates the program does not name play no part.
 * The kernels evaluate at most 16 predicate occurrences in conjunctive
 * form; a program that needs more fails with CQ_ERR_UNSUPPORTED. */
typedef enum {
  CQ_LT = 0, CQ_LE = 1, CQ_GT = 2, CQ_GE = 3, CQ_EQ = 4, CQ_NE = 5,
  CQ_BETWEEN = 6,  /* lo <= v <= hi (strings: strs[0] <= s <= strs[1]) */
  CQ_IN = 7        /* v in in_ints[0..n_in) (strings: s in strs[0..n_strs)) */
} cq_pred_op;

typedef struct {
  uint32_t col;                 /* table column index */
  int32_t op;                   /* cq_pred_op */
  int64_t lo, hi;               /* integer literals: comparisons use lo; BETWEEN uses lo..hi */
  const int64_t* in_ints;       /* IN list on an integer column (host) */
  uint32_t n_in;
  const char* const* strs;      /* string literals on a dictionary column (host) */
  const uint32_t* str_lens;     /* byte length of each literal; NULL = NUL-terminated */
  uint32_t n_strs;
  uint32_t or_group;            /* conjunctive form: 0 = a conjunct of its own; g > 0 = OR-ed
                                   with the plan's other predicates of group g */
  uint32_t negate;              /* nonzero: the predicate's complement (NOT) */
} cq_predicate;

/* One node of a filter program, in postfix order: PRED pushes predicate
 * `arg`'s truth for the row; AND / OR pop `arg` >= 1 values and push their
 * conjunction / disjunction; NOT complements the top value.  The program
 * must leave exactly one value; at most 64 nodes. */
typedef enum { CQ_NODE_PRED = 0, CQ_NODE_AND = 1, CQ_NODE_OR = 2, CQ_NODE_NOT = 3 } cq_node_kind;

typedef struct {
  int32_t kind;                 /* cq_node_kind */
  uint32_t arg;                 /* PRED: predicate index; AND / OR: operand count; NOT: unused */
} cq_filter_node;

/* STD and VAR follow Section 7 (computed from COUNT, SUM and the sum of the
 * squared values): the exact rational (n * sum(x^2) - sum(x)^2) / (n * n)
 * (population) or / (n * (n - 1)) (sample) rounded once to double, 0 when
 * the denominator is 0; STD is the square root of that double.  Their input
 * values must lie within +-2^31 of the column's packed base (index columns:
 * of its default), else planning fails with CQ_ERR_UNSUPPORTED.  Each takes
 * a hidden SUM of the same values, so a plan holds at most 16 aggregates
 * counting those. */
typedef enum {
  CQ_SUM = 0, CQ_COUNT = 1, CQ_MIN = 2, CQ_MAX = 3, CQ_AVG = 4,
  CQ_VAR_POP = 5, CQ_VAR_SAMP = 6, CQ_STD_POP = 7, CQ_STD_SAMP = 8
} cq_agg_op;

/* An aggregate's input is column `col`, or, with an expression, the
 * position-wise result `col` (expr) `col2` of two columns (Section 6:
 * arithmetic on aligned columns, e.g. c1 + c2 after alignment), evaluated
 * once per aligned segment in segment mode and once per row otherwise.
 * Expressions take SUM, MIN, MAX and AVG over non-dictionary columns
 * (CQ_ERR_INVALID_ARG otherwise); the columns' value ranges must keep every
 * result within int64, else planning fails with CQ_ERR_UNSUPPORTED.  Row-mode
 * plans with an expression run the generic row kernel. */
typedef enum { CQ_EXPR_NONE = 0, CQ_EXPR_ADD = 1, CQ_EXPR_SUB = 2, CQ_EXPR_MUL = 3 } cq_expr;

typedef struct {
  int32_t op;                   /* cq_agg_op; only MIN / MAX / COUNT take dictionary columns */
  uint32_t col;                 /* ignored for COUNT(*) */
  int32_t expr;                 /* cq_expr; CQ_EXPR_NONE: the column itself */
  uint32_t col2;                /* second operand of an expression */
} cq_aggregate;

typedef struct {
  const cq_predicate* preds;  uint32_t n_preds;     /* <= 16 */
  const uint32_t* group_by;   uint32_t n_group_by;  /* <= 8 */
  const cq_aggregate* aggs;   uint32_t n_aggs;      /* <= 16 */
  const cq_filter_node* filter; uint32_t n_filter;  /* optional filter program (host); 0 = the
                                                       conjunctive form */
} cq_plan;

/* Execution choices; zero-initialise for the defaults. */
typedef enum {
  CQ_EXEC_FUSED = 0,                 /* compressed-domain fused kernel (the method) */
  CQ_EXEC_DECOMPRESS_THEN_SCAN = 1   /* comparison path: expand every referenced column to
                                        flat device arrays, then a row-wise scan */
} cq_exec_mode;

typedef struct {
  int32_t mode;          /* cq_exec_mode */
  uint32_t tile_rows;    /* rows per tile: 1024, 2048, 4096 or 8192 (smaller ones are tried when
                            shared memory is short); 0 = the planner's choice, which may also be
                            6144 or 7168 rows for its 24- / 28-warp row shapes */
  uint32_t ctas_per_sm;  /* 0 = default (the planner picks); 1, 2, or 3 (segment mode only) */
  uint32_t stages;       /* bulk-copy pipeline depth (1..8); 0 = default (4, fewer if shared
                            memory is short, never below 2) */
  uint32_t table_slots;  /* shared-memory group-table slots per CTA (power of 2); 0 = default */
  uint32_t grid_ctas;    /* CTAs of the fused kernel; 0 = SMs x ctas_per_sm */
  uint32_t items_per_cta;  /* batches: work items per CTA the tiles are cut into
                              (load balance vs per-item overhead); 0 = default */
  uint32_t kernel;       /* 0 = the planner's choice.  Row mode (one-query launches): by default a
                            kernel specialised to the query's shape, compiled at run time on
                            first use and cached by the process (the environment variable
                            CQ_JIT=0 turns this off); 1 = the generic ahead-of-time kernel, which
                            reads the shape from the descriptor.  Segment mode: by default
                            tile by tile, or run by run (a k-way merge of the columns'
                            boundaries, work proportional to the runs) when the columns'
                            entries average 64 or more rows apart; 2 = tiles, 3 = runs */
  uint32_t hash_slots_log2;  /* key domains above 2^24 groups: initial slots of the global hash
                                table as a power of two (12..26); 0 = twice the groups that can
                                exist, 2^12 .. 2^22.  A table that fills is retried by
                                cq_result_wait with four times the slots, up to 2^26 */
} cq_exec_options;

/* ------------------------------------------------------------------ queries */

/* The conjunctive form the kernels evaluate for a plan's filter, computed on
 * the host (no device work): the predicate occurrences with or_group and
 * negate set, copied to out[0 .. *n_out).  The copies' literal pointers
 * (in_ints, strs, str_lens) still point into the caller's plan.  A plan
 * without a filter program comes back as given.  *n_out is set whenever the
 * program is valid, also when it exceeds cap (then CQ_ERR_INVALID_ARG).
 * Errors: CQ_ERR_INVALID_ARG (malformed program, or_group set beside a
 * program), CQ_ERR_UNSUPPORTED (more than 16 occurrences, or an expansion
 * beyond the work limit). */
int cq_filter_conjunctive(const cq_plan* plan, cq_predicate* out, uint32_t cap, uint32_t* n_out);

/* Plan the query on `table` and enqueue its kernels on `cuda_stream`
 * (NULL: the context's stream).  Asynchronous: returns once the work is
 * enqueued; the result handle owns every device buffer of the query.
 * Output columns are the group keys in group_by order, then the aggregates
 * in plan order.  Groups are the distinct key tuples of rows that pass every
 * predicate, in ascending lexicographic key order (dictionary keys by code,
 * i.e. by string); a plan without GROUP BY yields exactly one row (COUNT 0,
 * SUM 0, MIN / MAX / AVG 0 when nothing passes).
 * Tables of more than 2^31 rows run as several launches of at most 2^31 rows
 * each, with the exact SUM accumulators normalised in between.
 * Key domains (the product of the group-by columns' value ranges) up to
 * 2^24 groups are dense arrays; larger ones, up to 2^62, keep their groups in
 * an open-addressing hash table in device memory keyed by the packed key, and
 * finalize sorts the groups by key (Section 7, grouping phase).
 * Errors (synchronous): CQ_ERR_INVALID_ARG for a malformed plan,
 * CQ_ERR_UNSUPPORTED when the key domain exceeds 2^62 groups. */
int cq_query_run(cq_table* table, const cq_plan* plan, void* cuda_stream, cq_result** out);
int cq_query_run_ex(cq_table* table, const cq_plan* plan, const cq_exec_options* opts,
                    void* cuda_stream, cq_result** out);

/* Run n independent queries (tables[i], plans[i], any tables of the same
 * context, of any sizes) as ONE persistent fused launch.  No counterpart in
 * the paper, which runs one query at a time; the per-query method is the
 * one of cq_query_run.
 *
 * Each query's tiles are cut into work items of at most C tiles, C chosen so
 * that the batch has about items_per_cta items per CTA; items are ordered
 * larger first and a one-CTA-per-SM persistent kernel takes them from a
 * global counter.  Every item adds its partial aggregates into its own
 * query's accumulators, so results[i] equals cq_query_run's result for
 * query i exactly (integer aggregates are order-independent).
 *
 * The launch (upload of descriptors and work list, init, persistent kernel,
 * finalize) is a CUDA graph instantiated once per control-block capacity and
 * replayed for every later batch that fits it; only the upload size changes.
 * opts: mode must be CQ_EXEC_FUSED; tile_rows (0, 4096 or 8192; a query whose
 * shared memory does not fit 8192-row tiles gets 4096) and items_per_cta select the
 * shape (0 = the autotuned shape of cq_batch_tune for this kind of batch,
 * else tiles of 8192 rows, 4 items
 * per CTA); ctas_per_sm, stages and grid_ctas are ignored.
 * Asynchronous like cq_query_run; results[i] is owned by the caller (the
 * device buffers of the batch are freed when its last result is destroyed).
 * Errors (synchronous, no result is returned): those of cq_query_run for any
 * query (the message names the query), CQ_ERR_INVALID_ARG for n == 0 or
 * tables of different contexts, CQ_ERR_UNSUPPORTED for a table of more than
 * 2^31 rows or a key domain above 2^24 groups (run such a query alone). */
int cq_batch_run(uint32_t n, cq_table* const* tables, const cq_plan* plans,
                 const cq_exec_options* opts, void* cuda_stream, cq_result** results);

/* Autotuner for batches: run the batch once per candidate shape (tile rows
 * 4096 or 8192, 1 to 8 items per CTA), time each launch with
 * CUDA events (best of two runs after a warm-up), and remember the fastest
 * for batches of the same kind -- keyed by the number of queries and total
 * rows (powers of two) and the share of all-RLE/index queries -- so that
 * cq_batch_run with tile_rows == 0 uses it.  *best receives the chosen shape
 * and *best_us its launch time.  Synchronous; no results are kept. */
int cq_batch_tune(uint32_t n, cq_table* const* tables, const cq_plan* plans, void* cuda_stream,
                  cq_exec_options* best, double* best_us);

/* Wait up to timeout_us microseconds (UINT64_MAX = forever) for the query
 * to finish.  Returns CQ_OK, CQ_ERR_NOT_READY, or the query's own error
 * (CQ_ERR_OVERFLOW, CQ_ERR_TABLE_FULL, CQ_ERR_TIMEOUT, CQ_ERR_INVALID_ARG
 * for out-of-domain data met on the device, CQ_ERR_CUDA). */
int cq_result_wait(cq_result* res, uint64_t timeout_us);

/* Number of result rows (waits for the query). */
int cq_result_num_groups(cq_result* res, uint64_t* n);

/* Number of output columns and the byte width / kind of column i:
 * kind 0 int64 (keys, SUM, MIN, MAX), 1 uint64 (COUNT), 2 double (AVG). */
int cq_result_num_columns(cq_result* res, uint32_t* n);
int cq_result_column_kind(cq_result* res, uint32_t out_col, uint32_t* kind);

/* Copy output column out_col (num_groups x 8 bytes) to host_dst (waits). */
int cq_result_fetch(cq_result* res, uint32_t out_col, void* host_dst, uint64_t dst_bytes);

/* Device address of output column out_col (valid until cq_result_destroy). */
int cq_result_device_column(cq_result* res, uint32_t out_col, const void** dptr);

/* The dictionary string of key column key_col (must be a dictionary column)
 * in result row `row`; the pointer is into the column's host dictionary. */
int cq_result_key_string(cq_result* res, uint32_t key_col, uint64_t row,
                         const char** s, uint32_t* len);

/* Microseconds between the query's first and last kernel on the device
 * (CUDA events on the query's stream; waits for the query). */
int cq_result_device_time_us(cq_result* res, double* us);

/* Microseconds of the fused compressed-domain kernel alone (CUDA events
 * recorded on the query's stream immediately around that launch; waits). */
int cq_result_kernel_time_us(cq_result* res, double* us);

int cq_result_destroy(cq_result* res);

/* ------------------------------------------------------------------ alignment
 * Materialising form of the run-boundary alignment (Section 6, Alignment;
 * Algorithm 1 generalised from two to k RLE columns): the segments are the
 * common refinement of the k columns' runs -- the distinct union of all run
 * ends -- and for every segment and column the index of the run covering it.
 * cols: k RLE columns of equal n_rows.  seg_ends (int64[capacity]) and ridx
 * (int64[k * capacity], column-major: ridx[j * capacity + s]) are DEVICE
 * buffers; n_segments (host) receives the segment count.  When capacity is
 * smaller than the count nothing is written past it and CQ_ERR_SIZE_MISMATCH
 * is returned with *n_segments set (call with capacity 0 to size buffers).
 * Synchronous. */
int cq_align_segments(cq_ctx* ctx, cq_column* const* cols, uint32_t k, void* cuda_stream,
                      int64_t* seg_ends, int64_t* ridx, uint64_t capacity,
                      uint64_t* n_segments);

/* Allocation-free form of cq_align_segments, for callers that cannot
 * allocate device memory while they run (a memory budget owned by someone
 * else, a pre-sized arena, code that must stay out of the CUDA allocator).
 * The paper has no counterpart: this is an interface for such callers.
 * Inputs are raw DEVICE arrays instead of column handles: run_ends[j] holds
 * n_runs[j] exclusive run ends of column j (int64 when end_is_i64[j] is
 * non-zero, else int32), strictly increasing, the last equal to n_rows.
 * Outputs, capacity and the return value are those of cq_align_segments
 * (seg_ends / ridx are device buffers; *n_segments is host memory).
 * No device memory is allocated and none is freed: the only scratch is a
 * fixed device array of CQ_STATIC_ALIGN_MAX_TILES + 8 64-bit words (512 KB)
 * inside the library, held by every GPU that loads it until the process
 * exits; n_rows above CQ_STATIC_ALIGN_MAX_TILES * 4096 is rejected with
 * CQ_ERR_INVALID_ARG.  The first call in each device context (again after
 * cudaDeviceReset) looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and caches it; make that
 * first call before capturing any stream.  All calls share the array and it
 * keeps the last call's contents (the call clears what must start at zero),
 * so calls that overlap on the GPU -- from several host threads or streams --
 * race and must be serialised by the caller.  Synchronous on cuda_stream
 * (NULL: the legacy default stream) of the current device. */
#define CQ_STATIC_ALIGN_MAX_TILES 65536
int cq_align_segments_static(uint32_t k, const void* const* run_ends, const uint32_t* end_is_i64,
                             const uint64_t* n_runs, uint64_t n_rows, void* cuda_stream,
                             int64_t* seg_ends, int64_t* ridx, uint64_t capacity, uint64_t* n_segments);

/* ------------------------------------------------------------------ self-test
 * No counterpart in the paper: checks the failure path of the fused kernels'
 * device waits.  One device thread waits on a barrier that nothing will
 * complete, with the same bounded wait the kernels use on their bulk-copy
 * stages, limited to limit_us microseconds (1 us .. 5 s); *device_status
 * receives the status the wait left (CQ_ERR_TIMEOUT when it gave up, as it
 * must).  The context stays usable afterwards.  Synchronous on the
 * context's stream. */
int cq_selftest_bounded_wait(cq_ctx* ctx, uint32_t limit_us, int32_t* device_status);

/* Row-mode kernels specialised to a query's shape (cq_exec_options.kernel)
 * are compiled at run time, once per shape and process.  *compiles receives
 * how many this process compiled so far, *seconds the compile time they
 * took (either may be NULL).  No counterpart in the paper.  Always CQ_OK. */
int cq_jit_stats(uint64_t* compiles, double* seconds);

/* Compile, without loading, one of eight built-in shapes (variant 0 .. 7)
 * that between them exercise every encoding, predicate kind, clause form,
 * key mapping, aggregate layout and group table of the specialised row
 * kernel (4 and 5: the run-line table; 6 and 7: the serial walk of sorted
 * data): a check
 * of the run-time compiler that needs no GPU.  *seconds (may be NULL)
 * receives the compile time.  CQ_ERR_INVALID_ARG for another variant,
 * CQ_ERR_CUDA (with the compiler's log in cq_last_error) when compilation
 * fails. */
int cq_jit_check(uint32_t variant, double* seconds);

/* ------------------------------------------------------------------ serving
 * A serving loop over tables kept resident on the device (no counterpart in
 * the paper, which times warm queries one at a time; each query's method is
 * that of cq_query_run).  A background thread owns the launches:
 *  - admission: a submitted query is planned at once (plan errors are
 *    returned by cq_server_submit) and its device footprint -- result
 *    buffers and its share of the batch control block -- is computed; it is
 *    admitted to a launch only while the footprints of all queries in flight
 *    stay within memory_budget_bytes;
 *  - two lanes (n_streams >= 2): queries over tables of more than
 *    2^large_rows_log2 rows form the large lane -- planned like cq_query_run
 *    and launched alone; the others are batched.  A fused kernel fills every
 *    SM (one persistent CTA per SM, most of its shared memory), so launches
 *    run one after another on one stream, at most two queued: the waiting
 *    small queries go first, as one batch (cq_batch_run's persistent kernel),
 *    when nothing runs, max_batch are waiting or the oldest has waited
 *    max_wait_us; otherwise the oldest large query runs;
 *  - one lane (n_streams == 1): every query is batched, a batch launched
 *    when nothing runs, max_batch queries wait or the oldest has waited
 *    max_wait_us;
 *  - a query a batch cannot take (a key domain above 2^24 groups, a table
 *    above 2^31 rows) joins the large lane with either setting;
 *  - completion: launches in flight are polled; a finished query's result
 *    and latency (submission to observed completion) go to cq_server_wait.
 * Each query's result equals its cq_query_run result exactly. */
typedef struct cq_server cq_server;

typedef struct {
  uint64_t memory_budget_bytes;  /* admission limit on in-flight query footprints; 0 = 1 GiB */
  uint32_t max_batch;            /* most queries per launch; 0 = 256 */
  uint32_t n_streams;            /* 1: one lane (every query batched); >= 2 (<= 16): two lanes; 0 = 2 */
  uint32_t max_wait_us;          /* how long a partial batch may wait for company; 0 = 50 */
  uint32_t large_rows_log2;      /* tables above 2^this many rows use the large lane; 0 = 22 */
  uint32_t reserved[2];
} cq_server_options;

/* Start a serving loop on ctx (which it keeps alive until destroyed). */
int cq_server_create(cq_ctx* ctx, const cq_server_options* opts, cq_server** out);

/* Submit a query; *ticket identifies it.  Thread-safe.  The plan and its
 * literals are copied and the table's columns are held, so both handles may
 * be released after the call.  Errors: those of planning (CQ_ERR_INVALID_ARG,
 * CQ_ERR_UNSUPPORTED), CQ_ERR_BUSY when the query's footprint alone exceeds
 * the memory budget. */
int cq_server_submit(cq_server* srv, cq_table* table, const cq_plan* plan, uint64_t* ticket);

/* Wait up to timeout_us (UINT64_MAX = forever) for query `ticket`.  On
 * success *res receives its result handle (owned by the caller, already
 * complete) and *latency_us the time from submission to completion seen by
 * the loop.  CQ_ERR_NOT_READY on timeout (the ticket stays valid); a launch
 * error of the query's batch is returned once and ends the ticket.  Each
 * ticket is collected at most once. */
int cq_server_wait(cq_server* srv, uint64_t ticket, uint64_t timeout_us,
                   cq_result** res, double* latency_us);

/* Launches issued and queries completed so far. */
int cq_server_stats(cq_server* srv, uint64_t* launches, uint64_t* completed);

/* Finish every submitted query, stop the loop, free uncollected results. */
int cq_server_destroy(cq_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* CQ_H */
