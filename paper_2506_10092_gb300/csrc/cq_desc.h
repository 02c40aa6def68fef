// cq_desc.h -- device-visible descriptors of a planned query (columns,
// predicates, group keys, aggregates) and of a batch's work list.  Shared by
// the host planner, the ahead-of-time kernels and the kernels compiled at run
// time for one query shape; plain C++ with fixed-width integers only.
#pragma once

#include <stdint.h>

#include "../../include/cq.h"

namespace cq {

// ---------------------------------------------------------------- limits
constexpr int kMaxCols = 16;      // referenced columns per query
constexpr int kMaxPreds = 16;
constexpr int kSplitBits = 12;      // low limb of a split SUM accumulator (s32 == 3)
constexpr int kMaxKeys = 8;
constexpr int kMaxAggs = 16;
constexpr int kMaxBitmapCols = 8; // RLE / index columns per query
constexpr int kMaxPassBitmaps = 4; // row-mode predicates evaluated once per run
constexpr uint64_t kDenseMaxGroups = 1ull << 24;   // larger key domains use the global hash table
constexpr uint32_t kHashMinLog2 = 12;               // global hash table: 2^12 .. 2^26 slots
constexpr uint32_t kHashMaxLog2 = 26;
constexpr int kGlobalProbes = 256;                  // probe bound of the global hash table
constexpr unsigned long long kEmptyGroup = ~0ull;   // empty global (and 64-bit shared) key

enum Enc : uint8_t { ENC_RLE = 1, ENC_DICT = 2, ENC_INDEX = 3, ENC_PACKED = 4, ENC_PLAIN = 5 };

// Normalised predicate kinds.  Every comparison becomes an inclusive range
// or an inequality on the column's *raw* value: the logical value for RLE /
// index / plain columns, the unsigned field (code or offset) for dictionary
// and bit-packed columns (bit width < 64).
enum PredKind : uint8_t {
  PK_RANGE = 0,   // lo <= raw <= hi
  PK_NE = 1,      // raw != lo
  PK_BITMAP = 2,  // bit (raw - lo) of the aux bitmap; outside [lo, hi] fails
  PK_LIST = 3,    // raw in sorted aux list (binary search)
  PK_FALSE = 4,
  PK_TRUE = 5,
};

enum AggKind : uint8_t {
  AK_COUNT = 0,
  AK_SUM = 1,       // raw values (packed: offsets; finalize adds base * COUNT)
  AK_MIN = 2,
  AK_MAX = 3,
  AK_ISUM = 4,      // index column: sum of (value - default) over listed passing rows
  AK_IMIN = 5,      // index column: min over listed passing rows + listed count
  AK_IMAX = 6,
  AK_SUM2 = 7,      // VAR / STD: sum of squared raw values (shifted by the packed base, which
                    // leaves a variance unchanged); its SUM companion is aggregate `pair`
  AK_ISUM2 = 8,     // index column: sum of (value - default)^2 over listed passing rows
};

// Device view of one referenced column.
struct ColDesc {
  uint8_t enc;
  uint8_t v64;       // RLE/INDEX/PLAIN values are int64
  uint8_t e64;       // RLE ends / INDEX positions are int64
  uint8_t bw;        // PACKED/DICT bit width
  uint8_t bslot;     // RLE/INDEX: bitmap slot, 0xFF otherwise
  uint8_t raw_is_offset;  // PACKED with bw < 64: raw value is the unsigned offset
  uint16_t pad0;
  uint32_t stage_off;     // row-level columns: byte offset of the column inside a stage
  uint32_t stage_bytes;   // bytes staged per full tile
  int64_t base;      // PACKED base, INDEX default
  const void* vals;  // RLE run_values | PACKED/DICT words | INDEX values | PLAIN values
  const void* ends;  // RLE run_ends | INDEX positions
  uint64_t n;        // RLE n_runs | INDEX nnz | PACKED/DICT n_words | PLAIN n_rows
};

// A predicate's place in its clause of the conjunctive filter: a clause of
// its own (AND-ed in directly), or a member OR-ed into the clause, the last
// member then AND-ing the clause in.
enum { PC_ALONE = 0, PC_MEMBER = 1, PC_LAST = 2 };

struct PredDesc {
  uint8_t col;       // index into QueryDesc::cols
  uint8_t kind;
  uint8_t n32;       // raw values and bounds fit int32: evaluate in 32 bits (lo32 / hi32)
  uint8_t pbm;       // row mode, RLE / index column: slot of the tile pass bitmap the helper
                     // warp fills once per run / listed row (0xFF: evaluated per row)
  uint8_t neg;       // the complement of the test (NOT); pass bitmaps hold the complement
  uint8_t clause;    // PC_ALONE / PC_MEMBER / PC_LAST
  uint8_t pad_[2];
  uint32_t aux_off;  // 32-bit words into the aux area (bitmap or list of int64 as word pairs)
  uint32_t aux_len;  // bitmap words / list entries
  int32_t lo32, hi32;
  int64_t lo, hi;
};

struct KeyDesc {
  uint8_t col;
  uint8_t remap;     // 1: digit = rank of raw in a bitmap (IN-list) -- aux bitmap + prefix
  uint8_t n32;       // raw values read in 32 bits and |kmin| <= 2^30: digits in 32-bit arithmetic
  uint8_t pad0;
  uint32_t aux_off;  // bitmap words (remap)
  uint32_t aux_len;  // bitmap words (remap)
  uint64_t card;     // number of digit values
  uint64_t stride;   // gid = sum digit * stride (the packed key, ordered like the key tuple)
  int64_t kmin;      // digit = raw - kmin (remap: bitmap covers raw - kmin)
  uint32_t prefix_off; // remap: uint32 prefix popcounts per bitmap word in aux
  uint32_t list_off;   // remap: sorted raw values (int64 word pairs) for decoding ranks
};

struct AggDesc {
  uint8_t kind;
  uint8_t col;       // index into QueryDesc::cols (unused for COUNT)
  uint8_t sw;        // first 64-bit shared-memory accumulator word
  uint8_t wide;      // SUM accumulates 128-bit in shared memory (two words)
  uint8_t sw32;      // first 32-bit shared-memory accumulator word
  uint32_t gw;       // first global accumulator word
  uint8_t op;        // cq_agg_op (for finalize)
  uint8_t out_kind;  // 0 int64, 1 uint64, 2 double
  uint8_t red32;     // SUM: |raw| < 2^24 -> a warp batch (<= 128 values) is reduced in 32 bits
  uint8_t ubits;     // SUM with red32 and raw values in [0, 2^ubits): a warp's prefix sums fit
                     // ubits + 5 bits, so several SUMs share one 32-bit scan (0: not known)
  uint8_t w32;       // MIN/MAX: raw values fit int32 -> 32-bit shared accumulator, warp-reduced
  uint8_t n32;       // values read in 32 bits (narrow column and red32 / w32)
  uint8_t s32;       // SUM: shared accumulator is one 32-bit word (sw32): 1 unsigned, 2 signed;
                     // the flush period keeps it from wrapping; 3: two 32-bit limb words
                     // (sw32: the inputs' low kSplitBits bits, sw32 + 1: the rest), inputs
                     // in [0, 2^24), flush period <= 2^20 rows
  int64_t base;      // value added back at finalize (packed base or index default)
  uint8_t pair;      // AK_SUM2 / AK_ISUM2: the hidden SUM of the same values
  uint8_t expr;      // EXPR_*: the input is col (expr) col2 in actual values (base 0, 64-bit words)
  uint8_t col2;      // second operand's index into QueryDesc::cols
};

enum { EXPR_NONE = 0, EXPR_ADD = 1, EXPR_SUB = 2, EXPR_MUL = 3 };

struct QueryDesc {
  uint64_t n_rows;
  uint64_t n_tiles;        // tiles of this launch: [tile0, tile0 + n_tiles)
  uint64_t tile0;          // first tile of this launch (launches over 2^31 rows are split)
  uint32_t tile_rows;
  uint8_t n_cols, n_preds, n_keys, n_aggs;
  uint8_t seg_mode;        // 1: every referenced column is RLE/index -> items are segments
  uint8_t run_walk;        // segment mode walked run by run (no tiles): threads take equal shares
                           // of the entries of bitmap column run_slot and merge every column's
                           // boundaries over their rows
  uint8_t run_slot;
  uint8_t n_bitmaps;       // RLE/INDEX columns with a per-tile bitmap
  uint8_t n_row_cols;      // columns staged per tile (row mode)
  uint8_t stages;
  uint8_t ncw;             // row mode shape: 16 = one CTA of 16 compute warps per SM, 8 = two such CTAs,
                           // 24 / 28 = one CTA of 24 / 28 compute warps (6144 / 7168-row tiles)
  uint32_t stage_bytes;    // bytes of one stage (all row-level columns)
  uint32_t table_slots;    // shared-memory group-table slots (power of two)
  uint8_t table_dense;     // 1: slot = gid (gid domain fits the table)
  uint8_t line_mode;       // row mode, key 0 on an RLE column (grouping on runs, Section 7): the
                           // shared table is 2^line_log2 lines of line_inner slots, one line per
                           // run of that column (line = run ordinal mod lines), slot = line *
                           // line_inner + the other keys' packed digits; no hashing or probing
  uint8_t line_log2;
  uint8_t line_slot;       // bitmap slot of key 0's column
  uint32_t line_inner;     // slots per line = keys[0].stride
  uint32_t line_swz;       // a line's slot for inner digits x is x ^ (line & line_swz): the
                           // largest power of two (at most 32) dividing line_inner, minus one
  uint8_t n_sw;            // 64-bit shared accumulator words per slot
  uint8_t n_sw32;          // 32-bit shared accumulator words per slot (word 0 = COUNT)
  uint8_t n_gw;            // global accumulator words per group (word 0 = COUNT)
  uint8_t has_index_agg;
  uint8_t n_pbm;           // tile pass bitmaps: predicates 0 .. n_pbm-1 (row mode, RLE / index columns)
  uint32_t flush_rows;     // flush the shared table at least this often (rows)
  uint64_t n_groups;       // dense global domain
  uint8_t row_cols[kMaxCols];   // ColDesc indices of staged columns
  ColDesc cols[kMaxCols];
  PredDesc preds[kMaxPreds];
  KeyDesc keys[kMaxKeys];
  AggDesc aggs[kMaxAggs];
  const uint32_t* aux;     // device: bitmaps, prefix counts, sorted lists
  uint32_t aux_words;
  uint32_t smem_bytes;     // dynamic shared memory of the fused kernel
  // global state
  uint8_t ghash;             // 1: groups live in an open-addressing hash table of n_groups
                             // (a power of two) slots keyed by the packed 64-bit gid; 0: the
                             // dense domain, gid indexes the accumulators directly
  uint8_t key_bits;          // bits of the packed key (hash tables: the finalize sort's width)
  uint32_t sort_blocks;      // hash tables: CTAs of the finalize sort's passes
  unsigned long long* gkeys; // hash tables: [n_groups] packed keys, kEmptyGroup when free
  unsigned long long* skeys[2];  // hash tables: finalize sort buffers (keys)
  uint32_t* svals[2];            // ... and slot indices
  uint32_t* shist;               // ... per-block digit counts [256][sort_blocks]
  unsigned long long* gacc;  // [n_gw][n_groups]
  int* err;                  // device status word (cq_status, 0 = ok)
  unsigned long long* err_info;  // what / where / value of the first device error
  // outputs
  uint32_t n_out;
  uint8_t out_is_key[kMaxKeys + kMaxAggs];
  uint8_t out_index[kMaxKeys + kMaxAggs];
  void* out[kMaxKeys + kMaxAggs];  // device columns [n_groups capacity]
  unsigned long long* out_count;   // number of result rows
  unsigned int* block_counts;      // finalize scratch
};

// ---------------------------------------------------------------- batches
// One unit of a batch's work list: tiles [t_begin, t_begin + n_tiles) of query
// `query`.  A persistent kernel's CTAs take items in list order.
struct BatchItem {
  uint32_t query;
  uint32_t n_tiles;
  uint64_t t_begin;
};

// Header of a batch's control block (device memory, uploaded per launch):
// counts, the work counter and the arrays that follow the header.
struct BatchCtl {
  uint32_t n_queries;
  uint32_t n_items;
  uint32_t n_init_blocks;              // init blocks of all queries (kInitGroups groups each)
  uint32_t n_fin_blocks;               // finalize blocks of all queries (1024 groups each)
  unsigned long long next_item;        // work counter, 0 at upload
  const QueryDesc* descs;              // [n_queries]
  const BatchItem* items;              // [n_items], larger items first
  const uint32_t* init_first;          // [n_queries + 1] first init block of each query
  const uint32_t* fin_first;           // [n_queries + 1] first finalize block of each query
};

constexpr uint32_t kInitGroups = 1024;  // groups initialised per batch init block

}  // namespace cq
