// cq_oracle.cpp -- plain CPU oracle (test infrastructure only; see cq_oracle.h).
//
// What it computes is the plain SQL definition of the query:
//   1. decompress every referenced column to flat int64 rows (Section 3
//      encodings; each decoder below is written from the encoding's
//      definition, not from any fast path);
//   2. for every row, evaluate each predicate (Section 6, selection;
//      predicates on a dictionary column compare the *bytes* of the row's
//      string with the literal strings), complement it when negated, and
//      combine the truths with the logical operators of Section 5: the
//      filter program's AND / OR / NOT when the query has one, else the AND
//      of the conjuncts (an OR group is one conjunct);
//   3. for a passing row, look its group-by key tuple up in an ordered map
//      and update SUM (128-bit), COUNT, MIN, MAX (Section 7 aggregating
//      phase; App. A.2 worked example);
//   4. emit groups in ascending key order (torch.unique returns sorted
//      values, Section 2.2); AVG = SUM / COUNT in double.
// The compressed-domain method reaches exactly this result, so no tolerance
// is involved: integer results are compared bit for bit.
#include "cq_oracle.h"

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

namespace {

typedef __int128 i128;

// Unsigned 256-bit integer (two 128-bit limbs) for the exact sums of squares
// and the variance numerator.
typedef unsigned __int128 u128;
struct U256 {
  u128 lo = 0, hi = 0;
};

U256 add256(U256 a, U256 b) {
  U256 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1 : 0);
  return r;
}

U256 sub256(U256 a, U256 b) {   // a >= b
  U256 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1 : 0);
  return r;
}

// full product of two 128-bit values, schoolbook on 64-bit halves
U256 mul128(u128 a, u128 b) {
  const u128 m = ~(u128)0 >> 64;
  const u128 a0 = a & m, a1 = a >> 64, b0 = b & m, b1 = b >> 64;
  const u128 p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  const u128 mid = (p00 >> 64) + (p01 & m) + (p10 & m);
  U256 r;
  r.lo = (p00 & m) | (mid << 64);
  r.hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
  return r;
}

int bitlen256(U256 a) {
  int n = 0;
  if (a.hi) {
    n = 128;
    for (u128 x = a.hi; x; x >>= 1) ++n;
  } else {
    for (u128 x = a.lo; x; x >>= 1) ++n;
  }
  return n;
}

bool bit256(U256 a, int i) { return i < 128 ? ((a.lo >> i) & 1) : ((a.hi >> (i - 128)) & 1); }

bool ge256(U256 a, U256 b) { return a.hi != b.hi ? a.hi > b.hi : a.lo >= b.lo; }

U256 shl1(U256 a) {
  U256 r;
  r.hi = (a.hi << 1) | (a.lo >> 127);
  r.lo = a.lo << 1;
  return r;
}

// n / d rounded once to the nearest double (ties to even), d > 0: the
// quotient's bits are produced by long division until 64 significant bits
// are known; every further bit and the remainder fold into a sticky bit.
double div_round(U256 n, u128 d) {
  if (n.lo == 0 && n.hi == 0) return 0.0;
  U256 dd;
  dd.lo = d;
  U256 rem;
  uint64_t top = 0;     // leading quotient bits
  int got = 0;          // significant quotient bits in top
  int exp2 = 0;         // value = top * 2^exp2 (before rounding)
  bool sticky = false;
  // integer part: bits of n from the most significant down
  for (int i = bitlen256(n) - 1; i >= 0; --i) {
    rem = shl1(rem);
    if (bit256(n, i)) rem.lo |= 1;
    const bool q = ge256(rem, dd);
    if (q) rem = sub256(rem, dd);
    if (got < 64) {
      if (got || q) {
        top = (top << 1) | (q ? 1u : 0u);
        ++got;
      }
    } else {
      sticky = sticky || q;
      ++exp2;
    }
  }
  // fraction bits until 64 significant bits are known
  while (got < 64) {
    rem = shl1(rem);
    const bool q = ge256(rem, dd);
    if (q) rem = sub256(rem, dd);
    if (got || q) {
      top = (top << 1) | (q ? 1u : 0u);
      ++got;
    }
    --exp2;
  }
  sticky = sticky || rem.lo != 0 || rem.hi != 0;
  // top has 64 bits and the sticky lies below a double's rounding position
  return std::ldexp((double)(top | (sticky ? 1u : 0u)), exp2);
}

// Variance from n, the exact SUM s1 and sum of squares s2 (Section 7):
// (n * s2 - s1^2) / (n * n) for the population, / (n * (n - 1)) for a sample.
double variance(uint64_t n, i128 s1, U256 s2, bool sample) {
  const uint64_t den1 = sample ? n - 1 : n;
  if (n == 0 || den1 == 0) return 0.0;
  const u128 a1 = s1 < 0 ? (u128)(-s1) : (u128)s1;
  const U256 sq = mul128(a1, a1);
  const U256 ns2 = add256(mul128(s2.lo, (u128)n), [&] {
    U256 h = mul128(s2.hi, (u128)n);   // s2.hi * n * 2^128: its low limb shifts up
    U256 r;
    r.hi = h.lo;
    return r;
  }());
  const U256 num = sub256(ns2, sq);   // >= 0 (Cauchy-Schwarz)
  return div_round(num, (u128)n * (u128)den1);
}

struct Acc {
  uint64_t count = 0;
  std::vector<i128> sum;
  std::vector<U256> sq;     // sums of squares (VAR / STD)
  std::vector<int64_t> mn, mx;
  std::vector<bool> seen;
};

int cmp_bytes(const uint8_t* a, uint64_t la, const uint8_t* b, uint64_t lb) {
  uint64_t m = la < lb ? la : lb;
  int c = m ? std::memcmp(a, b, m) : 0;
  if (c != 0) return c < 0 ? -1 : 1;
  if (la == lb) return 0;
  return la < lb ? -1 : 1;
}

const uint8_t* dict_str(const orc_column& c, int64_t code, uint64_t* len) {
  uint64_t b = c.dict_offsets[code], e = c.dict_offsets[code + 1];
  *len = e - b;
  return c.dict_bytes + b;
}

// field i of an LSB-first bit stream over little-endian 32-bit words
uint64_t read_field(const uint32_t* words, uint64_t n_words, uint64_t i, uint32_t w) {
  unsigned __int128 bit = (unsigned __int128)i * w;
  uint64_t q = (uint64_t)(bit / 32);
  uint32_t s = (uint32_t)(bit % 32);
  unsigned __int128 window = 0;
  for (uint32_t k = 0; k < 3; ++k)
    if (q + k < n_words) window |= (unsigned __int128)words[q + k] << (32 * k);
  unsigned __int128 mask = (((unsigned __int128)1) << w) - 1;
  return (uint64_t)((window >> s) & mask);
}

int validate(const orc_column& c, uint64_t n_rows) {
  if (c.n_rows != n_rows) return ORC_ERR_ARG;
  switch (c.enc) {
    case ORC_RLE: {
      if (n_rows == 0) return c.n_runs == 0 ? ORC_OK : ORC_ERR_ARG;
      if (c.n_runs == 0) return ORC_ERR_ARG;
      int64_t prev = 0;
      for (uint64_t i = 0; i < c.n_runs; ++i) {
        if (c.run_ends[i] <= prev) return ORC_ERR_ARG;
        prev = c.run_ends[i];
      }
      return (uint64_t)prev == n_rows ? ORC_OK : ORC_ERR_ARG;
    }
    case ORC_PACKED:
    case ORC_DICT: {
      uint32_t wmax = c.enc == ORC_DICT ? 32 : 64;
      if (c.bit_width < 1 || c.bit_width > wmax) return ORC_ERR_ARG;
      if (c.n_words < (n_rows * c.bit_width + 31) / 32) return ORC_ERR_ARG;
      if (c.enc == ORC_DICT) {
        for (uint32_t i = 0; i + 1 < c.n_entries; ++i) {
          uint64_t la, lb;
          const uint8_t* a = dict_str(c, i, &la);
          const uint8_t* b = dict_str(c, i + 1, &lb);
          if (cmp_bytes(a, la, b, lb) >= 0) return ORC_ERR_ARG;   // sorted, unique
        }
      }
      return ORC_OK;
    }
    case ORC_INDEX: {
      for (uint64_t i = 0; i < c.nnz; ++i) {
        if (c.positions[i] < 0 || (uint64_t)c.positions[i] >= n_rows) return ORC_ERR_ARG;
        if (i && c.positions[i] <= c.positions[i - 1]) return ORC_ERR_ARG;
      }
      return ORC_OK;
    }
    case ORC_PLAIN:
      return ORC_OK;
    case ORC_PACKED_INDEX: {
      if (c.bit_width < 1 || c.bit_width > 64) return ORC_ERR_ARG;
      if (c.n_words < (n_rows * c.bit_width + 31) / 32) return ORC_ERR_ARG;
      for (uint64_t i = 0; i < c.nnz; ++i) {
        if (c.positions[i] < 0 || (uint64_t)c.positions[i] >= n_rows) return ORC_ERR_ARG;
        if (i && c.positions[i] <= c.positions[i - 1]) return ORC_ERR_ARG;
      }
      return ORC_OK;
    }
    case ORC_RLE_INDEX: {
      // walk rows in order: each next row must start a run or be listed
      uint64_t cursor = 0, i = 0, k = 0;
      while (i < c.n_runs || k < c.nnz) {
        if (i < c.n_runs && c.run_starts[i] == (int64_t)cursor) {
          if (c.run_ends[i] <= c.run_starts[i]) return ORC_ERR_ARG;
          cursor = (uint64_t)c.run_ends[i++];
        } else if (k < c.nnz && c.positions[k] == (int64_t)cursor) {
          ++cursor;
          ++k;
        } else {
          return ORC_ERR_ARG;   // a gap, an overlap or an unsorted entry
        }
      }
      return cursor == n_rows ? ORC_OK : ORC_ERR_ARG;
    }
  }
  return ORC_ERR_ARG;
}

}  // namespace

extern "C" int orc_decode(const orc_column* cp, uint64_t rb, uint64_t re, int64_t* out) {
  const orc_column& c = *cp;
  if (re < rb || re > c.n_rows) return ORC_ERR_ARG;
  switch (c.enc) {
    case ORC_RLE: {
      // the run holding row r is the first run whose exclusive end exceeds r
      uint64_t i = std::upper_bound(c.run_ends, c.run_ends + c.n_runs, (int64_t)rb) - c.run_ends;
      for (uint64_t r = rb; r < re; ++r) {
        while ((int64_t)r >= c.run_ends[i]) ++i;
        out[r - rb] = c.run_values[i];
      }
      return ORC_OK;
    }
    case ORC_PACKED:
      for (uint64_t r = rb; r < re; ++r)
        out[r - rb] = (int64_t)((uint64_t)c.base + read_field(c.words, c.n_words, r, c.bit_width));
      return ORC_OK;
    case ORC_DICT:
      for (uint64_t r = rb; r < re; ++r) {
        uint64_t code = read_field(c.words, c.n_words, r, c.bit_width);
        if (code >= c.n_entries) return ORC_ERR_ARG;
        out[r - rb] = (int64_t)code;
      }
      return ORC_OK;
    case ORC_INDEX: {
      for (uint64_t r = rb; r < re; ++r) out[r - rb] = c.default_value;
      uint64_t k = std::lower_bound(c.positions, c.positions + c.nnz, (int64_t)rb) - c.positions;
      for (; k < c.nnz && (uint64_t)c.positions[k] < re; ++k) out[c.positions[k] - rb] = c.idx_values[k];
      return ORC_OK;
    }
    case ORC_PLAIN:
      for (uint64_t r = rb; r < re; ++r) out[r - rb] = c.values[r];
      return ORC_OK;
    case ORC_PACKED_INDEX: {
      // the packed field, replaced by the listed value on listed rows
      for (uint64_t r = rb; r < re; ++r)
        out[r - rb] = (int64_t)((uint64_t)c.base + read_field(c.words, c.n_words, r, c.bit_width));
      uint64_t k = std::lower_bound(c.positions, c.positions + c.nnz, (int64_t)rb) - c.positions;
      for (; k < c.nnz && (uint64_t)c.positions[k] < re; ++k) out[c.positions[k] - rb] = c.idx_values[k];
      return ORC_OK;
    }
    case ORC_RLE_INDEX:
      // row r: the listed value, else the value of the run starting at or
      // before r (validate() has checked that one of them covers r)
      for (uint64_t r = rb; r < re; ++r) {
        const int64_t* p = std::lower_bound(c.positions, c.positions + c.nnz, (int64_t)r);
        if (p != c.positions + c.nnz && *p == (int64_t)r) {
          out[r - rb] = c.idx_values[p - c.positions];
          continue;
        }
        const int64_t* s = std::upper_bound(c.run_starts, c.run_starts + c.n_runs, (int64_t)r);
        if (s == c.run_starts) return ORC_ERR_ARG;
        const uint64_t i = (uint64_t)(s - c.run_starts) - 1;
        if ((int64_t)r >= c.run_ends[i]) return ORC_ERR_ARG;
        out[r - rb] = c.run_values[i];
      }
      return ORC_OK;
  }
  return ORC_ERR_ARG;
}

struct orc_result {
  int status = ORC_OK;
  uint32_t n_keys = 0, n_aggs = 0;
  std::vector<int32_t> ops;
  std::vector<std::vector<int64_t>> keys;   // [group][k]
  std::vector<Acc> acc;
};

namespace {

struct Query {
  const orc_column* cols;
  uint32_t n_cols;
  const orc_pred* preds;
  uint32_t n_preds;
  const orc_node* filter;
  uint32_t n_filter;
  const uint32_t* gb;
  uint32_t n_gb;
  const orc_agg* aggs;
  uint32_t n_aggs;
  std::vector<uint32_t> used;                 // referenced columns
  std::vector<int> slot;                      // column -> position in `used`
  std::vector<std::vector<uint8_t>> str_pass; // per predicate on a DICT column: result per code
  std::vector<uint32_t> groups;               // distinct nonzero OR groups
};

bool eval_int(const orc_pred& p, int64_t v) {
  switch (p.op) {
    case ORC_LT: return v < p.lo;
    case ORC_LE: return v <= p.lo;
    case ORC_GT: return v > p.lo;
    case ORC_GE: return v >= p.lo;
    case ORC_EQ: return v == p.lo;
    case ORC_NE: return v != p.lo;
    case ORC_BETWEEN: return p.lo <= v && v <= p.hi;
    case ORC_IN:
      for (uint32_t i = 0; i < p.n_in; ++i)
        if (p.in_ints[i] == v) return true;
      return false;
  }
  return false;
}

bool eval_str(const orc_pred& p, const uint8_t* s, uint64_t ls) {
  auto c = [&](uint32_t i) { return cmp_bytes(s, ls, p.strs[i], p.str_lens[i]); };
  switch (p.op) {
    case ORC_LT: return c(0) < 0;
    case ORC_LE: return c(0) <= 0;
    case ORC_GT: return c(0) > 0;
    case ORC_GE: return c(0) >= 0;
    case ORC_EQ: return c(0) == 0;
    case ORC_NE: return c(0) != 0;
    case ORC_BETWEEN: return c(0) >= 0 && c(1) <= 0;
    case ORC_IN:
      for (uint32_t i = 0; i < p.n_strs; ++i)
        if (c(i) == 0) return true;
      return false;
  }
  return false;
}

// Truth of predicate i on the row, complemented when it is negated
// (Section 5.3, NOT of a mask).
bool atom(const Query& q, uint32_t i, const std::vector<int64_t>& row) {
  const orc_pred& p = q.preds[i];
  const int64_t v = row[q.slot[p.col]];
  const bool t = q.cols[p.col].enc == ORC_DICT ? q.str_pass[i][v] != 0 : eval_int(p, v);
  return p.negate ? !t : t;
}

// Whether the row passes the filter: the postfix program over the
// predicates' truths (Sections 5.1-5.3: AND, OR, NOT of masks) when there is
// one, else the conjunction of the or_group-0 predicates and, for each
// group g > 0, the disjunction of its predicates.
bool row_passes(const Query& q, const std::vector<int64_t>& row, std::vector<uint8_t>& stack) {
  if (q.n_filter) {
    stack.clear();
    for (uint32_t k = 0; k < q.n_filter; ++k) {
      const orc_node& nd = q.filter[k];
      if (nd.kind == ORC_NODE_PRED) {
        stack.push_back(atom(q, nd.arg, row) ? 1 : 0);
      } else if (nd.kind == ORC_NODE_NOT) {
        stack.back() = stack.back() ? 0 : 1;
      } else {
        const bool is_and = nd.kind == ORC_NODE_AND;
        bool r = is_and;
        for (uint32_t j = 0; j < nd.arg; ++j) {
          const bool x = stack.back() != 0;
          stack.pop_back();
          r = is_and ? (r && x) : (r || x);
        }
        stack.push_back(r ? 1 : 0);
      }
    }
    return stack.back() != 0;
  }
  for (uint32_t i = 0; i < q.n_preds; ++i)
    if (q.preds[i].or_group == 0 && !atom(q, i, row)) return false;
  for (uint32_t g : q.groups) {
    bool any = false;
    for (uint32_t i = 0; i < q.n_preds && !any; ++i)
      if (q.preds[i].or_group == g) any = atom(q, i, row);
    if (!any) return false;
  }
  return true;
}

typedef std::map<std::vector<int64_t>, Acc> GroupMap;

// The input value of aggregate g at this row: the column's value, or the
// exact result of the expression (false when it leaves the int64 range).
bool agg_value(const Query& q, const orc_agg& g, const std::vector<int64_t>& row, int64_t* v) {
  const int64_t x = row[q.slot[g.col]];
  if (g.expr == ORC_EXPR_NONE) {
    *v = x;
    return true;
  }
  const i128 a = x, b = row[q.slot[g.col2]];
  const i128 r = g.expr == ORC_EXPR_ADD ? a + b : (g.expr == ORC_EXPR_SUB ? a - b : a * b);
  if (r > (i128)INT64_MAX || r < (i128)INT64_MIN) return false;
  *v = (int64_t)r;
  return true;
}

bool update(const Query& q, Acc& a, const std::vector<int64_t>& row) {
  if (a.sum.empty()) {
    a.sq.assign(q.n_aggs, U256());
    a.sum.assign(q.n_aggs, 0);
    a.mn.assign(q.n_aggs, 0);
    a.mx.assign(q.n_aggs, 0);
    a.seen.assign(q.n_aggs, false);
  }
  a.count += 1;
  for (uint32_t i = 0; i < q.n_aggs; ++i) {
    const orc_agg& g = q.aggs[i];
    if (g.op == ORC_COUNT) continue;
    int64_t v;
    if (!agg_value(q, g, row, &v)) return false;
    const orc_column& c = q.cols[g.col];
    if (g.op == ORC_SUM || g.op == ORC_AVG || g.op >= ORC_VAR_POP) a.sum[i] += (i128)v;
    if (g.op >= ORC_VAR_POP) {
      const u128 m = v < 0 ? (u128)(-(i128)v) : (u128)v;
      a.sq[i] = add256(a.sq[i], mul128(m, m));
    }
    if (g.op == ORC_MIN || g.op == ORC_MAX) {
      if (!a.seen[i]) {
        a.mn[i] = a.mx[i] = v;
        a.seen[i] = true;
      } else if (c.enc == ORC_DICT) {        // dictionary: order of the strings
        uint64_t l0, l1, l2;
        const uint8_t* s0 = dict_str(c, v, &l0);
        const uint8_t* s1 = dict_str(c, a.mn[i], &l1);
        const uint8_t* s2 = dict_str(c, a.mx[i], &l2);
        if (cmp_bytes(s0, l0, s1, l1) < 0) a.mn[i] = v;
        if (cmp_bytes(s0, l0, s2, l2) > 0) a.mx[i] = v;
      } else {
        if (v < a.mn[i]) a.mn[i] = v;
        if (v > a.mx[i]) a.mx[i] = v;
      }
    }
  }
  return true;
}

void merge_into(const Query& q, GroupMap& dst, const GroupMap& src) {
  for (const auto& kv : src) {
    auto it = dst.find(kv.first);
    if (it == dst.end()) { dst.insert(kv); continue; }
    Acc& a = it->second;
    const Acc& b = kv.second;
    a.count += b.count;
    for (uint32_t i = 0; i < q.n_aggs; ++i) {
      const orc_agg& g = q.aggs[i];
      a.sum[i] += b.sum[i];
      a.sq[i] = add256(a.sq[i], b.sq[i]);
      if (!b.seen[i]) continue;
      if (!a.seen[i]) { a.mn[i] = b.mn[i]; a.mx[i] = b.mx[i]; a.seen[i] = true; continue; }
      const orc_column& c = q.cols[g.col];
      if (c.enc == ORC_DICT) {
        uint64_t l1, l2;
        const uint8_t* s1; const uint8_t* s2;
        s1 = dict_str(c, b.mn[i], &l1); s2 = dict_str(c, a.mn[i], &l2);
        if (cmp_bytes(s1, l1, s2, l2) < 0) a.mn[i] = b.mn[i];
        s1 = dict_str(c, b.mx[i], &l1); s2 = dict_str(c, a.mx[i], &l2);
        if (cmp_bytes(s1, l1, s2, l2) > 0) a.mx[i] = b.mx[i];
      } else {
        a.mn[i] = std::min(a.mn[i], b.mn[i]);
        a.mx[i] = std::max(a.mx[i], b.mx[i]);
      }
    }
  }
}

int scan_chunk(const Query& q, uint64_t rb, uint64_t re, GroupMap& groups) {
  const uint64_t n = re - rb;
  std::vector<std::vector<int64_t>> flat(q.used.size(), std::vector<int64_t>(n));
  for (size_t u = 0; u < q.used.size(); ++u) {
    int rc = orc_decode(&q.cols[q.used[u]], rb, re, flat[u].data());
    if (rc != ORC_OK) return rc;
  }
  std::vector<int64_t> row(q.used.size());
  std::vector<int64_t> key(q.n_gb);
  std::vector<uint8_t> stack;
  for (uint64_t r = 0; r < n; ++r) {
    for (size_t u = 0; u < q.used.size(); ++u) row[u] = flat[u][r];
    if (!row_passes(q, row, stack)) continue;
    for (uint32_t k = 0; k < q.n_gb; ++k) key[k] = row[q.slot[q.gb[k]]];
    if (!update(q, groups[key], row)) return ORC_ERR_OVERFLOW;
  }
  return ORC_OK;
}

}  // namespace

extern "C" int orc_query(const orc_column* cols, uint32_t n_cols, uint64_t n_rows,
                         const orc_pred* preds, uint32_t n_preds,
                         const orc_node* filter, uint32_t n_filter,
                         const uint32_t* group_by, uint32_t n_group_by,
                         const orc_agg* aggs, uint32_t n_aggs,
                         const uint64_t* row_ranges, uint32_t n_ranges,
                         uint32_t n_threads, orc_result** out) {
  *out = nullptr;
  Query q{cols, n_cols, preds, n_preds, filter, n_filter, group_by, n_group_by, aggs, n_aggs, {}, {}, {}, {}};
  // the filter program must be well formed: every operand present, one
  // value left; OR groups are not combined with a program
  if (n_filter && !filter) return ORC_ERR_ARG;
  {
    uint32_t depth = 0;
    for (uint32_t k = 0; k < n_filter; ++k) {
      const orc_node& nd = filter[k];
      if (nd.kind == ORC_NODE_PRED) {
        if (nd.arg >= n_preds) return ORC_ERR_ARG;
        ++depth;
      } else if (nd.kind == ORC_NODE_NOT) {
        if (depth < 1) return ORC_ERR_ARG;
      } else if (nd.kind == ORC_NODE_AND || nd.kind == ORC_NODE_OR) {
        if (nd.arg < 1 || nd.arg > depth) return ORC_ERR_ARG;
        depth -= nd.arg - 1;
      } else {
        return ORC_ERR_ARG;
      }
    }
    if (n_filter && depth != 1) return ORC_ERR_ARG;
  }
  for (uint32_t i = 0; i < n_preds; ++i) {
    const uint32_t g = preds[i].or_group;
    if (g && n_filter) return ORC_ERR_ARG;
    if (g && std::find(q.groups.begin(), q.groups.end(), g) == q.groups.end()) q.groups.push_back(g);
  }
  q.slot.assign(n_cols, -1);
  auto use = [&](uint32_t c) {
    if (c >= n_cols) return false;
    if (q.slot[c] < 0) { q.slot[c] = (int)q.used.size(); q.used.push_back(c); }
    return true;
  };
  for (uint32_t i = 0; i < n_preds; ++i) if (!use(preds[i].col)) return ORC_ERR_ARG;
  for (uint32_t i = 0; i < n_group_by; ++i) if (!use(group_by[i])) return ORC_ERR_ARG;
  for (uint32_t i = 0; i < n_aggs; ++i) {
    if (aggs[i].op < ORC_SUM || aggs[i].op > ORC_STD_SAMP) return ORC_ERR_ARG;
    if (aggs[i].op == ORC_COUNT) continue;
    if (!use(aggs[i].col)) return ORC_ERR_ARG;
    if (cols[aggs[i].col].enc == ORC_DICT && aggs[i].op != ORC_MIN && aggs[i].op != ORC_MAX)
      return ORC_ERR_ARG;
    if (aggs[i].expr < ORC_EXPR_NONE || aggs[i].expr > ORC_EXPR_MUL) return ORC_ERR_ARG;
    if (aggs[i].expr != ORC_EXPR_NONE) {
      const int32_t op = aggs[i].op;
      if (op != ORC_SUM && op != ORC_MIN && op != ORC_MAX && op != ORC_AVG) return ORC_ERR_ARG;
      if (!use(aggs[i].col2)) return ORC_ERR_ARG;
      if (cols[aggs[i].col].enc == ORC_DICT || cols[aggs[i].col2].enc == ORC_DICT) return ORC_ERR_ARG;
    }
  }
  for (uint32_t c : q.used) if (validate(cols[c], n_rows) != ORC_OK) return ORC_ERR_ARG;
  // A predicate on a dictionary column is a function of the row's string;
  // it is evaluated once per dictionary entry by comparing bytes.
  q.str_pass.resize(n_preds);
  for (uint32_t i = 0; i < n_preds; ++i) {
    const orc_pred& p = preds[i];
    const orc_column& c = cols[p.col];
    if (c.enc != ORC_DICT) {
      if (p.n_strs) return ORC_ERR_ARG;
      continue;
    }
    uint32_t need = p.op == ORC_IN ? p.n_strs : (p.op == ORC_BETWEEN ? 2u : 1u);
    if (p.op != ORC_IN && p.n_strs < need) return ORC_ERR_ARG;
    q.str_pass[i].resize(c.n_entries);
    for (uint32_t code = 0; code < c.n_entries; ++code) {
      uint64_t l;
      const uint8_t* s = dict_str(c, code, &l);
      q.str_pass[i][code] = eval_str(p, s, l) ? 1 : 0;
    }
  }
  // chunks of at most 1M rows over the requested row ranges
  std::vector<std::pair<uint64_t, uint64_t>> chunks;
  const uint64_t CH = 1u << 20;
  auto add_range = [&](uint64_t b, uint64_t e) {
    for (uint64_t x = b; x < e; x += CH) chunks.push_back({x, std::min(e, x + CH)});
  };
  if (row_ranges && n_ranges) {
    for (uint32_t i = 0; i < n_ranges; ++i) {
      uint64_t b = row_ranges[2 * i], e = row_ranges[2 * i + 1];
      if (b > e || e > n_rows) return ORC_ERR_ARG;
      add_range(b, e);
    }
  } else {
    add_range(0, n_rows);
  }
  if (n_threads < 1) n_threads = 1;
  if (n_threads > chunks.size()) n_threads = chunks.empty() ? 1 : (uint32_t)chunks.size();
  std::vector<GroupMap> maps(n_threads);
  std::vector<int> rcs(n_threads, ORC_OK);
  std::atomic<size_t> next{0};
  auto worker = [&](uint32_t t) {
    for (;;) {
      size_t i = next.fetch_add(1);
      if (i >= chunks.size()) break;
      int rc = scan_chunk(q, chunks[i].first, chunks[i].second, maps[t]);
      if (rc != ORC_OK) { rcs[t] = rc; break; }
    }
  };
  if (n_threads == 1) {
    worker(0);
  } else {
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < n_threads; ++t) th.emplace_back(worker, t);
    for (auto& x : th) x.join();
  }
  for (int rc : rcs) if (rc != ORC_OK) return rc;
  GroupMap& all = maps[0];
  for (uint32_t t = 1; t < n_threads; ++t) merge_into(q, all, maps[t]);
  if (n_group_by == 0 && all.empty()) {          // no GROUP BY: one row even if nothing passes
    Acc a;
    a.sum.assign(n_aggs, 0); a.mn.assign(n_aggs, 0); a.mx.assign(n_aggs, 0); a.seen.assign(n_aggs, false);
    a.sq.assign(n_aggs, U256());
    all[std::vector<int64_t>()] = a;
  }
  orc_result* r = new orc_result;
  r->n_keys = n_group_by;
  r->n_aggs = n_aggs;
  for (uint32_t i = 0; i < n_aggs; ++i) r->ops.push_back(aggs[i].op);
  for (auto& kv : all) {
    Acc& a = kv.second;
    if (a.sum.empty()) { a.sum.assign(n_aggs, 0); a.mn.assign(n_aggs, 0); a.mx.assign(n_aggs, 0); a.seen.assign(n_aggs, false); a.sq.assign(n_aggs, U256()); }
    for (uint32_t i = 0; i < n_aggs; ++i) {
      if (aggs[i].op == ORC_SUM) {
        i128 s = a.sum[i];
        if (s > (i128)INT64_MAX || s < (i128)INT64_MIN) r->status = ORC_ERR_OVERFLOW;
      }
    }
    r->keys.push_back(kv.first);
    r->acc.push_back(a);
  }
  *out = r;
  return ORC_OK;
}

extern "C" int orc_result_status(const orc_result* r) { return r->status; }
extern "C" uint64_t orc_result_num_groups(const orc_result* r) { return r->keys.size(); }

extern "C" void orc_result_keys(const orc_result* r, uint32_t k, int64_t* out) {
  for (size_t g = 0; g < r->keys.size(); ++g) out[g] = r->keys[g][k];
}

extern "C" void orc_result_agg(const orc_result* r, uint32_t a, void* out) {
  int op = r->ops[a];
  for (size_t g = 0; g < r->acc.size(); ++g) {
    const Acc& x = r->acc[g];
    switch (op) {
      case ORC_SUM: ((int64_t*)out)[g] = (int64_t)x.sum[a]; break;   // meaningful when status is OK
      case ORC_COUNT: ((uint64_t*)out)[g] = x.count; break;
      case ORC_MIN: ((int64_t*)out)[g] = x.seen[a] ? x.mn[a] : 0; break;
      case ORC_MAX: ((int64_t*)out)[g] = x.seen[a] ? x.mx[a] : 0; break;
      case ORC_AVG:
        // the compiler's __int128 -> double conversion rounds to nearest even
        ((double*)out)[g] = x.count ? (double)x.sum[a] / (double)x.count : 0.0;
        break;
      case ORC_VAR_POP:
      case ORC_VAR_SAMP:
        ((double*)out)[g] = variance(x.count, x.sum[a], x.sq[a], op == ORC_VAR_SAMP);
        break;
      case ORC_STD_POP:
      case ORC_STD_SAMP:
        ((double*)out)[g] = std::sqrt(variance(x.count, x.sum[a], x.sq[a], op == ORC_STD_SAMP));
        break;
    }
  }
}

extern "C" void orc_result_sum128(const orc_result* r, uint32_t a, uint64_t* lo, int64_t* hi) {
  for (size_t g = 0; g < r->acc.size(); ++g) {
    unsigned __int128 u = (unsigned __int128)r->acc[g].sum[a];
    lo[g] = (uint64_t)u;
    hi[g] = (int64_t)(uint64_t)(u >> 64);
  }
}

extern "C" void orc_result_free(orc_result* r) { delete r; }

extern "C" double orc_div_round(const uint64_t* n4, const uint64_t* d2) {
  U256 n;
  n.lo = ((u128)n4[1] << 64) | n4[0];
  n.hi = ((u128)n4[3] << 64) | n4[2];
  const u128 d = ((u128)d2[1] << 64) | d2[0];
  return d ? div_round(n, d) : 0.0;
}

extern "C" int orc_align(uint32_t k, const int64_t* const* run_ends, const uint64_t* n_runs,
                         uint64_t n_rows, uint64_t* n_segments, int64_t* seg_ends, int64_t* ridx) {
  // Segments are the common refinement of all columns' runs: the distinct
  // union of every exclusive run end.  The run of column j covering the
  // segment that ends at e is the first run of j whose end is >= e.
  std::vector<int64_t> all;
  for (uint32_t j = 0; j < k; ++j) {
    if (n_rows && (n_runs[j] == 0 || run_ends[j][n_runs[j] - 1] != (int64_t)n_rows)) return ORC_ERR_ARG;
    for (uint64_t i = 0; i < n_runs[j]; ++i) {
      if (i && run_ends[j][i] <= run_ends[j][i - 1]) return ORC_ERR_ARG;
      all.push_back(run_ends[j][i]);
    }
  }
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  *n_segments = all.size();
  if (seg_ends) for (size_t s = 0; s < all.size(); ++s) seg_ends[s] = all[s];
  if (ridx)
    for (uint32_t j = 0; j < k; ++j)
      for (size_t s = 0; s < all.size(); ++s)
        ridx[j * all.size() + s] = std::lower_bound(run_ends[j], run_ends[j] + n_runs[j], all[s]) - run_ends[j];
  return ORC_OK;
}

// Get Join Index: the definition written out -- for each left row in order,
// the right rows holding the same value, in order.
extern "C" int orc_join_index(const orc_column* left, const orc_column* right, uint64_t* n_pairs,
                              int64_t* left_rows, int64_t* right_rows) {
  if (!left || !right || !n_pairs) return ORC_ERR_ARG;
  if (validate(*left, left->n_rows) != ORC_OK || validate(*right, right->n_rows) != ORC_OK) return ORC_ERR_ARG;
  std::vector<int64_t> lv(left->n_rows), rv(right->n_rows);
  if (orc_decode(left, 0, left->n_rows, lv.data()) != ORC_OK) return ORC_ERR_ARG;
  if (orc_decode(right, 0, right->n_rows, rv.data()) != ORC_OK) return ORC_ERR_ARG;
  std::map<int64_t, std::vector<int64_t>> rows_of;   // right value -> its rows, ascending
  for (uint64_t j = 0; j < rv.size(); ++j) rows_of[rv[j]].push_back((int64_t)j);
  uint64_t n = 0;
  for (uint64_t i = 0; i < lv.size(); ++i) {
    auto it = rows_of.find(lv[i]);
    if (it == rows_of.end()) continue;
    for (int64_t j : it->second) {
      if (left_rows) left_rows[n] = (int64_t)i;
      if (right_rows) right_rows[n] = j;
      ++n;
    }
  }
  *n_pairs = n;
  return ORC_OK;
}

// Apply Join Index: gather the column's values at the given rows.
extern "C" int orc_apply_join_index(const orc_column* c, const int64_t* rows, uint64_t n, int64_t* out) {
  if (!c || (n && (!rows || !out))) return ORC_ERR_ARG;
  if (validate(*c, c->n_rows) != ORC_OK) return ORC_ERR_ARG;
  std::vector<int64_t> v(c->n_rows);
  if (orc_decode(c, 0, c->n_rows, v.data()) != ORC_OK) return ORC_ERR_ARG;
  for (uint64_t k = 0; k < n; ++k) {
    if (rows[k] < 0 || (uint64_t)rows[k] >= c->n_rows) return ORC_ERR_ARG;
    out[k] = v[rows[k]];
  }
  return ORC_OK;
}
