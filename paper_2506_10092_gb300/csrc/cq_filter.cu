// cq_filter.cu -- a plan's boolean filter brought to the form the kernels
// evaluate (host code).
//
// Section 5 defines AND, OR and NOT over mask columns, and Section 5.3
// rewrites composite masks with De Morgan's laws and the distributive law.
// The kernels evaluate a filter as a conjunction of clauses, each clause the
// OR of predicates or their complements (conjunctive normal form): a row's
// truth for every predicate occurrence is computed once per run / row and
// combined by bit operations in the tile (see the filter phases).  A plan
// in that form passes through unchanged.  A plan with a filter program is
// rewritten here:
//   1. the postfix program is parsed into a tree (operands checked);
//   2. NOT is moved down to the predicates (De Morgan: NOT of an AND is the
//      OR of the complements, NOT of an OR the AND of the complements, and a
//      double complement cancels);
//   3. AND is distributed over OR: the clauses of an AND are its operands'
//      clauses; those of an OR are the unions of one clause from each operand;
//   4. each clause keeps a literal once; a clause holding a predicate and its
//      complement always holds and is dropped, as is a clause containing
//      another clause (the smaller one implies it); repeated clauses go.
// The result lists each occurrence of a predicate as its own entry with
// or_group and negate set.
#include "cq_internal.h"

#include <algorithm>
#include <vector>

namespace cq {

namespace {

constexpr uint32_t kMaxNodes = 64;
constexpr size_t kMaxClausesWork = 512;    // clauses held while distributing
constexpr size_t kMaxLiteralsWork = 4096;  // literals held while distributing

typedef std::vector<uint32_t> Clause;      // sorted literals: 2 * pred + negated

struct Node {
  int32_t kind;
  uint32_t arg;
  std::vector<uint32_t> kids;
};

size_t literal_count(const std::vector<Clause>& cs) {
  size_t n = 0;
  for (const Clause& c : cs) n += c.size();
  return n;
}

// Clause set of node i, complemented when `neg` (steps 2-3).  Returns false
// when the intermediate form outgrows the work limits.
bool to_cnf(const std::vector<Node>& t, uint32_t i, bool neg, const cq_plan& p, std::vector<Clause>* out) {
  const Node& nd = t[i];
  if (nd.kind == CQ_NODE_PRED) {
    const bool n = neg != (p.preds[nd.arg].negate != 0);
    out->assign(1, Clause{2 * nd.arg + (n ? 1u : 0u)});
    return true;
  }
  if (nd.kind == CQ_NODE_NOT) return to_cnf(t, nd.kids[0], !neg, p, out);
  // an AND (or a complemented OR) concatenates; an OR (or a complemented AND)
  // distributes
  const bool concat = (nd.kind == CQ_NODE_AND) != neg;
  std::vector<Clause> acc;
  if (!concat) acc.assign(1, Clause{});
  for (uint32_t k : nd.kids) {
    std::vector<Clause> sub;
    if (!to_cnf(t, k, neg, p, &sub)) return false;
    if (concat) {
      acc.insert(acc.end(), sub.begin(), sub.end());
    } else {
      if (acc.size() * sub.size() > kMaxClausesWork) return false;
      std::vector<Clause> prod;
      prod.reserve(acc.size() * sub.size());
      for (const Clause& a : acc)
        for (const Clause& b : sub) {
          Clause c;
          std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(c));
          prod.push_back(std::move(c));
        }
      acc.swap(prod);
    }
    if (acc.size() > kMaxClausesWork || literal_count(acc) > kMaxLiteralsWork) return false;
  }
  out->swap(acc);
  return true;
}

// Step 4 on a clause set.
void simplify(std::vector<Clause>* cs) {
  std::vector<Clause> keep;
  for (Clause& c : *cs) {
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    bool taut = false;
    for (size_t j = 1; j < c.size(); ++j)
      if ((c[j] >> 1) == (c[j - 1] >> 1)) taut = true;  // p and NOT p (adjacent once sorted)
    if (!taut) keep.push_back(c);
  }
  std::sort(keep.begin(), keep.end(), [](const Clause& a, const Clause& b) {
    return a.size() != b.size() ? a.size() < b.size() : a < b;
  });
  keep.erase(std::unique(keep.begin(), keep.end()), keep.end());
  std::vector<Clause> out;
  for (const Clause& c : keep) {
    bool subsumed = false;
    for (const Clause& d : out)
      if (std::includes(c.begin(), c.end(), d.begin(), d.end())) {
        subsumed = true;
        break;
      }
    if (!subsumed) out.push_back(c);
  }
  cs->swap(out);
}

}  // namespace

int normalize_filter(const cq_plan* in, NormFilter* out) {
  out->preds.clear();
  out->plan = *in;
  if (!in->n_filter) return CQ_OK;
  if (!in->filter) return set_error(CQ_ERR_INVALID_ARG, "filter program is NULL");
  if (in->n_filter > kMaxNodes) return set_error(CQ_ERR_INVALID_ARG, "filter program exceeds %u nodes", kMaxNodes);
  if (in->n_preds && !in->preds) return set_error(CQ_ERR_INVALID_ARG, "plan array is NULL");
  for (uint32_t i = 0; i < in->n_preds; ++i)
    if (in->preds[i].or_group)
      return set_error(CQ_ERR_INVALID_ARG, "predicate %u: or_group must be 0 when the plan has a filter program", i);
  // step 1: parse
  std::vector<Node> t;
  std::vector<uint32_t> st;
  for (uint32_t k = 0; k < in->n_filter; ++k) {
    const cq_filter_node& f = in->filter[k];
    Node nd{f.kind, f.arg, {}};
    switch (f.kind) {
      case CQ_NODE_PRED:
        if (f.arg >= in->n_preds)
          return set_error(CQ_ERR_INVALID_ARG, "filter node %u: no predicate %u", k, f.arg);
        break;
      case CQ_NODE_NOT:
        if (st.empty()) return set_error(CQ_ERR_INVALID_ARG, "filter node %u: NOT without an operand", k);
        nd.kids.push_back(st.back());
        st.pop_back();
        break;
      case CQ_NODE_AND:
      case CQ_NODE_OR:
        if (f.arg < 1 || f.arg > st.size())
          return set_error(CQ_ERR_INVALID_ARG, "filter node %u: %u operands requested, %zu available", k, f.arg,
                           st.size());
        nd.kids.assign(st.end() - f.arg, st.end());
        st.resize(st.size() - f.arg);
        break;
      default:
        return set_error(CQ_ERR_INVALID_ARG, "filter node %u: bad kind %d", k, f.kind);
    }
    t.push_back(std::move(nd));
    st.push_back((uint32_t)t.size() - 1);
  }
  if (st.size() != 1)
    return set_error(CQ_ERR_INVALID_ARG, "filter program leaves %zu values (one expected)", st.size());
  // steps 2-4
  std::vector<Clause> cs;
  if (!to_cnf(t, st[0], false, *in, &cs))
    return set_error(CQ_ERR_UNSUPPORTED, "filter program grows beyond %zu clauses in conjunctive normal form",
                     kMaxClausesWork);
  simplify(&cs);
  const size_t lits = literal_count(cs);
  if (lits > (size_t)kMaxPreds)
    return set_error(CQ_ERR_UNSUPPORTED,
                     "filter program needs %zu predicate occurrences in conjunctive normal form (at most %d)", lits,
                     kMaxPreds);
  uint32_t g = 0;
  for (const Clause& c : cs) {
    ++g;
    for (uint32_t l : c) {
      cq_predicate p = in->preds[l >> 1];
      p.or_group = c.size() > 1 ? g : 0;
      p.negate = l & 1u;
      out->preds.push_back(p);
    }
  }
  out->plan.preds = out->preds.empty() ? nullptr : out->preds.data();
  out->plan.n_preds = (uint32_t)out->preds.size();
  out->plan.filter = nullptr;
  out->plan.n_filter = 0;
  return CQ_OK;
}

}  // namespace cq

extern "C" int cq_filter_conjunctive(const cq_plan* plan, cq_predicate* out, uint32_t cap, uint32_t* n_out) {
  cq::clear_error();
  if (!plan || !n_out) return cq::set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  cq::NormFilter nf;
  const int rc = cq::normalize_filter(plan, &nf);
  if (rc != CQ_OK) return rc;
  const cq_plan& p = nf.plan;
  if (p.n_preds && !p.preds) return cq::set_error(CQ_ERR_INVALID_ARG, "plan array is NULL");
  *n_out = p.n_preds;
  if (p.n_preds > cap || (p.n_preds && !out))
    return cq::set_error(CQ_ERR_INVALID_ARG, "%u predicates do not fit the %u given", p.n_preds, cap);
  for (uint32_t i = 0; i < p.n_preds; ++i) out[i] = p.preds[i];
  return CQ_OK;
}
