"""The library's rewrite of filter programs to conjunctive form (host code,
no GPU): for random programs the form it returns is equivalent to the
program under every assignment of truth values to the predicates; the
simplifications and the errors are the documented ones."""
import itertools

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_tree

COUNT = [dg.Agg("count")]


@pytest.fixture(scope="module")
def cq():
    from paper_2506_10092_gb300 import cq as _cq
    return _cq


def preds(k, neg=()):
    # distinguishable predicates: the literal is the index
    return [dg.Pred(0, "lt", i, neg=i in neg) for i in range(k)]


def program_value(prog, truth, negs):
    st = []
    for kind, arg in prog:
        if kind == "pred":
            st.append(truth[arg] != negs[arg])
        elif kind == "not":
            st.append(not st.pop())
        else:
            top = [st.pop() for _ in range(arg)]
            st.append(all(top) if kind == "and" else any(top))
    assert len(st) == 1
    return st[0]


def cnf_value(form, truth):
    clauses = {}
    for idx, g, ng in form:
        lit = truth[idx] != bool(ng)
        if g == 0:
            if not lit:
                return False
        else:
            clauses[g] = clauses.get(g, False) or lit
    return all(clauses.values())


@pytest.mark.parametrize("seed", range(60))
def test_random_programs_are_equivalent(cq, seed):
    rng = np.random.default_rng(8000 + seed)
    k = int(rng.integers(1, 6))
    negs = [bool(rng.random() < 0.3) for _ in range(k)]
    prog = random_tree(rng, k, max_depth=int(rng.integers(1, 4)))
    plan = dg.Plan(preds(k, [i for i in range(k) if negs[i]]), [], COUNT, filter=prog)
    try:
        form = cq.cq_filter_conjunctive(plan)
    except cq.CQError as e:
        assert e.status == cq.CQ_ERR_UNSUPPORTED        # more than 16 occurrences
        return
    assert len(form) <= 16
    for truth in itertools.product([False, True], repeat=k):
        assert cnf_value(form, truth) == program_value(prog, truth, negs), (prog, form, truth)
    # no clause repeats a predicate, none is a single-member group
    groups = {}
    for idx, g, _ in form:
        if g:
            groups.setdefault(g, []).append(idx)
    for members in groups.values():
        assert len(members) >= 2 and len(set(members)) == len(members)


def test_simplifications(cq):
    P = preds(3)
    f = lambda prog: sorted(cq.cq_filter_conjunctive(dg.Plan(P, [], COUNT, filter=prog)))
    # De Morgan: NOT (a AND b) is one clause of complements; NOT (a OR b) two
    assert f([("pred", 0), ("pred", 1), ("and", 2), ("not", 0)]) == [(0, 1, 1), (1, 1, 1)]
    assert f([("pred", 0), ("pred", 1), ("or", 2), ("not", 0)]) == [(0, 0, 1), (1, 0, 1)]
    # double negation, one-operand AND / OR
    assert f([("pred", 2), ("not", 0), ("not", 0)]) == [(2, 0, 0)]
    assert f([("pred", 2), ("and", 1), ("or", 1)]) == [(2, 0, 0)]
    # a OR NOT a always holds: no predicate left
    assert f([("pred", 0), ("pred", 0), ("not", 0), ("or", 2)]) == []
    # absorption: a AND (a OR b) is a
    assert f([("pred", 0), ("pred", 0), ("pred", 1), ("or", 2), ("and", 2)]) == [(0, 0, 0)]
    # a repeated literal and a repeated clause are kept once
    assert f([("pred", 1), ("pred", 1), ("or", 2), ("pred", 1), ("and", 2)]) == [(1, 0, 0)]
    # distribution: a OR (b AND c) = (a OR b) AND (a OR c)
    assert f([("pred", 0), ("pred", 1), ("pred", 2), ("and", 2), ("or", 2)]) == [(0, 1, 0), (0, 2, 0), (1, 1, 0),
                                                                                (2, 2, 0)]
    # a predicate's own negate flag and a NOT node cancel
    Pn = preds(2, neg=[1])
    assert sorted(cq.cq_filter_conjunctive(dg.Plan(Pn, [], COUNT, filter=[("pred", 1), ("not", 0)]))) == [(1, 0, 0)]


def test_conjunctive_plans_pass_through(cq):
    P = [dg.Pred(0, "lt", 0, group=3), dg.Pred(0, "lt", 1, neg=True), dg.Pred(0, "lt", 2, group=3, neg=True)]
    assert cq.cq_filter_conjunctive(dg.Plan(P, [], COUNT)) == [(0, 3, 0), (1, 0, 1), (2, 3, 1)]


def test_growth_beyond_sixteen_occurrences_is_unsupported(cq):
    # (a1 AND b1) OR ... OR (a5 AND b5): 2^5 clauses of 5 literals
    prog = []
    for i in range(5):
        prog += [("pred", 2 * i), ("pred", 2 * i + 1), ("and", 2)]
    prog.append(("or", 5))
    with pytest.raises(cq.CQError) as e:
        cq.cq_filter_conjunctive(dg.Plan(preds(10), [], COUNT, filter=prog))
    assert e.value.status == cq.CQ_ERR_UNSUPPORTED


@pytest.mark.parametrize("prog,group", [
    ([("and", 2)], 0),
    ([("not", 0)], 0),
    ([("pred", 0), ("pred", 1)], 0),
    ([("pred", 7)], 0),
    ([("pred", 0), ("or", 0)], 0),
    ([("pred", 0), ("pred", 1), ("and", 3)], 0),
    ([("pred", 0)], 5),
    ([("pred", 0)] + [("not", 0)] * 64, 0),          # more than 64 nodes
])
def test_malformed_programs_are_rejected(cq, prog, group):
    P = preds(2)
    P[0].group = group
    with pytest.raises(cq.CQError) as e:
        cq.cq_filter_conjunctive(dg.Plan(P, [], COUNT, filter=prog))
    assert e.value.status == cq.CQ_ERR_INVALID_ARG


def test_bad_node_kind_is_rejected(cq):
    from paper_2506_10092_gb300.cq import PlanStruct, cq_filter_node, lib
    import ctypes as C
    ps = PlanStruct(dg.Plan(preds(1), [], COUNT, filter=[("pred", 0)]))
    bad = (cq_filter_node * 1)(cq_filter_node(9, 0))
    ps.s.filter, ps.s.n_filter = C.addressof(bad), 1
    n = C.c_uint32()
    assert lib.cq_filter_conjunctive(C.byref(ps.s), None, 0, C.byref(n)) == cq.CQ_ERR_INVALID_ARG
