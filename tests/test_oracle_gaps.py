"""Pins for the oracle's near-tie record (the per-query smallest relative gap of a deciding
comparison).  The record decides which queries a GPU run in FP32 may legitimately resolve
differently from the FP64 oracle, so it is pinned three ways:

* hand traces: on tiny graphs traced by hand (Section 2's search, the batched form, Section
  4.1's shortlist, Section 4.3's re-rank), the oracle lists exactly the deciding comparisons
  the trace makes, in order, with their kind;
* planted near-ties on a one-dimensional geometry (each node's walk distance is the square
  of one float32 value, exact in float64): a pair 1 ulp apart placed so that exactly one
  comparison of a given kind sees it gives exactly that pair's relative gap; a pair that
  only sits side by side in the result set (never compared in a deciding way) leaves the
  record unchanged; the walk-only record ignores the output order;
* completeness: perturbing every node's distance by less than an eighth of the recorded gap
  leaves every returned id and every visit count unchanged (a deciding comparison missing
  from the record would let such a perturbation change the result).
"""
import numpy as np
import pytest

import oracle
from oracle import refine
from test_oracle_search import ADJ, CODES, Q0, integer_index, tiny_index

WALK_KINDS = {"upper_second", "upper_move", "runner", "outside", "break", "end", "batch_next",
              "batch_outside", "batch_end", "shortlist"}


def rel(a, b):
    return abs(a - b) / max(abs(a), abs(b))


# ------------------------------------------------------------------------------------------
# hand traces
def test_trace_plain_walk():
    # The walk of test_oracle_search.test_hand_traced_level0_walk at ef = 2 (distances 0:18,
    # 1:13, 2:10, 3:2, 4:4, 5:32).  Expand 0 (nothing to compare): 1 and 2 enter W, 0 is
    # evicted (best outside: 0), 5 rejected.  Pop 2 against runner-up 1, and against the best
    # outside 0; 4 enters and evicts 1 (best outside: 1).  Pop 4 against 1 / 1; 3 enters,
    # evicts 2 (best outside: 2).  Pop 3 against 1 / 2.  Pop 1: further than the worst of W
    # (4): the walk breaks; at the end the worst of W (4) against the best outside (2).
    # Output: 3 against 4.
    ix = tiny_index(CODES, ADJ)
    r, tr = oracle.trace(lambda: oracle.search(ix, Q0, k=1, ef=2, shortlist=-1))
    assert tr == [("runner", 2, 1), ("outside", 2, 0), ("runner", 4, 1), ("outside", 4, 1),
                  ("runner", 3, 1), ("outside", 3, 2), ("break", 4, 1), ("end", 4, 2), ("out_walk", 3, 4)]
    assert r["gap"][0] == 3 / 13 and r["gap_walk"][0] == 3 / 13       # 10 against 13
    assert r["next_dist"][0] == 4.0


def test_trace_upper_descent():
    # test_oracle_search.test_hand_traced_upper_descent: from 5 move to 0 (only neighbour),
    # at 0 the best neighbour 2 beats the runner-up 5 and the current node, at 2 the only
    # neighbour 0 does not beat it.  Level 0 from 2 (ef 2): pop 4 against 0 / 0, pop 3
    # against 0 / 2, pop 0 ends the walk against the worst of W (4), which then meets the
    # best outside (2); output 3 against 4 (k = 2 = |W|: nothing follows).
    ix = tiny_index(CODES, ADJ, upper={5: [0], 0: [5, 2], 2: [0]}, ep=5, max_level=1)
    r, tr = oracle.trace(lambda: oracle.search(ix, Q0, k=2, ef=2, shortlist=-1))
    assert tr == [("upper_move", 0, 5), ("upper_second", 2, 5), ("upper_move", 2, 0),
                  ("upper_move", 0, 2), ("runner", 4, 0), ("outside", 4, 0), ("runner", 3, 0),
                  ("outside", 3, 2), ("break", 4, 0), ("end", 4, 2), ("out_walk", 3, 4)]
    assert np.isinf(r["next_dist"][0])


def test_trace_batched_walk():
    # Batched form, beam 2, ef 2.  Step 1 takes 0 alone; 1, 2, 5 are scored, W = {2, 1},
    # best outside 0 (18).  Step 2 takes 2 and 1 (the last taken, 1, against the best outside
    # 0; nothing unexpanded follows it); 4 and 3 are scored, W = {3, 4}, best outside 2.
    # Step 3 takes 3 and 4 (4 against 2); nothing new.  End: the worst of W (4) against 2.
    ix = tiny_index(CODES, ADJ)
    r, tr = oracle.trace(lambda: oracle.search(ix, Q0, k=1, ef=2, shortlist=-1, beam=2))
    assert tr == [("batch_outside", 1, 0), ("batch_outside", 4, 2), ("batch_end", 4, 2),
                  ("out_walk", 3, 4)]
    assert r["stats"][0].tolist() == [6, 5, 0]


def test_trace_batched_next_unexpanded():
    # Batched form, beam 2, ef 4.  Step 1 takes 0; W = {2 (10), 1 (13), 0 (18, expanded),
    # 5 (32)}.  Step 2 takes 2 and 1: the last taken (1) against the next unexpanded member
    # (5); no node is outside W yet.  4 and 3 enter: W = {3, 4, 2, 1}, best outside 0 (18).
    # Step 3 takes 3 and 4: no unexpanded member follows; 4 against the best outside 0.  End:
    # the worst of W (1) against 0.
    ix = tiny_index(CODES, ADJ)
    r, tr = oracle.trace(lambda: oracle.search(ix, Q0, k=1, ef=4, shortlist=-1, beam=2))
    assert tr == [("batch_next", 1, 5), ("batch_outside", 4, 0), ("batch_end", 1, 0), ("out_walk", 3, 4)]


def test_trace_shortlist_and_refined_output():
    # W = {3 (2), 4 (4)} as in test_trace_plain_walk; node 3 refines to 6.25 (codeword 1),
    # node 4 keeps 4.  shortlist 1, k = 1: the shortlist boundary 3 | 4 is compared, one
    # candidate is refined, nothing follows it.  shortlist 0, k = 2: both refined, the
    # output order 4 | 3 is compared on refined distances.
    B = np.tile(refine.e0(), (256, 1))
    B[1, :2] = 0.5
    beta = np.zeros(6, np.uint8)
    beta[3] = 1
    ix = tiny_index(CODES, ADJ, beta=beta, B=B)
    r, tr = oracle.trace(lambda: oracle.search(ix, Q0, k=1, ef=2, shortlist=1))
    assert tr[-1] == ("shortlist", 3, 4) and all(t[0] != "out_refined" for t in tr)
    assert r["ids"][0].tolist() == [3] and r["gap"][0] == r["gap_walk"][0]
    r, tr = oracle.trace(lambda: oracle.search(ix, Q0, k=2, ef=2, shortlist=0))
    assert tr[-1] == ("out_refined", 4, 3) and all(t[0] != "shortlist" for t in tr)
    assert r["ids"][0].tolist() == [4, 3]
    # the output order decides only gap, not gap_walk
    assert r["gap"][0] == min(r["gap_walk"][0], rel(4.0, 6.25))


def test_gap_is_the_minimum_over_the_traced_comparisons(rng):
    # On random integer-geometry indexes (exact distances), the two recorded minima are
    # the relative gaps of the traced comparisons folded by hand: identical code rows are
    # skipped, any other exact tie counts as 0, the walk record covers kinds 1-10 only.
    for trial in range(20):
        ix = integer_index(rng)
        Q = rng.integers(-8, 9, size=(30, 4)).astype(np.float32)
        xh1 = ix.C1.astype(np.float64)[ix.codes1.astype(np.int64), np.arange(4)]
        beam = [1, 2, 4][trial % 3]
        for q in range(30):
            r, tr = oracle.trace(lambda: oracle.search(ix, Q[q:q + 1], k=3, ef=[2, 5, 9][q % 3], shortlist=-1,
                                                       beam=beam))
            d = lambda e: float(((Q[q] - xh1[e]) ** 2).sum())
            g, gw = np.inf, np.inf
            for kind, a, b in tr:
                if d(a) == d(b):
                    if np.array_equal(ix.codes1[a], ix.codes1[b]):
                        continue
                    x = 0.0
                else:
                    x = rel(d(a), d(b))
                g = min(g, x)
                if kind in WALK_KINDS:
                    gw = min(gw, x)
            assert r["gap"][0] == g and r["gap_walk"][0] == gw


# ------------------------------------------------------------------------------------------
# planted near-ties on a line: node i has code i and walk distance vals[i]^2 (query at 0)
A = np.float32(30.0)
A1 = np.nextafter(A, np.float32(31.0))            # 1 ulp above: distances 900 and A1^2
NEAR = rel(float(A) ** 2, float(A1) ** 2)


def line_index(vals, adj, upper=None, ep=0, max_level=0):
    N = len(vals)
    C1 = np.zeros((256, 1), np.float32)
    C1[:N, 0] = vals
    adj = [list(r) + [-1] * (6 - len(r)) for r in adj]
    return tiny_index(np.arange(N)[:, None], adj, upper=upper, ep=ep, max_level=max_level, d=1, M1=1, M2=1,
                      C1=C1)


QL = np.zeros((1, 1), np.float32)
S, T = np.float32(50.0), np.float32(1.0)           # a far seed (2500) and a near target (1)

# (name, values, adjacency, search kwargs, kind expected to see the planted pair, the pair)
PLANTED = [
    # s -> a, b: popping a, b is the runner-up in C; a leads to t
    ("runner", [S, A, A1, T], [[1, 2], [3], [], []], dict(k=1, ef=8), "runner", (1, 2)),
    # ef 1: a enters W, b is the best outside when a is expanded; t then evicts a
    ("outside", [S, A, A1, T], [[1, 2], [3], [], []], dict(k=1, ef=1), "outside", (1, 2)),
    # ef 2: f is expanded while c is still in W; t evicts c; popping c ends the walk against f,
    # and c is then the best node outside W, met by the worst inside (f) at the end
    ("break", [S, A, A1, T], [[1], [2, 3], [], []], dict(k=1, ef=2), ("break", "end"), (1, 2)),
    # ef 1: C runs empty with a in W and b the best node left out
    ("end", [S, A, A1], [[1], [2], []], dict(k=1, ef=1), "end", (1, 2)),
    # beam 2, ef 4: step 2 takes t1 and a; b is the next unexpanded member
    ("batch_next", [S, np.float32(10.0), A, A1], [[1, 2, 3], [], [], []], dict(k=1, ef=4, beam=2),
     "batch_next", (2, 3)),
    # beam 2, ef 1: a is taken with b the best outside; t then evicts a
    ("batch_outside", [S, A, A1, T], [[1, 2], [3], [], []], dict(k=1, ef=1, beam=2), "batch_outside", (1, 2)),
    # beam 2, ef 1: a's expansion scores b, which stays outside; nothing is left to take
    ("batch_end", [S, A, A1], [[1], [2], []], dict(k=1, ef=1, beam=2), "batch_end", (1, 2)),
    # W = t, a, b, s: with a shortlist of 2 the boundary is a | b
    ("shortlist", [S, A, A1, T], [[1], [2, 3], [], []], dict(k=1, ef=8, shortlist=2), "shortlist", (1, 2)),
    # no refinement, k = 2: the 2nd returned (a) against the 3rd (b)
    ("out_walk", [S, A, A1, T], [[1], [2, 3], [], []], dict(k=2, ef=8, shortlist=-1), "out_walk", (1, 2)),
    # refinement with e0 codewords (refined = walk distance), k = 2: a | b on refined distances
    ("out_refined", [S, A, A1, T], [[1], [2, 3], [], []], dict(k=2, ef=8, shortlist=0), "out_refined", (1, 2)),
]


@pytest.mark.parametrize("name,vals,adj,kw,kind,pair", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_near_tie(name, vals, adj, kw, kind, pair):
    ix = line_index(vals, adj)
    kw = dict(kw)
    kw.setdefault("shortlist", -1)
    r, tr = oracle.trace(lambda: oracle.search(ix, QL, **kw))
    kinds = {kind} if isinstance(kind, str) else set(kind)
    seen = [t for t in tr if set(t[1:]) == set(pair)]
    assert seen and {t[0] for t in seen} == kinds, tr
    assert r["gap"][0] == NEAR
    if kinds <= WALK_KINDS:
        assert r["gap_walk"][0] == NEAR
    else:
        assert r["gap_walk"][0] > 1e-3           # the walk itself is decided clearly


def test_planted_upper_level_near_ties():
    # level 1: e (ep) -> a, b: the best neighbour a against the runner-up b; a then against e
    vals = [S, A, A1, T]
    ix = line_index(vals, [[], [3], [], []], upper={0: [1, 2], 1: [0], 2: [0]}, ep=0, max_level=1)
    r, tr = oracle.trace(lambda: oracle.search(ix, QL, k=1, ef=8, shortlist=-1))
    assert [t for t in tr if set(t[1:]) == {1, 2}] == [("upper_second", 1, 2)]
    assert r["gap"][0] == NEAR and r["gap_walk"][0] == NEAR
    # level 1: e (ep, A1) -> a (A): the move from e to a is decided by the planted pair
    ix = line_index([A1, A, T], [[], [2], []], upper={0: [1], 1: [0]}, ep=0, max_level=1)
    r, tr = oracle.trace(lambda: oracle.search(ix, QL, k=1, ef=8, shortlist=-1))
    assert {t[0] for t in tr if set(t[1:]) == {0, 1}} == {"upper_move"}
    assert r["gap"][0] == NEAR and r["ids"][0].tolist() == [2]


def test_near_tie_that_decides_nothing_leaves_the_record_unchanged():
    # s -> a -> b -> t, ef 8: a and b (1 ulp apart) end up side by side in W, but C never
    # holds both, nothing is evicted, and only t | a is output: the record is t against a
    ix = line_index([S, A, A1, T], [[1], [2], [3], []])
    r, tr = oracle.trace(lambda: oracle.search(ix, QL, k=1, ef=8, shortlist=-1, return_w=True))
    assert r["w_ids"][0, :4].tolist() == [3, 1, 2, 0]
    assert tr == [("out_walk", 3, 1)]
    assert r["gap"][0] == rel(1.0, 900.0) and r["gap_walk"][0] == np.inf
    # batched: a and b taken in the same step are not compared with each other
    ix = line_index([S, A, A1, T], [[1, 2], [3], [], []])
    r, tr = oracle.trace(lambda: oracle.search(ix, QL, k=1, ef=8, shortlist=-1, beam=2))
    assert all(set(t[1:]) != {1, 2} for t in tr)
    assert r["gap"][0] == rel(1.0, 900.0)


def test_exact_tie_of_different_code_rows_is_unresolved():
    # two nodes at exactly the same distance with different codes (+30 and -30 on the line):
    # identical only by arithmetic, so the record is 0 (identical code rows are exempt,
    # test_oracle_search.test_ties_broken_by_smaller_id)
    ix = line_index([S, A, -A, T], [[1, 2], [3], [], []])
    r = oracle.search(ix, QL, k=1, ef=8, shortlist=-1)
    assert r["gap"][0] == 0.0


# ------------------------------------------------------------------------------------------
# completeness: perturbations below the recorded gap change nothing
def random_line_index(rng):
    N = int(rng.integers(20, 200))
    vals = np.sort(rng.uniform(1.0, 2.0, N)).astype(np.float32)
    vals = rng.permutation(np.unique(vals))
    N = len(vals)
    deg = 6
    adj = np.full((N, deg), -1, np.int32)
    for i in range(N):
        k = rng.integers(1, deg + 1)
        adj[i, :k] = rng.choice(np.delete(np.arange(N), i), size=k, replace=False)
    up = rng.choice(N, size=10, replace=False)
    upper = {int(v): list(rng.choice(np.setdiff1d(up, [v]), size=3, replace=False)) for v in up}
    C1 = np.zeros((256, 1), np.float32)
    C1[:N, 0] = vals
    ix = tiny_index(np.arange(N)[:, None], adj, upper=upper, ep=int(up[0]), max_level=1, d=1, M1=1, M2=1, C1=C1)
    return ix, vals


@pytest.mark.parametrize("beam", [1, 2, 4])
def test_perturbation_below_the_gap_changes_nothing(rng, beam):
    checked = 0
    for trial in range(2500):
        ix, vals = random_line_index(rng)
        kw = dict(k=int(rng.choice([1, 3, 8])), ef=int(rng.choice([1, 2, 4, 8, 16])),
                  shortlist=int(rng.choice([-1, 0, 2])), beam=beam, tcap=int(rng.choice([0, 0, 25])))
        r = oracle.search(ix, QL, **kw)
        g = r["gap"][0]
        if not g > 1e-4:
            continue
        eps = g / 8
        eta = rng.uniform(-eps, eps, len(vals))
        pv = (vals.astype(np.float64) * np.sqrt(1.0 + eta)).astype(np.float32)
        # every node's distance moved by less than g/8 relative (rounding included)
        assert np.all(np.abs(pv.astype(np.float64) ** 2 / vals.astype(np.float64) ** 2 - 1) < eps + 1e-6)
        ix.C1[:len(vals), 0] = pv
        p = oracle.search(ix, QL, **kw)
        assert np.array_equal(p["ids"], r["ids"]), (trial, kw)
        assert np.array_equal(p["stats"], r["stats"]), (trial, kw)
        checked += 1
    assert checked > 1200
