"""Pins of the oracle's Leiden form (oracle.refine, oracle.louvain with
refine=True), CPU only.

The refinement (Traag, Waltman and van Eck 2019; the paper's Sec. 5.2 and
Sec. 6 expect its findings to extend to Leiden) is greedy and bucketed here:
a vertex that is still a singleton and well connected to its community C of
P merges into the refined community inside C with the largest exact
modularity gain, if that gain is positive; a vertex that any decision of the
bucket chose as its target stays.  The pins check it against what
modularity itself fixes (exact gains from oracle.modularity, which is pinned
against networkx), against properties that hold by construction
(containment in P, connected refined communities, the well-connectedness
condition of every vertex that moved) and against the invariance of
modularity under aggregation; the whole-run pins of the Louvain form are
repeated with refinement on.
"""
import os
from collections import deque
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2501_19004_gb300 import graphgen as gg

from test_oracle_pins import (GOLDEN, csr_from_dense, exact_q, plain_q_dense, random_graph,  # noqa: F401
                              set_partitions)

LEIDEN = oracle.Config(refine=True)


def dense_of(g):
    n = g.n
    W = np.zeros((n, n), dtype=np.int64)
    w = np.ones(g.nnz, dtype=np.int64) if g.weights is None else g.weights.astype(np.int64)
    for i in range(n):
        for k in range(int(g.offsets[i]), int(g.offsets[i + 1])):
            W[i, g.cols[k]] += w[k]
    return W


def well_connected(W, bound, v):
    """Leiden's condition for a vertex (modularity, resolution 1):
    w(v, C - v) >= K_v (Sigma_C - K_v) / 2m, with C = bound[v]."""
    K = W.sum(1)
    two_m = int(W.sum())
    C = np.nonzero(bound == bound[v])[0]
    inside = int(sum(W[v, u] for u in C if u != v))
    return two_m * inside >= int(K[v]) * (int(K[C].sum()) - int(K[v]))


def connected_within(W, members):
    members = set(int(x) for x in members)
    start = next(iter(members))
    seen, todo = {start}, deque([start])
    while todo:
        a = todo.popleft()
        for b in members:
            if b not in seen and W[a, b] > 0:
                seen.add(b)
                todo.append(b)
    return seen == members


def expected_sweep(g, W, bound, buckets=1, pass_=0, seed=0):
    """The refinement from its definition: bucket by bucket (the schedule's
    hash at iteration 255), every well-connected vertex that is still a
    singleton and was not chosen decides against the current refined
    partition R, by the exact gain Q(R with v joined to T) - Q(R) over the
    refined communities T of its neighbours inside its community of P
    (lowest T on ties, positive gains only); targets are marked chosen, and
    the other movers are applied."""
    n = g.n
    R = np.arange(n, dtype=np.int32)
    chosen = np.zeros(n, dtype=bool)
    bk = np.array([oracle.bucket(v, pass_, 255, seed, buckets) for v in range(n)])
    elig = [well_connected(W, bound, v) for v in range(n)]
    for b in range(buckets):
        q0 = exact_q(g, R)
        target = {}
        for v in range(n):
            if bk[v] != b or not elig[v] or chosen[v]:
                continue
            best, best_t = None, None
            for T in sorted({int(R[u]) for u in range(n) if u != v and W[v, u] > 0 and bound[u] == bound[v]}):
                m = R.copy()
                m[v] = T
                gain = exact_q(g, m) - q0
                if best is None or gain > best:
                    best, best_t = gain, T
            if best is not None and best > 0:
                target[v] = best_t
        for t in target.values():
            chosen[t] = True
        for v, t in target.items():
            if not chosen[v]:
                R[v] = t
    return R


def random_bound(rng, n, groups):
    return rng.integers(0, groups, size=n).astype(np.int32)


# ------------------------------------------------------ the refinement step
@pytest.mark.parametrize("buckets", [1, 3, 4])
def test_refine_is_the_definition(buckets):
    rng = np.random.default_rng(71 + buckets)
    cases = 0
    for trial in range(40):
        n = int(rng.integers(5, 14))
        W = random_graph(rng, n, p=0.5, wmax=4, self_loops=bool(trial % 3 == 0))
        g = csr_from_dense(W)
        bound = random_bound(rng, n, int(rng.integers(1, 4)))
        pass_ = int(rng.integers(0, 3))
        got = oracle.refine(g, bound, pass_=pass_, seed=trial, buckets=buckets)
        want = expected_sweep(g, W, bound, buckets, pass_, trial)
        assert np.array_equal(got, want), (trial, got, want)
        cases += int((got != np.arange(n)).any())
    assert cases >= 20  # most cases merge something, so the comparison bites


def test_refine_ties_go_to_the_lowest_id():
    # a star inside one community: every leaf's only candidate is the hub,
    # and the hub sees equal gains to every leaf and takes leaf 1
    n = 6
    W = np.zeros((n, n), dtype=np.int64)
    for leaf in range(1, n):
        W[0, leaf] = W[leaf, 0] = 1
    g = csr_from_dense(W)
    got = oracle.refine(g, np.zeros(n, dtype=np.int32), buckets=1)
    # the hub chose leaf 1, the leaves chose the hub: both stay, leaves 2..5 join the hub
    assert list(got) == [0, 1, 0, 0, 0, 0]


def test_refine_invariants_with_buckets():
    rng = np.random.default_rng(5)
    graphs = [gg.sbm(300, 30, 0.3, 0.02, seed=2), gg.rmat(9, 8, seed=4), gg.grid(20, 0.05, seed=1)]
    for g in graphs:
        W = dense_of(g)
        for bound in (oracle.louvain(g, oracle.Config(max_passes=1)).membership,
                      random_bound(rng, g.n, 3), np.zeros(g.n, dtype=np.int32)):
            bound = np.asarray(bound, dtype=np.int32)
            for B in (1, 4, 7):
                ref = oracle.refine(g, bound, pass_=1, buckets=B)
                assert np.array_equal(ref[ref], ref)                  # every id is a member (its seed)
                assert np.array_equal(bound[ref], bound)              # refined communities lie inside P
                for s in np.unique(ref):
                    assert connected_within(W, np.nonzero(ref == s)[0])
                for v in np.nonzero(ref != np.arange(g.n))[0]:
                    assert well_connected(W, bound, v)
                assert np.unique(ref).size >= np.unique(bound).size


def test_refine_special_cases():
    g = gg.rmat(8, 8, seed=2)
    n = g.n
    assert np.array_equal(oracle.refine(g, np.arange(n, dtype=np.int32)), np.arange(n))   # nothing to merge
    # two disjoint cliques, one community each: every member merges
    W = np.zeros((10, 10), dtype=np.int64)
    for blk in (range(0, 5), range(5, 10)):
        for a in blk:
            for b in blk:
                if a != b:
                    W[a, b] = 1
    gc = csr_from_dense(W)
    ref = oracle.refine(gc, np.array([0] * 5 + [5] * 5, dtype=np.int32), buckets=4)
    assert np.unique(ref[:5]).size <= 2 and np.unique(ref[5:]).size <= 2
    assert set(ref[:5]).isdisjoint(set(ref[5:]))


def test_aggregating_a_refinement_keeps_the_partition_q():
    rng = np.random.default_rng(9)
    for g in (gg.sbm(400, 40, 0.25, 0.02, seed=3), gg.rmat(10, 8, seed=6)):
        for bound in (oracle.louvain(g, oracle.Config(max_passes=1)).membership, random_bound(rng, g.n, 4)):
            bound = np.asarray(bound, dtype=np.int32)
            ref = oracle.refine(g, bound, buckets=4)
            ids, dense = np.unique(ref, return_inverse=True)
            off, col, w = oracle.aggregate(g, dense.astype(np.int32), ids.size)
            h = gg.CSR(off, col, w.astype(np.int32), "super")
            # each super-vertex starts in its community of P
            rep = {}
            for v in range(g.n):
                rep[bound[v]] = min(rep.get(bound[v], 1 << 40), int(dense[v]))
            init = np.empty(ids.size, dtype=np.int32)
            for v in range(g.n):
                init[dense[v]] = rep[bound[v]]
            assert exact_q(h, init) == exact_q(g, bound)


# ------------------------------------------------------------ whole runs
@pytest.mark.parametrize("B", [1, 4])
def test_whole_run_refines_over_four_times_the_buckets(B):
    """A whole run refines each pass's P in one sweep over 4B buckets: the
    second pass's n' is the number of refined communities of that sweep
    (and not of a sweep over B buckets, which differs on every graph
    here)."""
    for g in (gg.rmat(12, 16, seed=7), gg.sbm(400, 40, 0.25, 0.02, seed=3), gg.grid(48, 0.02, seed=5),
              gg.rmat(11, 8, seed=3, weight_range=(1, 5))):
        P = oracle.louvain(g, oracle.Config(refine=True, max_passes=1, buckets=B)).membership  # the pass cap gives P
        r = oracle.louvain(g, oracle.Config(refine=True, max_passes=2, buckets=B))
        assert r.passes == 2
        n1 = int(r.pass_stats[1][0])
        assert np.unique(oracle.refine(g, P, pass_=0, buckets=4 * B)).size == n1
        assert np.unique(oracle.refine(g, P, pass_=0, buckets=B)).size != n1


@pytest.mark.parametrize("B", [1, 4])
def test_next_pass_starts_from_p(B):
    """Disjoint cliques: pass 0 finds the cliques (P) and the refinement
    splits some of them into pieces.  The next pass starts every piece in
    its clique's community of P, which is already optimal, so its first
    iteration moves nothing and the run converges there; from singletons the
    pieces of a clique would have to move together again."""
    split = 0
    for sizes in ((5, 5), (6, 7, 8), (12, 12, 12, 12)):
        n = sum(sizes)
        W = np.zeros((n, n), dtype=np.int64)
        o = 0
        for k in sizes:
            W[o:o + k, o:o + k] = 1
            o += k
        np.fill_diagonal(W, 0)
        r = oracle.louvain(csr_from_dense(W), oracle.Config(refine=True, buckets=B))
        assert r.passes == 2 and r.communities == len(sizes)
        assert r.iter_stats[1][0][1] == 0 and r.pass_stats[1][2] == 1
        split += int(r.pass_stats[1][0] > len(sizes))  # more pieces than cliques
    assert split >= 1


def test_leiden_two_disjoint_cliques():
    W = np.zeros((10, 10), dtype=np.int64)
    for blk in (range(0, 5), range(5, 10)):
        for a in blk:
            for b in blk:
                if a != b:
                    W[a, b] = 1
    r = oracle.louvain(csr_from_dense(W), oracle.Config(refine=True, check_invariants=True))
    assert list(r.membership) == [0] * 5 + [1] * 5


def test_leiden_ring_of_cliques_reaches_closed_form():
    rows = [line.split() for line in open(os.path.join(GOLDEN, "ring_of_cliques.txt")) if line[0] != "#"]
    for r_, k, m, qn, qd in [tuple(map(int, x)) for x in rows]:
        g = gg.ring_of_cliques(r_, k)
        res = oracle.louvain(g, oracle.Config(refine=True, check_invariants=True))
        assert Fraction(res.q_num, res.q_den) == Fraction(qn, qd), (r_, k)
        assert np.array_equal(res.membership, np.arange(r_ * k) // k)


def test_leiden_bounded_by_brute_force_optimum():
    rng = np.random.default_rng(17)
    for trial in range(8):
        n = int(rng.integers(4, 9))
        W = random_graph(rng, n, p=0.45, wmax=4)
        g = csr_from_dense(W)
        best = max(plain_q_dense(W, np.array(p)) for p in set_partitions(n))
        res = oracle.louvain(g, oracle.Config(refine=True, check_invariants=True))
        assert res.modularity <= best + 1e-12
        assert abs(res.modularity - plain_q_dense(W, res.membership)) < 1e-12
        assert res.modularity >= plain_q_dense(W, np.arange(n)) - 1e-12


def test_leiden_karate_club_below_published_optimum():
    nx = pytest.importorskip("networkx")
    q_opt = float(open(os.path.join(GOLDEN, "karate_club.txt")).read().split("q_opt")[1].split()[0])
    G = nx.karate_club_graph()
    u, v = zip(*G.edges())
    res = oracle.louvain(gg.from_pairs(34, u, v), LEIDEN)
    assert 0.38 < res.modularity <= q_opt + 1e-7


@pytest.mark.parametrize("make", [lambda: gg.sbm(1000, 100, 0.1, 0.002, seed=1), lambda: gg.rmat(12, 16, seed=7),
                                  lambda: gg.grid(64, 0.02, seed=5)])
def test_leiden_invariants_and_monotone_q(make):
    """Sigma' sums to 2m after every bucket; every pass starts from the
    previous pass's P, whose modularity the aggregation keeps, so the
    per-pass modularity never decreases and the last one is the final Q."""
    g = make()
    res = oracle.louvain(g, oracle.Config(refine=True, check_invariants=True))
    ps = res.pass_stats[:res.passes]
    qs = [Fraction((int(r[4]) << 64) + (int(r[5]) & (2**64 - 1)), res.two_m ** 2) for r in ps]
    assert all(b >= a for a, b in zip(qs, qs[1:])), qs
    assert qs[-1] == Fraction(res.q_num, res.q_den)
    _, num, den = oracle.modularity(g, res.membership)
    assert (num, den) == (res.q_num, res.q_den)
    used = np.unique(res.membership)
    assert used[0] == 0 and used[-1] == res.communities - 1


def test_leiden_planted_partition_recovered():
    g = gg.sbm(1000, 100, 0.1, 0.002, seed=1)
    res = oracle.louvain(g, LEIDEN)
    # at least 9 of the 10 blocks recovered by majority, as for the Louvain form
    blocks = np.arange(1000) // 100
    hits = 0
    for b in range(10):
        vals, cnt = np.unique(res.membership[blocks == b], return_counts=True)
        hits += cnt.max() >= 90
    assert hits >= 9


def test_leiden_independent_of_thread_count():
    g = gg.rmat(12, 16, seed=3)
    a = oracle.louvain(g, oracle.Config(refine=True, num_threads=1))
    b = oracle.louvain(g, oracle.Config(refine=True, num_threads=4))
    assert np.array_equal(a.membership, b.membership)
    assert np.array_equal(a.pass_stats, b.pass_stats) and np.array_equal(a.iter_stats, b.iter_stats)


def test_leiden_pass_cap_returns_p_not_its_refinement():
    """With the pass cap reached after an aggregation, the memberships are
    the last pass's P (each super-vertex's community), not the refined
    super-vertices."""
    g = gg.rmat(11, 16, seed=5)
    one = oracle.louvain(g, oracle.Config(refine=True, max_passes=1))
    assert one.passes == 1
    first = oracle.louvain(g, oracle.Config(max_passes=1))  # pass 0 of both forms is the same local moving
    assert one.communities == int(first.pass_stats[0, 3])
    _, num, den = oracle.modularity(g, one.membership)
    q_pass = (int(first.pass_stats[0, 4]) << 64) + (int(first.pass_stats[0, 5]) & (2**64 - 1))
    assert Fraction(num, den) == Fraction(q_pass, first.two_m ** 2)
