"""Pins of the CPU oracle against facts the paper and mathematics fix.

Each group below pins one oracle function to something other than itself:
a library routine (networkx modularity), exact rational arithmetic on every
possible move, brute-force enumeration of partitions, closed forms (ring of
cliques, disjoint cliques, singletons, one community), published hash
vectors, and invariants of the method (Sigma sums, modularity invariance
under aggregation).  A plausible mistake in the oracle -- a dropped self-loop
term, a sign error in Eq. 2, a wrong tie rule, a transposed aggregation --
fails at least one of them.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2501_19004_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def csr_from_dense(W):
    """CSR (rows sorted) from a symmetric non-negative integer matrix; the
    diagonal entry, if any, is a self-loop stored once."""
    W = np.asarray(W, dtype=np.int64)
    n = W.shape[0]
    off = [0]
    cols, ws = [], []
    for i in range(n):
        for j in range(n):
            if W[i, j]:
                cols.append(j)
                ws.append(int(W[i, j]))
        off.append(len(cols))
    return gg.CSR(np.array(off, dtype=np.int64), np.array(cols, dtype=np.int32),
                  np.array(ws, dtype=np.int32), "dense")


def random_graph(rng, n, p=0.5, wmax=5, self_loops=False):
    W = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                W[i, j] = W[j, i] = rng.integers(1, wmax + 1)
        if self_loops and rng.random() < 0.3:
            W[i, i] = 2 * rng.integers(1, wmax + 1)
    if W.sum() == 0:
        W[0, 1] = W[1, 0] = 1
    return W


def exact_q(g, memb):
    _, num, den = oracle.modularity(g, memb)
    return Fraction(num, den)


def set_partitions(n):
    """All set partitions of range(n) as restricted growth strings."""
    a = [0] * n

    def rec(i, mx):
        if i == n:
            yield list(a)
            return
        for v in range(mx + 2):
            a[i] = v
            yield from rec(i + 1, max(mx, v))

    if n == 0:
        yield []
        return
    a[0] = 0
    yield from rec(1, 0)


def plain_q_dense(W, memb):
    """Textbook modularity of a dense symmetric matrix (self-loop stored once on the diagonal)."""
    W = np.asarray(W, dtype=np.float64)
    k = W.sum(1)
    two_m = W.sum()
    same = np.equal.outer(memb, memb)
    return float(((W - np.outer(k, k) / two_m) * same).sum() / two_m)


# ---------------------------------------------------- Eq. 1: modularity
def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(1)
    for trial in range(40):
        n = int(rng.integers(2, 25))
        W = random_graph(rng, n, p=0.3, wmax=7)
        g = csr_from_dense(W)
        memb = rng.integers(0, max(1, n // 3), size=n).astype(np.int32)
        q, _, _ = oracle.modularity(g, memb)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        for i in range(n):
            for j in range(i + 1, n):
                if W[i, j]:
                    G.add_edge(i, j, weight=int(W[i, j]))
        comms = [set(np.nonzero(memb == c)[0].tolist()) for c in np.unique(memb)]
        qn = nx.algorithms.community.modularity(G, comms, weight="weight")
        assert abs(q - qn) < 1e-12, (trial, q, qn)


def test_modularity_special_cases():
    rng = np.random.default_rng(2)
    for _ in range(10):
        n = int(rng.integers(3, 15))
        W = random_graph(rng, n, p=0.4)
        g = csr_from_dense(W)
        k = W.sum(1)
        two_m = int(W.sum())
        # one community: Q = 0 exactly
        assert exact_q(g, np.zeros(n, dtype=np.int32)) == 0
        # all singletons (no self-loops): Q = -sum K_i^2 / (2m)^2
        assert exact_q(g, np.arange(n, dtype=np.int32)) == Fraction(-int((k * k).sum()), two_m * two_m)


def test_modularity_ring_of_cliques_closed_form():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ring_of_cliques.txt")) if l[0] != "#"]
    for r, k, m, qn, qd in [tuple(map(int, x)) for x in rows]:
        g = gg.ring_of_cliques(r, k)
        assert g.nnz == 2 * m
        memb = (np.arange(r * k) // k).astype(np.int32)
        assert exact_q(g, memb) == Fraction(qn, qd)
        assert exact_q(g, memb) == 1 - Fraction(r, m) - Fraction(1, r)


# ------------------------------------------------ Eq. 2: delta-modularity
@pytest.mark.parametrize("self_loops", [False, True])
def test_delta_modularity_equals_exact_difference(self_loops):
    """2m^2 * dQ from Eq. 2 equals 2m^2 * (Q(after) - Q(before)) exactly, for
    every vertex and every target community, self-loops included."""
    rng = np.random.default_rng(3 + self_loops)
    for _ in range(12):
        n = int(rng.integers(2, 10))
        W = random_graph(rng, n, p=0.5, self_loops=self_loops)
        g = csr_from_dense(W)
        two_m = int(W.sum())
        two_m_sq = Fraction(two_m * two_m, 2)
        memb = rng.integers(0, n, size=n).astype(np.int32)
        q0 = exact_q(g, memb)
        for i in range(n):
            for c in range(n):
                after = memb.copy()
                after[i] = c
                want = (exact_q(g, after) - q0) * two_m_sq
                got = oracle.delta_modularity_scaled(g, memb, i, c)
                assert want == got, (i, c, want, got)


def test_delta_modularity_float_form_of_eq2():
    """Eq. 2 as printed, evaluated in floating point, agrees with the scaled
    integer form divided by 2m^2."""
    rng = np.random.default_rng(5)
    W = random_graph(rng, 9, p=0.6)
    g = csr_from_dense(W)
    n = 9
    memb = rng.integers(0, 4, size=n).astype(np.int32)
    two_m = W.sum()
    m = two_m / 2.0
    K = W.sum(1).astype(np.float64)
    Sig = np.zeros(n)
    for v in range(n):
        Sig[memb[v]] += K[v]
    for i in range(n):
        d = memb[i]
        for c in range(4):
            if c == d:
                continue
            K_ic = sum(W[i, j] for j in range(n) if j != i and memb[j] == c)
            K_id = sum(W[i, j] for j in range(n) if j != i and memb[j] == d)
            dq = (K_ic - K_id) / m - K[i] * (K[i] + Sig[c] - Sig[d]) / (2 * m * m)
            got = oracle.delta_modularity_scaled(g, memb, i, c) / (2 * m * m)
            assert abs(dq - got) < 1e-12


# -------------------------------------------- Algorithm 5 body: decisions
@pytest.mark.parametrize("pickless", [False, True])
def test_decide_is_brute_force_argmax(pickless):
    """The decision is the neighbour community with the largest exact
    modularity gain (lowest id among ties); a move needs a positive gain and,
    in Pick-Less mode, a target id below the current one."""
    rng = np.random.default_rng(7 + pickless)
    checked_moves = 0
    for _ in range(30):
        n = int(rng.integers(2, 10))
        W = random_graph(rng, n, p=0.5, wmax=3, self_loops=rng.random() < 0.5)
        g = csr_from_dense(W)
        two_m = int(W.sum())
        memb = rng.integers(0, n, size=n).astype(np.int32)
        q0 = exact_q(g, memb)
        for i in range(n):
            d = int(memb[i])
            cands = sorted({int(memb[j]) for j in range(n) if j != i and W[i, j]} - {d})
            best, best_c = None, None
            for c in cands:
                after = memb.copy()
                after[i] = c
                dq = exact_q(g, after) - q0
                if best is None or dq > best:
                    best, best_c = dq, c
            want_move = best is not None and best > 0 and not (pickless and best_c > d)
            moves, target, gain = oracle.decide(g, memb, i, pickless)
            assert moves == want_move, (i, memb, best, best_c)
            if moves:
                checked_moves += 1
                assert target == best_c
                assert Fraction(gain) == best * Fraction(two_m * two_m, 2)
    assert checked_moves > 10


def test_decide_tie_goes_to_lowest_id():
    # path 1 - 0 - 2 with symmetric neighbours: both moves of 0 gain the same
    W = np.zeros((5, 5), dtype=np.int64)
    for a, b in [(0, 1), (0, 2), (1, 3), (2, 4)]:
        W[a, b] = W[b, a] = 1
    g = csr_from_dense(W)
    memb = np.array([0, 3, 4, 3, 4], dtype=np.int32)
    moves, target, _ = oracle.decide(g, memb, 0)
    assert moves and target == 3
    memb = np.array([0, 4, 3, 4, 3], dtype=np.int32)
    moves, target, _ = oracle.decide(g, memb, 0)
    assert moves and target == 3


# ------------------------------------------- Algorithm 3 / 6: aggregation
def test_aggregate_matches_brute_force_and_preserves_q():
    rng = np.random.default_rng(11)
    for _ in range(20):
        n = int(rng.integers(2, 30))
        W = random_graph(rng, n, p=0.25, wmax=9, self_loops=rng.random() < 0.5)
        g = csr_from_dense(W)
        ncomm = int(rng.integers(1, n + 1))
        memb = rng.integers(0, ncomm, size=n).astype(np.int32)
        memb[:ncomm] = np.arange(ncomm)  # every community used
        rng.shuffle(memb)
        off, col, w = oracle.aggregate(g, memb, ncomm)
        want = np.zeros((ncomm, ncomm), dtype=np.int64)
        for i in range(n):
            for j in range(n):
                want[memb[i], memb[j]] += W[i, j]
        got = np.zeros((ncomm, ncomm), dtype=np.int64)
        for c in range(ncomm):
            row = col[off[c]:off[c + 1]]
            assert np.all(np.diff(row) > 0)  # sorted, no duplicates
            got[c, row] = w[off[c]:off[c + 1]]
        assert np.array_equal(got, want)
        # Q of the identity on the super-graph equals Q of the membership
        sg = gg.CSR(off, col, w.astype(np.int32), "super")
        assert exact_q(sg, np.arange(ncomm, dtype=np.int32)) == exact_q(g, memb)


# ---------------------------------------------------- the schedule's hash
def test_fmix32_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "murmur3_fmix32.txt")) if l[0] != "#"]
    assert rows
    for seed, want in rows:
        assert oracle.fmix32(int(seed, 16)) == int(want, 16)


def test_bucket_balance_and_variation():
    n = 1 << 14
    for (p, t, b) in [(0, 0, 4), (1, 3, 4), (2, 7, 3), (0, 19, 8)]:
        counts = np.bincount([oracle.bucket(i, p, t, 0, b) for i in range(n)], minlength=b)
        exp = n / b
        sd = np.sqrt(n * (1 / b) * (1 - 1 / b))
        assert np.all(np.abs(counts - exp) < 5 * sd), counts
    a = [oracle.bucket(i, 0, 0, 0, 4) for i in range(256)]
    bb = [oracle.bucket(i, 0, 1, 0, 4) for i in range(256)]
    c = [oracle.bucket(i, 0, 0, 99, 4) for i in range(256)]
    assert a != bb and a != c
    assert all(oracle.bucket(i, 0, 0, 0, 1) == 0 for i in range(50))


# --------------------------------------------- Algorithm 1 / 4: whole run
def test_two_disjoint_cliques():
    W = np.zeros((10, 10), dtype=np.int64)
    for blk in (range(0, 5), range(5, 10)):
        for a in blk:
            for b in blk:
                if a != b:
                    W[a, b] = 1
    r = oracle.louvain(csr_from_dense(W), oracle.Config(check_invariants=True))
    assert list(r.membership) == [0] * 5 + [1] * 5


def test_ring_of_cliques_reaches_closed_form():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ring_of_cliques.txt")) if l[0] != "#"]
    for r_, k, m, qn, qd in [tuple(map(int, x)) for x in rows]:
        g = gg.ring_of_cliques(r_, k)
        res = oracle.louvain(g, oracle.Config(check_invariants=True))
        assert Fraction(res.q_num, res.q_den) == Fraction(qn, qd), (r_, k)
        assert np.array_equal(res.membership, np.arange(r_ * k) // k)


def test_louvain_bounded_by_brute_force_optimum():
    rng = np.random.default_rng(13)
    for trial in range(8):
        n = int(rng.integers(4, 9))
        W = random_graph(rng, n, p=0.45, wmax=4)
        g = csr_from_dense(W)
        best = max(plain_q_dense(W, np.array(p)) for p in set_partitions(n))
        res = oracle.louvain(g, oracle.Config(check_invariants=True))
        assert res.modularity <= best + 1e-12
        assert abs(res.modularity - plain_q_dense(W, res.membership)) < 1e-12
        # the result is never worse than all-singletons
        assert res.modularity >= plain_q_dense(W, np.arange(n)) - 1e-12


def test_karate_club_below_published_optimum():
    nx = pytest.importorskip("networkx")
    q_opt = float(open(os.path.join(GOLDEN, "karate_club.txt")).read().split("q_opt")[1].split()[0])
    G = nx.karate_club_graph()
    u, v = zip(*G.edges())
    g = gg.from_pairs(34, u, v)
    res = oracle.louvain(g)
    assert 0.38 < res.modularity <= q_opt + 1e-7


def test_invariants_and_monotone_q_on_sbm():
    g = gg.sbm(1000, 100, 0.1, 0.002, seed=1)
    res = oracle.louvain(g, oracle.Config(check_invariants=True))
    ps = res.pass_stats[:res.passes]
    qs = [Fraction((int(r[4]) << 64) + (int(r[5]) & (2**64 - 1)), res.two_m ** 2) for r in ps]
    assert all(b >= a for a, b in zip(qs, qs[1:])), qs
    # the last per-pass Q is the final Q (modularity is invariant under aggregation)
    assert qs[-1] == Fraction(res.q_num, res.q_den)
    # super-graph sizes shrink; |Gamma| of pass p is n' of pass p+1
    for a, b in zip(ps, ps[1:]):
        assert b[0] == a[3] and b[1] <= a[1]
    # planted partition: at least 9 of the 10 blocks are recovered by majority
    blocks = np.arange(1000) // 100
    hits = 0
    for b in range(10):
        vals, cnt = np.unique(res.membership[blocks == b], return_counts=True)
        hits += cnt.max() >= 90
    assert hits >= 9
    assert set(np.unique(res.membership)) == set(range(res.communities))


def test_result_independent_of_thread_count():
    g = gg.rmat(12, 8, seed=3)
    a = oracle.louvain(g, oracle.Config(num_threads=1))
    b = oracle.louvain(g, oracle.Config(num_threads=4))
    assert np.array_equal(a.membership, b.membership)
    assert np.array_equal(a.iter_stats, b.iter_stats)
    oracle.louvain(g, oracle.Config(num_threads=0))


def test_isolated_vertices_stay_singletons_and_edge_cases():
    g = gg.rmat(10, 4, seed=5)
    deg = np.diff(g.offsets)
    res = oracle.louvain(g)
    iso = np.nonzero(deg == 0)[0]
    assert len(iso) > 0
    comm_sizes = np.bincount(res.membership)
    assert np.all(comm_sizes[res.membership[iso]] == 1)
    # no edges at all
    e = gg.CSR(np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    r = oracle.louvain(e)
    assert list(r.membership) == list(range(5)) and r.modularity == 0.0
    # empty graph
    z = gg.CSR(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    assert oracle.louvain(z).membership.shape == (0,)


def test_iteration_records_are_consistent():
    g = gg.sbm(1000, 100, 0.1, 0.002, seed=1)
    cfg = oracle.Config()
    res = oracle.louvain(g, cfg)
    tau = cfg.tolerance
    for p, its in enumerate(res.iterations()):
        li = len(its)
        assert li == res.pass_stats[p, 2]
        for t, (ev, mv, gain) in enumerate(its):
            assert 0 <= mv <= ev and gain >= 0 and (mv == 0) == (gain == 0)
            dq = float(2 * gain) / float(res.two_m ** 2)
            if t < li - 1:
                assert dq > tau
        if li < cfg.max_iterations:
            assert float(2 * its[-1][2]) / float(res.two_m ** 2) <= tau
        tau /= cfg.tolerance_drop
    # pass 0 evaluates every vertex in its first iteration
    assert res.iter_stats[0, 0, 0] == g.n


def test_pickless_and_bucket_settings_change_the_run_but_not_validity():
    g = gg.sbm(600, 60, 0.15, 0.005, seed=9)
    base = oracle.louvain(g)
    for cfg in (oracle.Config(pickless_period=0), oracle.Config(buckets=1), oracle.Config(buckets=7),
                oracle.Config(schedule_seed=12345)):
        r = oracle.louvain(g, cfg)
        assert abs(r.modularity - base.modularity) < 0.05
        assert set(np.unique(r.membership)) == set(range(r.communities))


def test_fully_simultaneous_decisions_collapse_a_mixed_sbm():
    """Why the schedule has buckets: with one bucket every vertex decides
    against the same snapshot, and on a planted partition with heavy mixing
    (about 45% of each vertex's edges leave its block) the moves that each
    raise modularity alone pile onto the same communities and swap back and
    forth (the community swaps of Sec. 4.3.1): the second pass hits the
    iteration cap and modularity falls to well under half.  Two or four
    buckets, where later decisions see earlier moves, stay near the planted
    partition's modularity."""
    g = gg.sbm(3000, 50, 0.3, 0.004, seed=4)
    one = oracle.louvain(g, oracle.Config(buckets=1))
    assert one.modularity < 0.3
    assert int(one.pass_stats[1, 2]) == oracle.Config().max_iterations
    for B in (2, 4):
        assert oracle.louvain(g, oracle.Config(buckets=B)).modularity > 0.52


def test_passes_form_a_refinement_chain_with_conserved_weight():
    """Each pass moves super-vertices of the previous pass's communities
    (Algorithm 1), so the partition after p + 1 passes is a coarsening of the
    one after p passes; and aggregating the input by any of them keeps its
    total weight 2m (Algorithm 3).  With the pass cap at p the memberships
    are the communities found by the first p passes."""
    for g in (gg.grid(64, 0.02, seed=5), gg.sbm(3000, 50, 0.3, 0.004, seed=4), gg.rmat(13, 12, seed=21,
                                                                                          weight_range=(1, 3))):
        full = oracle.louvain(g)
        assert full.passes >= 3
        chain = [oracle.louvain(g, oracle.Config(max_passes=p)).membership for p in range(1, full.passes + 1)]
        chain.append(full.membership)
        for fine, coarse in zip(chain, chain[1:]):
            # every community of the finer partition lies inside one community of the coarser
            ncomm = int(fine.max()) + 1
            first = np.full(ncomm, -1, dtype=np.int64)
            first[fine[::-1]] = coarse[::-1]
            assert np.array_equal(first[fine], coarse)
            assert int(np.unique(coarse).shape[0]) <= ncomm
        for memb in chain:
            o, c, w = oracle.aggregate(g, memb, int(memb.max()) + 1)
            assert int(w.sum()) == g.total_weight()


def test_pass_loop_stopping_rules_at_their_boundaries():
    """Algorithm 1's two stopping rules exactly at their boundaries.

    A pass whose local moving ends in a single iteration (l_i = 1) ends the
    run as converged: on a ring of cliques with r <= k, merging two cliques
    lowers modularity, so the second pass makes no move and the run stops
    there with exit reason 1, not through the shrink test.  And aggregation
    goes on while |Gamma|/n' <= tau_agg (the algorithm's strict '>' for
    stopping): a triangle next to seven isolated vertices leaves 8 of 10
    communities, exactly tau_agg = 0.8, so the run must aggregate and stop
    in the second pass."""
    ring = oracle.louvain(gg.ring_of_cliques(8, 10))
    assert ring.passes == 2 and ring.exit_reason == 1
    assert int(ring.pass_stats[1, 2]) == 1 and int(ring.pass_stats[1, 3]) == 8
    tri = gg.from_pairs(10, [0, 1, 0], [1, 2, 2])
    r = oracle.louvain(tri)
    assert (int(r.pass_stats[0, 0]), int(r.pass_stats[0, 3])) == (10, 8)
    assert r.passes == 2 and r.exit_reason == 1
    # with tau_agg just below 0.8 the first pass is the last
    r = oracle.louvain(tri, oracle.Config(aggregation_tolerance=0.79))
    assert r.passes == 1 and r.exit_reason == 2


def test_final_modularity_is_the_last_pass_modularity():
    """Aggregation keeps modularity (Q of the super-vertex graph under C'
    equals Q of the input under the looked-up memberships), and so does the
    dendrogram lookup.  So the run's final exact numerator equals the one
    recorded at the end of its last pass, whichever rule ended the run."""
    cases = [gg.sbm(1000, 100, 0.1, 0.002, seed=1), gg.grid(64, 0.02, seed=5),
             gg.rmat(13, 12, seed=21, weight_range=(1, 3)), gg.ring_of_cliques(8, 10),
             gg.from_pairs(10, [0, 1, 0], [1, 2, 2]), gg.sbm(3000, 50, 0.3, 0.004, seed=4)]
    reasons = set()
    for g in cases:
        for cfg in (oracle.Config(), oracle.Config(max_passes=2)):
            r = oracle.louvain(g, cfg)
            hi, lo = int(r.pass_stats[r.passes - 1, 4]), int(r.pass_stats[r.passes - 1, 5])
            assert (hi << 64) + (lo & (2**64 - 1)) == r.q_num, (g.n, cfg.max_passes)
            reasons.add(r.exit_reason)
    assert reasons == {0, 1, 2}  # every way a run can end is covered
