"""GPU path vs the CPU oracle, through the C ABI.

The plain method is deterministic integer arithmetic on both sides, so the
bar is bit-exactness: memberships, per-iteration evaluated/move counts and
exact gains, per-pass sizes and iteration counts, and the exact modularity
numerator and denominator (hence Q within 1e-9, trivially).
"""
import numpy as np
import pytest

import oracle
from paper_2501_19004_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2501_19004_gb300 import louvain as lv  # noqa: E402


def to_oracle_cfg(c: "lv.Config") -> oracle.Config:
    return oracle.Config(max_passes=c.max_passes, max_iterations=c.max_iterations, tolerance=c.tolerance,
                         tolerance_drop=c.tolerance_drop, aggregation_tolerance=c.aggregation_tolerance,
                         pickless_period=c.pickless_period, buckets=c.buckets, schedule_seed=c.schedule_seed)


def assert_same(res: "lv.Result", ref: "oracle.Result", check_pass_q=True):
    assert res.passes == ref.passes, (res.passes, ref.passes)
    P = ref.passes
    # per pass: n', nnz', l_i, |Gamma|
    assert np.array_equal(res.pass_stats[:P, :4], ref.pass_stats[:P, :4]), (res.pass_stats[:P], ref.pass_stats[:P])
    if check_pass_q:
        assert np.array_equal(res.pass_stats[:P, 4:], ref.pass_stats[:P, 4:])
    # per iteration: evaluated, moves, exact gain
    for p in range(P):
        li = int(ref.pass_stats[p, 2])
        assert np.array_equal(res.iter_stats[p, :li], ref.iter_stats[p, :li]), (p, res.iter_stats[p, :li],
                                                                                   ref.iter_stats[p, :li])
    assert res.exit_reason == ref.exit_reason
    assert res.communities == ref.communities
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)
    assert abs(res.modularity - ref.modularity) <= 1e-9


def run_both(g, cfg=None, device_input=True):
    cfg = cfg or lv.Config()
    cfg.record_pass_modularity = True
    graph = lv.DeviceCSR.from_host(g) if device_input else g
    res = lv.run(graph, cfg)
    ref = oracle.louvain(g, to_oracle_cfg(cfg))
    return res, ref


CASES = {
    "sbm1000": lambda: gg.sbm(1000, 100, 0.1, 0.002, seed=1),
    "sbm_mixed": lambda: gg.sbm(3000, 50, 0.3, 0.004, seed=4),
    "rmat12": lambda: gg.rmat(12, 16, seed=7),
    "rmat14_weighted": lambda: gg.rmat(14, 8, seed=3, weight_range=(1, 5)),
    "rmat16_hubs": lambda: gg.rmat(16, 16, seed=7),
    "rmat18_hubs": lambda: gg.rmat(18, 16, seed=7),  # 172 vertices above 4096 (wide bin), 19 above 8192
    "rmat19_hubs": lambda: gg.rmat(19, 16, seed=7),  # one vertex above 32768 (global tables)
    "grid96": lambda: gg.grid(96, 0.02, seed=11),
    "ring8x10": lambda: gg.ring_of_cliques(8, 10),
    "batched_sbm_0": lambda: gg.batched_sbm(0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_plain_bit_exact(name):
    g = CASES[name]()
    res, ref = run_both(g)
    assert_same(res, ref)


@pytest.mark.parametrize("cfg", [
    dict(pickless_period=0), dict(buckets=1), dict(buckets=7), dict(schedule_seed=0xDEADBEEF12345),
    dict(max_passes=1), dict(max_passes=2), dict(max_passes=0), dict(tolerance=0.0, max_iterations=7),
    dict(aggregation_tolerance=1.0), dict(tolerance_drop=1.0),
])
def test_plain_bit_exact_across_settings(cfg):
    g = gg.rmat(13, 12, seed=21, weight_range=(1, 3))
    res, ref = run_both(g, lv.Config(**cfg))
    assert_same(res, ref)


@pytest.mark.parametrize("buckets,window", [(1, 0), (2, 0), (1, 4096), (4, 4096), (2, 50000)])
def test_hub_rounds_bit_exact(buckets, window):
    """Small table windows put the hub and big-community tables through many
    rounds; results must not change."""
    g = gg.rmat(19, 16, seed=7)
    res, ref = run_both(g, lv.Config(buckets=buckets, table_window=window))
    assert_same(res, ref)


def test_host_and_device_inputs_agree_and_runs_repeat():
    g = gg.rmat(13, 16, seed=5)
    a, ref = run_both(g, device_input=False)
    assert_same(a, ref)
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(record_pass_modularity=True)) as ctx:
        r1 = ctx.run().result()
        r2 = ctx.run().result()
    assert_same(r1, ref)
    assert_same(r2, ref)


def test_edge_cases():
    # isolated vertices only
    e = gg.CSR(np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    res, ref = run_both(e)
    assert_same(res, ref)
    # a single edge, a single vertex, an empty graph
    for g in (gg.from_pairs(2, [0], [1]), gg.CSR(np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), None)):
        res, ref = run_both(g, device_input=False)
        assert_same(res, ref)
    z = gg.CSR(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    res = lv.run(z)
    assert res.membership.shape == (0,)
    # stars: one hub with many leaves, in the wide bin (8999 leaves) and
    # in the global-table bin (40000 leaves)
    for n in (9000, 40001):
        u = np.zeros(n - 1, dtype=np.int64)
        v = np.arange(1, n, dtype=np.int64)
        star = gg.from_pairs(n, u, v)
        res, ref = run_both(star)
        assert_same(res, ref)


def _pendant_paths(p):
    """A hub (vertex 0) with p paths of length two: 0 - a_k - b_k.  Once each
    pair (a_k, b_k) forms a community, the hub's row holds p distinct
    communities of two members each: none of them a known singleton."""
    a = np.arange(1, p + 1, dtype=np.int64)
    return gg.from_pairs(2 * p + 1, np.concatenate([np.zeros(p, dtype=np.int64), a]), np.concatenate([a, a + p]))


def test_wide_bin_spills_to_its_global_table():
    """Hubs of degree 4097..32768 keep at most 12288 distinct non-singleton
    communities in shared memory; more go to the block's global table.  Both
    sizes, and the largest wide degree, are bit-exact against the oracle."""
    for p in (10000, 20000, 32768):
        g = _pendant_paths(p)
        res, ref = run_both(g)
        assert_same(res, ref)
        assert res.iter_stats[0, 1, 0] > 0  # the hub was evaluated again after the pairs formed


def test_rows_with_repeated_columns():
    """Input rows that are not strictly increasing (here every row listed
    twice, a multigraph) turn the known-singleton shortcut off for the input
    graph: results still equal the oracle's, which sums repeated entries."""
    for base in (gg.from_pairs(12001, np.zeros(12000, dtype=np.int64), np.arange(1, 12001, dtype=np.int64)),
                 gg.rmat(13, 16, seed=4)):
        deg = np.diff(base.offsets)
        off = np.concatenate([[0], np.cumsum(2 * deg)]).astype(np.int64)
        cols = np.concatenate([np.concatenate([base.cols[base.offsets[i]:base.offsets[i + 1]]] * 2)
                               for i in range(base.n)]).astype(np.int32)
        g = gg.CSR(off, cols, None)
        res, ref = run_both(g)
        assert_same(res, ref)


def test_modularity_of_matches_oracle():
    rng = np.random.default_rng(3)
    for g in (gg.sbm(1000, 100, 0.1, 0.002, seed=1), gg.grid(40, 0.02, seed=2), gg.rmat(12, 8, seed=9)):
        for k in (1, 7, g.n):
            memb = rng.integers(0, k, size=g.n).astype(np.int32)
            q, num, den = lv.louvain_modularity_of(g, memb)
            rq, rnum, rden = oracle.modularity(g, memb)
            assert (num, den) == (rnum, rden) and q == rq
            dq, dnum, dden = lv.louvain_modularity_of(lv.DeviceCSR.from_host(g), torch.from_numpy(memb).cuda())
            assert (dnum, dden) == (rnum, rden)


def test_errors_are_statuses_not_crashes():
    g = gg.rmat(8, 4, seed=1)
    bad = gg.CSR(g.offsets.copy(), g.cols.copy(), None)
    bad.cols[3] = g.n + 5
    with pytest.raises(lv.LouvainError) as ei:
        lv.Louvain(bad)
    assert ei.value.status == 1
    bad2 = gg.CSR(g.offsets.copy(), g.cols.copy(), np.ones(g.nnz, dtype=np.int32))
    bad2.weights[0] = 0
    with pytest.raises(lv.LouvainError):
        lv.Louvain(bad2)
    with pytest.raises(lv.LouvainError) as ei:
        lv.Louvain(lv.DeviceCSR.from_host(bad))
    assert ei.value.status == 1
    # 2m >= 2^32 is refused
    big = gg.CSR(np.array([0, 1, 3, 4], dtype=np.int64), np.array([1, 0, 2, 1], dtype=np.int32),
                 np.full(4, 2**31 - 1, dtype=np.int32))
    with pytest.raises(lv.LouvainError) as ei:
        lv.Louvain(big)
    assert ei.value.status == 6
    # asymmetric graph refused when asked to check
    asym = gg.CSR(np.array([0, 1, 1], dtype=np.int64), np.array([1], dtype=np.int32), None)
    with pytest.raises(lv.LouvainError):
        lv.Louvain(asym, lv.Config(check_symmetry=True))
    # results before run
    ctx = lv.Louvain(g)
    with pytest.raises(lv.LouvainError) as ei:
        lv.louvain_modularity(ctx.ctx)
    assert ei.value.status == 7
    ctx.close()


def test_modularity_of_refuses_membership_ids_out_of_range():
    """An id outside [0, n) is refused with a status, on host and device
    input, and nothing is written for it; a valid call afterwards still
    agrees with the oracle."""
    g = gg.rmat(10, 8, seed=3)
    memb = (np.arange(g.n) % 13).astype(np.int32)
    for bad_id in (-1, g.n, 2**31 - 1):
        m = memb.copy()
        m[7] = bad_id
        for graph, mm in ((g, m), (lv.DeviceCSR.from_host(g), torch.from_numpy(m).cuda())):
            with pytest.raises(lv.LouvainError) as ei:
                lv.louvain_modularity_of(graph, mm)
            assert ei.value.status == 1
    q, num, den = lv.louvain_modularity_of(g, memb)
    assert oracle.modularity(g, memb)[1:] == (num, den)


def test_probe_bound_gives_hash_overflow_status(tmp_path):
    """Algorithm 7's "failed" result: a library built with a probe bound of
    one slot (LOUVAIN_MAX_PROBES=1, same sources) gives up on colliding
    inserts; the run returns LOUVAIN_E_HASH_OVERFLOW as a status (no fault),
    the context stays usable (a second run returns the same status, results
    are refused as not ready), and the product library still runs the same
    graph bit-exactly.  Shared tables (warp and block bins) and the hubs'
    global tables (R-MAT scale 19) both reach the bound."""
    from paper_2501_19004_gb300 import build
    path = build.build(force=True, defines=["LOUVAIN_MAX_PROBES=1"], lib=str(tmp_path / "liblouvain_probe1.so"),
                       objdir=str(tmp_path / "obj"))
    for g in (gg.rmat(14, 16, seed=7), gg.rmat(19, 16, seed=7)):
        dg = lv.DeviceCSR.from_host(g)
        with lv.using_library(path):
            with lv.Louvain(dg) as ctx:
                for _ in range(2):
                    with pytest.raises(lv.LouvainError) as ei:
                        ctx.run()
                    assert ei.value.status == 4  # LOUVAIN_E_HASH_OVERFLOW
                    assert "probe" in lv.louvain_last_error(ctx.ctx)
                with pytest.raises(lv.LouvainError) as ei:
                    lv.louvain_modularity(ctx.ctx)
                assert ei.value.status == 7  # no result of a failed run
        ref = oracle.louvain(g, oracle.Config())
        res = lv.run(dg)
        assert np.array_equal(res.membership, ref.membership)
        assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)
