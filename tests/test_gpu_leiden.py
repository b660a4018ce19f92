"""The Leiden form (refine = 1) on the GPU against the oracle, through the C
ABI.

The refinement is deterministic integer arithmetic on both sides, like the
plain method, so the bar is the same: bit-exact memberships, per-iteration
and per-pass records (n' of every pass is the number of refined communities
of the one before), the exit reason and the exact modularity.  The cases
reach every decision bin on the filtered rows (thread and group bins on SBM
and grid rows, the wide bin on R-MAT 18, the global-table hub path on
R-MAT 19), weighted rows, the pass cap (the memberships are then the last
pass's P), the launch schedules, and the refused combinations.
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

from test_gpu_parity import CASES, assert_same, to_oracle_cfg  # noqa: E402


def run_leiden(g, cfg=None, schedule=None, device_input=True):
    cfg = cfg or lv.Config()
    cfg.refine = True
    cfg.record_pass_modularity = True
    graph = lv.DeviceCSR.from_host(g) if device_input else g
    with lv.Louvain(graph, cfg) as ctx:
        if schedule:
            ctx.set_schedule(schedule)
        res = ctx.run().result()
    ocfg = to_oracle_cfg(cfg)
    ocfg.refine = True
    return res, oracle.louvain(g, ocfg)


@pytest.mark.parametrize("name", sorted(CASES))
def test_leiden_bit_exact(name):
    res, ref = run_leiden(CASES[name]())
    assert_same(res, ref)


@pytest.mark.parametrize("cfg", [dict(buckets=1), dict(buckets=7), dict(pickless_period=0), dict(max_passes=1),
                                 dict(max_passes=2), dict(aggregation_tolerance=1.0), dict(tolerance=0.0,
                                                                                            max_iterations=5)])
def test_leiden_config_variants(cfg):
    for g in (gg.rmat(14, 8, seed=3, weight_range=(1, 5)), gg.sbm(3000, 50, 0.3, 0.004, seed=4)):
        res, ref = run_leiden(g, lv.Config(**cfg))
        assert_same(res, ref)


@pytest.mark.parametrize("sched", [dict(concurrent=1), dict(graphs=1), dict(graphs=2, concurrent=1),
                                   dict(group_max=16, half_max=16, warp_max=64)])
def test_leiden_schedules(sched):
    g = gg.rmat(18, 16, seed=7)
    res, ref = run_leiden(g, schedule=sched)
    assert_same(res, ref)


def test_leiden_repeated_runs_and_host_input():
    g = gg.rmat(15, 16, seed=2)
    cfg = lv.Config(refine=True)
    with lv.Louvain(g, cfg) as ctx:  # host input
        a = ctx.run().result()
        b = ctx.run().result()
    assert np.array_equal(a.membership, b.membership)
    ref = oracle.louvain(g, oracle.Config(refine=True))
    assert np.array_equal(a.membership, ref.membership) and (a.q_num, a.q_den) == (ref.q_num, ref.q_den)


def test_leiden_differs_from_louvain_and_connects_communities():
    """On R-MAT 14 the Leiden form returns a different partition of higher
    modularity than the Louvain form (as the oracle does), and its
    communities are connected where the Louvain form leaves some split."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    g = gg.rmat(14, 16, seed=7)
    plain = lv.run(lv.DeviceCSR.from_host(g))
    leiden = lv.run(lv.DeviceCSR.from_host(g), lv.Config(refine=True))
    assert leiden.modularity > plain.modularity

    def split(memb):
        rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
        same = memb[rows] == memb[g.cols]
        A = csr_matrix((np.ones(int(same.sum())), (rows[same], g.cols[same])), shape=(g.n, g.n))
        _, lab = connected_components(A, directed=False)
        pairs = np.unique(np.stack([memb, lab]), axis=1)
        return int((np.bincount(pairs[0]) > 1).sum())

    assert split(plain.membership) > 0 and split(leiden.membership) == 0


def test_leiden_refused_combinations():
    g = gg.sbm(1000, 100, 0.1, 0.002, seed=1)
    dg = lv.DeviceCSR.from_host(g)
    for bad in (dict(asynchronous=True), dict(mode=lv.MODE_LEARNED, model=np.zeros(lv.louvain_model_size(),
                                                                                   dtype=np.float32)),
                dict(trace_capacity=100)):
        with pytest.raises(lv.LouvainError):
            lv.Louvain(dg, lv.Config(refine=True, **bad))
    union, vo = gg.concat([gg.batched_sbm(k) for k in range(3)])
    with pytest.raises(lv.LouvainError):
        lv.LouvainBatch(lv.DeviceCSR.from_host(union), vo, lv.Config(refine=True))
    with lv.Louvain(dg, lv.Config(refine=True)) as ctx:
        with pytest.raises(lv.LouvainError):
            ctx.run_passes(1)
        res = ctx.run().result()  # the context stays usable
    ref = oracle.louvain(g, oracle.Config(refine=True))
    assert np.array_equal(res.membership, ref.membership)


@pytest.mark.parametrize("buckets,window", [(1, 4096), (4, 4096)])
def test_leiden_hub_rounds(buckets, window):
    """Small table windows put the hub tables of local moving and of the
    refinement, and the big-community merge tables, through many rounds."""
    res, ref = run_leiden(gg.rmat(19, 16, seed=7), lv.Config(buckets=buckets, table_window=window))
    assert_same(res, ref)


def test_leiden_edge_cases():
    # isolated vertices only, a single edge, a single vertex
    for g in (gg.CSR(np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), None), gg.from_pairs(2, [0], [1]),
              gg.CSR(np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), None)):
        res, ref = run_leiden(g, device_input=False)
        assert_same(res, ref)
    z = gg.CSR(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    assert lv.run(z, lv.Config(refine=True)).membership.shape == (0,)
    # stars: the hub in the wide bin (8999 leaves) and in the global-table bin (40000 leaves)
    for n in (9000, 40001):
        star = gg.from_pairs(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n, dtype=np.int64))
        res, ref = run_leiden(star)
        assert_same(res, ref)
