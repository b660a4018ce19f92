"""Batched runs vs the CPU oracle run on each graph alone, through the C ABI.

A batch must give every graph exactly the result of its own run: the same
memberships (dense local ids), the same exact modularity numerator and
denominator, pass count, community count and exit reason, and per pass the
same (n', l_i, |Gamma|).
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


def to_oracle_cfg(c):
    return oracle.Config(max_passes=c.max_passes, max_iterations=c.max_iterations, tolerance=c.tolerance,
                         tolerance_drop=c.tolerance_drop, aggregation_tolerance=c.aggregation_tolerance,
                         pickless_period=c.pickless_period, buckets=c.buckets, schedule_seed=c.schedule_seed)


def empty(n):
    return gg.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), None)


# small graphs of the batched planted-partition workload (n <= 2,400)
SMALL_BSBM = [0, 1, 3, 8, 10, 19, 22, 27, 28, 30, 33, 36]


def mixed_graphs():
    gs = [gg.batched_sbm(g) for g in SMALL_BSBM[:6]]
    gs += [gg.ring_of_cliques(6, 5), empty(0), empty(5), gg.from_pairs(2, [0], [1]),
           gg.rmat(12, 16, seed=7), gg.grid(40, 0.02, seed=2)]
    gs += [gg.batched_sbm(g) for g in SMALL_BSBM[6:]]
    return gs


def check_batch(graphs, cfg, device_input=True):
    union, vo = gg.concat(graphs)
    src = lv.DeviceCSR.from_host(union) if device_input else union
    with lv.LouvainBatch(src, vo, cfg) as b:
        res = b.run().result()
    oc = to_oracle_cfg(cfg)
    P = max(cfg.max_passes, 1)
    for k, g in enumerate(graphs):
        memb, q, num, den, passes, comms, why = res.graph(k)
        ref = oracle.louvain(g, oc)
        assert passes == ref.passes, (k, passes, ref.passes)
        assert why == ref.exit_reason, (k, why, ref.exit_reason)
        assert comms == ref.communities, (k, comms, ref.communities)
        assert np.array_equal(memb, ref.membership), k
        assert (num, den) == (ref.q_num, ref.q_den), (k, num, den, ref.q_num, ref.q_den)
        assert abs(q - ref.modularity) <= 1e-9
        assert int(res.summary[k, 6]) == g.total_weight()
        pr = res.pass_records[k, :min(passes, P)]
        rp = ref.pass_stats[:min(passes, P)][:, [0, 2, 3]]
        assert np.array_equal(pr, rp), (k, pr, rp)
    return res


def test_batch_matches_single_runs():
    check_batch(mixed_graphs(), lv.Config())


def test_batch_host_input_and_repeat():
    graphs = [gg.batched_sbm(g) for g in SMALL_BSBM[:5]]
    union, vo = gg.concat(graphs)
    with lv.LouvainBatch(union, vo) as b:
        r1 = b.run().result()
        r2 = b.run().result()
    assert np.array_equal(r1.membership, r2.membership)
    assert np.array_equal(r1.summary, r2.summary)
    check_batch(graphs, lv.Config(), device_input=False)


@pytest.mark.parametrize("cfg", [
    dict(max_passes=1), dict(max_passes=2), dict(max_passes=0), dict(aggregation_tolerance=1.0),
    dict(buckets=1), dict(buckets=7, schedule_seed=12345), dict(tolerance=0.0, max_iterations=6),
    dict(pickless_period=0),
])
def test_batch_settings(cfg):
    graphs = [gg.batched_sbm(g) for g in SMALL_BSBM[:4]] + [gg.rmat(11, 8, seed=3), gg.ring_of_cliques(4, 6)]
    check_batch(graphs, lv.Config(**cfg))


def test_batch_weighted_and_hubs():
    # a weighted graph and an R-MAT graph whose hubs (up to degree 9767) take the
    # 512-thread and wide bins, next
    # to unit-weight graphs, which the union stores with weight 1
    graphs = [gg.rmat(14, 8, seed=3, weight_range=(1, 5)), gg.batched_sbm(1), gg.rmat(16, 16, seed=7),
              gg.batched_sbm(10)]
    check_batch(graphs, lv.Config())


def test_batch_single_graph_equals_plain_run():
    g = gg.rmat(13, 12, seed=21, weight_range=(1, 3))
    union, vo = gg.concat([g])
    with lv.LouvainBatch(lv.DeviceCSR.from_host(union), vo) as b:
        r = b.run().result()
    single = lv.run(lv.DeviceCSR.from_host(g))
    memb, q, num, den, passes, comms, why = r.graph(0)
    assert np.array_equal(memb, single.membership)
    assert (num, den, passes, comms, why) == (single.q_num, single.q_den, single.passes, single.communities,
                                              single.exit_reason)


def test_batch_errors():
    a, b = gg.ring_of_cliques(3, 4), gg.ring_of_cliques(3, 4)
    union, vo = gg.concat([a, b])
    # an entry that leaves its graph
    bad = gg.CSR(union.offsets.copy(), union.cols.copy(), None)
    bad.cols[0] = 20
    with pytest.raises(lv.LouvainError) as ei:
        lv.LouvainBatch(bad, vo)
    assert ei.value.status == 1
    # offsets that do not cover the union, or decrease
    for v in (np.array([0, 12, 23]), np.array([1, 12, 24]), np.array([0, 14, 12, 24])):
        with pytest.raises(lv.LouvainError):
            lv.LouvainBatch(union, v)
    # learned mode and traces are refused
    with pytest.raises(lv.LouvainError):
        lv.LouvainBatch(union, vo, lv.Config(mode=lv.MODE_LEARNED, model=np.zeros(lv.louvain_model_size(),
                                                                                   dtype=np.float32)))
    with pytest.raises(lv.LouvainError):
        lv.LouvainBatch(union, vo, lv.Config(trace_capacity=100))
    # one graph's 2m >= 2^32 is refused even though each entry is valid
    big = gg.CSR(np.array([0, 1, 3, 4], dtype=np.int64), np.array([1, 0, 2, 1], dtype=np.int32),
                 np.full(4, 2**31 - 1, dtype=np.int32))
    u2, vo2 = gg.concat([a, big])
    with pytest.raises(lv.LouvainError) as ei:
        lv.LouvainBatch(u2, vo2)
    assert ei.value.status == 6
    # a batch has no single modularity
    with lv.LouvainBatch(union, vo) as bb:
        bb.run()
        with pytest.raises(lv.LouvainError):
            lv.louvain_modularity(bb.ctx)
