"""Launch schedules, the autotuner and graph replay never change results.

Every schedule (bin thresholds, blocks per SM, CUDA-graph replay of the
local-moving iterations) must give the oracle's memberships and exact
modularity bit for bit, for single graphs and batches.
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


def check_single(g, res):
    ref = oracle.louvain(g, oracle.Config())
    assert res.passes == ref.passes
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)
    P = ref.passes
    assert np.array_equal(res.pass_stats[:P, :4], ref.pass_stats[:P, :4])


SCHEDULES = [
    dict(group_max=16, half_max=16),                       # no group bins
    dict(group_max=32, half_max=32, warp_max=64),          # 65..1024 in 128-thread blocks
    dict(group_max=48, half_max=128, warp_max=128),        # no warp bin
    dict(group_max=64, half_max=96, warp_max=256),
    dict(move_thread=1, move_warp=1, move_mid=1, move_block=1, move_hub=1, move_group=1,
         merge_thread=1, merge_warp=1, merge_mid=1, merge_block=1, merge_big=1),
    dict(move_thread=16, move_warp=16, move_mid=16, move_block=16, move_group=16, merge_warp=16),
    dict(graphs=1),
    dict(graphs=1, group_max=16, half_max=16, warp_max=64, move_hub=2),
    dict(concurrent=1),
    dict(concurrent=1, graphs=1),
    dict(graphs=2),                                        # whole phase under device control
    dict(graphs=2, concurrent=1, group_max=32, half_max=64, warp_max=128),
]


@pytest.mark.parametrize("sched", SCHEDULES)
@pytest.mark.parametrize("name", ["rmat16_hubs", "rmat14_weighted", "grid64"])
def test_schedules_bit_exact(sched, name):
    g = {"rmat16_hubs": lambda: gg.rmat(16, 16, seed=7),
         "rmat14_weighted": lambda: gg.rmat(14, 8, seed=3, weight_range=(1, 5)),
         "grid64": lambda: gg.grid(64, 0.02, seed=5)}[name]()
    with lv.Louvain(lv.DeviceCSR.from_host(g)) as ctx:
        ctx.set_schedule(sched)
        got = ctx.schedule()
        for k, v in sched.items():
            assert got[k] == v
        r1 = ctx.run().result()
        r2 = ctx.run().result()  # replay graphs captured by the first run's passes are rebuilt per run
    check_single(g, r1)
    check_single(g, r2)


@pytest.mark.parametrize("mode", [1, 2])
def test_graph_replay_batch(mode):
    """Per-iteration replay (graphs = 1) and the device-controlled phase
    (graphs = 2: every graph's tolerance test on the device) on a batch: each
    graph's result and per-pass records equal its own oracle run."""
    graphs = [gg.batched_sbm(k) for k in (0, 1, 3, 8, 10)] + [gg.rmat(12, 16, seed=7)]
    union, vo = gg.concat(graphs)
    with lv.LouvainBatch(lv.DeviceCSR.from_host(union), vo) as b:
        b.set_schedule(dict(graphs=mode, concurrent=1))
        res = b.run().result()
        res2 = b.run().result()
    for r in (res, res2):
        for k, g in enumerate(graphs):
            memb, q, num, den, passes, comms, why = r.graph(k)
            ref = oracle.louvain(g, oracle.Config())
            assert np.array_equal(memb, ref.membership), k
            assert (num, den, passes, why) == (ref.q_num, ref.q_den, ref.passes, ref.exit_reason), k
            assert np.array_equal(r.pass_records[k, :passes, 1], ref.pass_stats[:passes, 2]), k  # l_i per pass


def test_autotune_keeps_results():
    g = gg.rmat(15, 16, seed=9)
    with lv.Louvain(lv.DeviceCSR.from_host(g)) as ctx:
        rep = ctx.autotune(max_runs=12)
        assert rep["runs"] <= 12 + 1
        assert rep["tuned_ms"] <= rep["start_ms"] + 1e-9
        assert len(rep["schedule"]) == len(lv.SCHEDULE_FIELDS)
        assert rep["trials"] and rep["trials"][0]["step"] == "start"
        after = ctx.result()  # the autotuner leaves a result of the chosen schedule
        again = ctx.run().result()
    check_single(g, after)
    check_single(g, again)


def test_autotune_measures_the_current_blocks_first():
    """The blocks-per-SM step times the current values before the
    candidates, so a bin keeps its value unless a candidate's kernel time
    beats it; the tuned schedule still gives the oracle's result."""
    g = gg.rmat(13, 16, seed=4)
    with lv.Louvain(lv.DeviceCSR.from_host(g)) as ctx:
        start = ctx.schedule()
        rep = ctx.autotune(max_runs=40)
        steps = [t["step"] for t in rep["trials"]]
        assert "blocks current" in steps
        k = steps.index("blocks current")
        assert steps[k + 1] == "blocks"
        current = rep["trials"][k]["schedule"]
        blocks = slice(3, 19)  # blocks per SM of the local-moving and aggregation bins
        assert current[blocks] == [start[f] for f in lv.SCHEDULE_FIELDS][blocks]
        assert rep["tuned_ms"] <= rep["start_ms"] + 1e-9
        res = ctx.result()
    check_single(g, res)


def test_autotune_batch():
    graphs = [gg.batched_sbm(k) for k in (0, 1, 3, 8)]
    union, vo = gg.concat(graphs)
    with lv.LouvainBatch(lv.DeviceCSR.from_host(union), vo) as b:
        rep = b.autotune(max_runs=10)
        res = b.result()
    assert rep["runs"] <= 11
    for k, g in enumerate(graphs):
        memb, q, num, den, passes, comms, why = res.graph(k)
        ref = oracle.louvain(g, oracle.Config())
        assert np.array_equal(memb, ref.membership)
        assert (num, den) == (ref.q_num, ref.q_den)


def test_bad_schedules_refused():
    g = gg.rmat(10, 8, seed=1)
    with lv.Louvain(g) as ctx:
        for bad in (dict(group_max=8), dict(group_max=65), dict(group_max=64, warp_max=32), dict(warp_max=300),
                    dict(half_max=200), dict(group_max=64, half_max=32),
                    dict(move_warp=0), dict(move_hub=4), dict(merge_big=5), dict(graphs=3), dict(move_thread=65),
                    dict(concurrent=3)):
            before = ctx.schedule()
            with pytest.raises(lv.LouvainError) as ei:
                ctx.set_schedule(bad)
            assert ei.value.status == 1
            assert ctx.schedule() == before


@pytest.mark.parametrize("name", ["grid96_many_iterations", "rmat19_hubs", "sbm_iteration_cap"])
def test_device_controlled_phase(name):
    """graphs = 2: each pass's local-moving phase is one graph launch whose
    conditional while node repeats the iteration until the device-side
    tolerance test stops it (no host synchronisation per iteration).  The
    iteration counts, per-iteration records and results equal the oracle's,
    also with the hub path (static rounds) and at the iteration cap."""
    cfg = lv.Config()
    if name == "grid96_many_iterations":
        g = gg.grid(96, 0.02, seed=3, weight_range=(1, 8))
    elif name == "rmat19_hubs":
        g = gg.rmat(19, 16, seed=7)
    else:
        g = gg.sbm(3000, 50, 0.3, 0.004, seed=4)
        cfg = lv.Config(tolerance=0.0, max_iterations=7)  # every phase runs to the cap
    with lv.Louvain(lv.DeviceCSR.from_host(g), cfg) as ctx:
        ctx.set_schedule(dict(graphs=2, concurrent=1))
        res = ctx.run().result()
        st = ctx.stats()
        res2 = ctx.run().result()
    ref = oracle.louvain(g, oracle.Config(tolerance=cfg.tolerance, max_iterations=cfg.max_iterations))
    for r in (res, res2):
        assert r.passes == ref.passes
        P = ref.passes
        assert np.array_equal(r.iter_stats[:P], ref.iter_stats[:P])
        assert np.array_equal(r.pass_stats[:P, :4], ref.pass_stats[:P, :4])
        assert np.array_equal(r.membership, ref.membership)
        assert (r.q_num, r.q_den) == (ref.q_num, ref.q_den)
    assert st["iterations"] == int(ref.pass_stats[:ref.passes, 2].sum())
