"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (concurrent bins, CUDA-graph replay, the batched context).

- R-MAT scale 24: bit-exact against a full oracle run (memberships, per-pass
  records, exact modularity), in the Louvain and in the Leiden form.
- The 4,096-graph batch: one batched run of all graphs; 32 graphs sampled
  with a stride are checked bit-exactly against the oracle run on each.
- The 8192 x 8192 grid: bit-exact against a full oracle run.
- R-MAT scale 27 (4.2 billion entries, the learned-skip evaluation graph):
  bit-exact against a full oracle run on the host cores (memberships,
  per-iteration and per-pass records, exact modularity), plus the oracle's
  modularity of the GPU's memberships; and the learned-skip form with the
  stored predictor against the plain form on the same graph: higher
  throughput (event-timed whole runs) with a modularity within 1e-3 of the
  plain result.
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
from paper_2501_19004_gb300 import predictor  # noqa: E402

FAST = dict(concurrent=1, graphs=1)


def test_rmat24_bit_exact_full_size():
    g = gg.rmat(24, 16, seed=7)
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(record_pass_modularity=True)) as ctx:
        ctx.set_schedule(FAST)
        res = ctx.run().result()
    ref = oracle.louvain(g, oracle.Config())
    assert res.passes == ref.passes
    P = ref.passes
    assert np.array_equal(res.pass_stats[:P, :4], ref.pass_stats[:P, :4])
    assert np.array_equal(res.pass_stats[:P, 4:], ref.pass_stats[:P, 4:])
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)
    assert abs(res.modularity - ref.modularity) <= 1e-9


def test_rmat24_leiden_bit_exact_full_size():
    g = gg.rmat(24, 16, seed=7)
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(refine=True, record_pass_modularity=True)) as ctx:
        ctx.set_schedule(FAST)
        res = ctx.run().result()
    ref = oracle.louvain(g, oracle.Config(refine=True))
    assert res.passes == ref.passes and res.exit_reason == ref.exit_reason
    P = ref.passes
    assert np.array_equal(res.pass_stats[:P], ref.pass_stats[:P])
    assert np.array_equal(res.iter_stats[:P], ref.iter_stats[:P])
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)


def test_batch4096_sampled_bit_exact():
    union, vo = gg.batched_sbm_union(4096)
    with lv.LouvainBatch(lv.DeviceCSR.from_host(union), vo) as b:
        b.set_schedule(dict(concurrent=1))
        res = b.run().result()
    assert res.summary.shape[0] == 4096
    for k in range(0, 4096, 128):
        g = gg.batched_sbm(k)
        memb, q, num, den, passes, comms, why = res.graph(k)
        ref = oracle.louvain(g, oracle.Config())
        assert np.array_equal(memb, ref.membership), k
        assert (num, den, passes, comms, why) == (ref.q_num, ref.q_den, ref.passes, ref.communities,
                                                  ref.exit_reason), k
    # every graph's memberships are dense local ids
    for k in range(0, 4096, 97):
        memb = res.graph(k)[0]
        assert memb.min() == 0 and memb.max() == int(res.summary[k, 1]) - 1


def test_grid8192_bit_exact_full_size():
    g = gg.grid(8192, 0.02, seed=11)
    with lv.Louvain(lv.DeviceCSR.from_host(g)) as ctx:
        ctx.set_schedule(FAST)
        res = ctx.run().result()
    q, num, den = oracle.modularity(g, res.membership)
    assert (num, den) == (res.q_num, res.q_den)
    used = np.unique(res.membership)
    assert used[0] == 0 and used[-1] == res.communities - 1 and used.shape[0] == res.communities
    ref = oracle.louvain(g, oracle.Config())
    assert res.passes == ref.passes
    assert np.array_equal(res.pass_stats[:ref.passes, :4], ref.pass_stats[:ref.passes, :4])
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)


@pytest.fixture(scope="module")
def rmat27():
    return gg.rmat(27, 16, seed=13)


def _best_run(dg, cfg, runs=3):
    """(fastest event-timed run in ms, stats of the last run, result)"""
    with lv.Louvain(dg, cfg) as ctx:
        ctx.set_schedule(dict(concurrent=1))
        ctx.run()  # warm-up: device code loaded, workspaces sized
        ms = []
        for _ in range(runs):
            ctx.run()
            st = ctx.stats()
            ms.append(st["run_ms"])
        return min(ms), st, ctx.result()


@pytest.mark.slow
def test_rmat27_learned_skip_beats_plain(rmat27):
    """The learned-skip form, with the stored predictor (trained on R-MAT
    20-22 traces) and the settings it was trained for, against the plain
    form on the R-MAT scale-27 graph: fewer evaluations, less time per run,
    and a modularity within 1e-3 of the plain result, on a partition whose
    modularity the oracle confirms."""
    model = predictor.load_default()
    assert model is not None
    dg = lv.DeviceCSR.from_host(rmat27)
    t_plain, st_plain, plain = _best_run(dg, lv.Config())
    t_learned, st_learned, learned = _best_run(dg, predictor.default_config(model))
    del dg
    torch.cuda.empty_cache()
    assert st_learned["skipped"] > 0
    assert st_learned["evaluated"] < st_plain["evaluated"]
    assert abs(learned.modularity - plain.modularity) <= 1e-3, (learned.modularity, plain.modularity)
    assert t_learned < t_plain, (t_learned, t_plain)
    q, num, den = oracle.modularity(rmat27, learned.membership)
    assert (num, den) == (learned.q_num, learned.q_den)


@pytest.mark.slow
def test_rmat27_bit_exact_full_size(rmat27):
    """4.2 billion entries, in the benchmark's launch configuration: the
    GPU's run against a complete oracle run (OpenMP over the host cores,
    about 110 GB of host memory), element by element."""
    g = rmat27
    dg = lv.DeviceCSR.from_host(g)
    with lv.Louvain(dg, lv.Config(record_pass_modularity=True)) as ctx:
        ctx.set_schedule(FAST)
        res = ctx.run().result()
    del dg
    torch.cuda.empty_cache()
    q, num, den = oracle.modularity(g, res.membership)
    assert (num, den) == (res.q_num, res.q_den)
    used = np.unique(res.membership)
    assert used[0] == 0 and used[-1] == res.communities - 1 and used.shape[0] == res.communities
    ref = oracle.louvain(g, oracle.Config())
    assert (res.passes, res.exit_reason, res.communities) == (ref.passes, ref.exit_reason, ref.communities)
    P = ref.passes
    assert np.array_equal(res.pass_stats[:P], ref.pass_stats[:P])
    assert np.array_equal(res.iter_stats[:P], ref.iter_stats[:P])
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)
