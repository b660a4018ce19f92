"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (concurrent bins, CUDA-graph replay, the batched context).

- R-MAT scale 24 (the default benchmark workload): bit-exact against a full
  oracle run (memberships, per-pass records, exact modularity).
- The 4,096-graph batch: one batched run of all graphs; 32 graphs sampled
  with a stride are checked bit-exactly against the oracle run on each.
- The 8192 x 8192 grid: bit-exact against a full oracle run.
- R-MAT scale 27 (4.2 billion entries, the learned-skip evaluation graph):
  bit-exact against a full oracle run on the host cores (memberships,
  per-iteration and per-pass records, exact modularity), plus the oracle's
  modularity of the GPU's memberships.
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


@pytest.mark.slow
def test_rmat27_bit_exact_full_size():
    """4.2 billion entries, in the benchmark's launch configuration: the
    GPU's run against a complete oracle run (OpenMP over the host cores,
    about 110 GB of host memory), element by element."""
    g = gg.rmat(27, 16, seed=13)
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
