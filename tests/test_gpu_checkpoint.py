"""Pass-level stop, resume and checkpoints of a run, through the C ABI.

Stopping a run between two passes, resuming it in the same context, or
saving its state and restoring it into a fresh context must not change any
result: memberships, exact modularity and the per-pass and per-iteration
records equal the CPU oracle's uninterrupted run bit for bit.  Damaged or
mismatched checkpoints are refused with a status, and the context stays
usable.
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

E_INVAL, E_STATE = 1, 7
HEADER = 20

GRAPHS = {
    "rmat14_weighted": lambda: gg.rmat(14, 8, seed=3, weight_range=(1, 5)),
    "rmat16_hubs": lambda: gg.rmat(16, 16, seed=7),
    "grid96": lambda: gg.grid(96, 0.02, seed=11),
    "sbm_mixed": lambda: gg.sbm(3000, 50, 0.3, 0.004, seed=4),
}


def cfg(**kw):
    c = lv.Config(**kw)
    c.record_pass_modularity = True
    return c


def to_oracle_cfg(c):
    return oracle.Config(max_passes=c.max_passes, max_iterations=c.max_iterations, tolerance=c.tolerance,
                         tolerance_drop=c.tolerance_drop, aggregation_tolerance=c.aggregation_tolerance,
                         pickless_period=c.pickless_period, buckets=c.buckets, schedule_seed=c.schedule_seed)


def assert_same_as_oracle(res, ref):
    assert res.passes == ref.passes
    P = ref.passes
    assert np.array_equal(res.pass_stats[:P], ref.pass_stats[:P])
    for p in range(P):
        li = int(ref.pass_stats[p, 2])
        assert np.array_equal(res.iter_stats[p, :li], ref.iter_stats[p, :li]), p
    assert res.exit_reason == ref.exit_reason
    assert res.communities == ref.communities
    assert np.array_equal(res.membership, ref.membership)
    assert (res.q_num, res.q_den) == (ref.q_num, ref.q_den)


def assert_same(a, b):
    assert (a.passes, a.communities, a.exit_reason) == (b.passes, b.communities, b.exit_reason)
    assert np.array_equal(a.membership, b.membership)
    assert (a.q_num, a.q_den) == (b.q_num, b.q_den)
    assert np.array_equal(a.pass_stats, b.pass_stats)
    assert np.array_equal(a.iter_stats, b.iter_stats)


def status_of(fn):
    with pytest.raises(lv.LouvainError) as ei:
        fn()
    return ei.value.status


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_stop_and_resume_in_place(name):
    g = GRAPHS[name]()
    c = cfg()
    ref = oracle.louvain(g, to_oracle_cfg(c))
    assert ref.passes >= 2, "the case must have a pass boundary to stop at"
    for step in (1, 2):
        with lv.Louvain(lv.DeviceCSR.from_host(g), c) as ctx:
            stopped = ctx.run_passes(step)
            assert stopped == (ref.passes > step)
            stops = 1 if stopped else 0
            while stopped:
                assert status_of(lambda: lv.louvain_modularity(ctx.ctx)) == E_STATE
                stopped = ctx.resume(1)
                stops += stopped
            assert stops == max(0, ref.passes - 1 - (step - 1))
            res = ctx.result()
            assert ctx.stats()["passes"] == ref.passes
        assert_same_as_oracle(res, ref)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_checkpoint_into_fresh_context(name):
    g = GRAPHS[name]()
    c = cfg()
    ref = oracle.louvain(g, to_oracle_cfg(c))
    for step in range(1, ref.passes):
        with lv.Louvain(lv.DeviceCSR.from_host(g), c) as a:
            assert a.run_passes(step)
            buf = a.save_state()
            assert buf.dtype == np.uint8 and buf.nbytes % 8 == 0
            assert np.array_equal(a.save_state(), buf)  # saving does not change the state
        with lv.Louvain(g, c) as b:  # host input: a context of its own
            b.load_state(bytes(buf))
            assert not b.resume()
            res = b.result()
            b.stats()
            # the same checkpoint again, into a context that has finished a run
            b.load_state(buf)
            assert not b.resume()
            assert_same(b.result(), res)
        assert_same_as_oracle(res, ref)


@pytest.mark.parametrize("sched", [dict(graphs=1), dict(concurrent=1), dict(graphs=1, concurrent=1)])
def test_checkpoint_with_replay_and_concurrent_bins(sched):
    g = gg.rmat(16, 16, seed=7)
    c = cfg()
    ref = oracle.louvain(g, to_oracle_cfg(c))
    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as a:
        a.set_schedule(sched)
        assert a.run_passes(1)
        buf = a.save_state()
        assert not a.resume()
        assert_same_as_oracle(a.result(), ref)
    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as b:
        b.set_schedule(sched)
        b.load_state(buf)
        assert not b.resume()
        assert_same_as_oracle(b.result(), ref)


def test_learned_mode_checkpoint():
    from paper_2501_19004_gb300 import predictor
    g = gg.rmat(15, 16, seed=9)
    model = predictor.load_default()
    assert model is not None, "the stored predictor model is missing"
    c = cfg(mode=lv.MODE_LEARNED, model=model)
    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as a:
        full = a.run().result()
        assert full.passes >= 2
        assert a.run_passes(1)
        buf = a.save_state()
    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as b:
        b.load_state(buf)
        assert not b.resume()
        assert_same(b.result(), full)
        log = b.stats().get("learned_passes")
        assert log is not None and len(log) == full.passes
    # another model is another configuration
    other = model.copy()
    other[0] += 1.0
    with lv.Louvain(lv.DeviceCSR.from_host(g), cfg(mode=lv.MODE_LEARNED, model=other)) as d:
        assert status_of(lambda: d.load_state(buf)) == E_INVAL


def test_run_passes_that_finish():
    g = gg.rmat(13, 12, seed=21, weight_range=(1, 3))
    c = cfg()
    ref = oracle.louvain(g, to_oracle_cfg(c))
    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as ctx:
        assert not ctx.run_passes(100)
        assert_same_as_oracle(ctx.result(), ref)
        assert not ctx.run_passes(0)
        assert_same_as_oracle(ctx.result(), ref)
    c1 = cfg(max_passes=1)
    with lv.Louvain(lv.DeviceCSR.from_host(g), c1) as ctx:
        assert not ctx.run_passes(1)  # the pass cap ends the run: nothing to suspend
        assert_same_as_oracle(ctx.result(), oracle.louvain(g, to_oracle_cfg(c1)))


# --- refusals -------------------------------------------------------------

def fnv1a_words(words: np.ndarray) -> int:
    h = 0xcbf29ce484222325
    for w in words.astype(np.uint64).tolist():
        h = ((h ^ w) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def sections(buf, n0, T):
    """Byte ranges of the payload sections of a checkpoint."""
    h = buf[:HEADER * 8].view(np.int64)
    P, n, nnz, L = int(h[9]), int(h[10]), int(h[11]), int(h[17])
    pad8 = lambda b: (b + 7) // 8 * 8  # noqa: E731
    pos, out = HEADER * 8, {}
    for key, size in (("pass", P * 6 * 8), ("iter", P * T * 4 * 8), ("log", L * 24), ("C", pad8(4 * n0)),
                      ("K", 8 * n), ("off", 8 * (n + 1)), ("cols", pad8(4 * nnz)), ("w", pad8(4 * nnz))):
        out[key] = (pos, pos + size)
        pos += size
    assert pos == buf.nbytes
    return out, n, nnz


def reseal(buf):
    """Recompute the payload checksum of an edited checkpoint."""
    out = buf.copy()
    out[24:32] = np.array([fnv1a_words(out[HEADER * 8:].view(np.uint64))], dtype=np.uint64).view(np.uint8)
    return out


def test_refusals_and_recovery():
    g = gg.rmat(12, 16, seed=7)
    c = cfg()
    ref = oracle.louvain(g, to_oracle_cfg(c))
    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as a:
        # nothing suspended yet
        assert status_of(lambda: a.save_state()) == E_STATE
        assert status_of(lambda: a.resume()) == E_STATE
        a.run()
        assert status_of(lambda: a.save_state()) == E_STATE
        assert status_of(lambda: a.resume()) == E_STATE
        assert a.run_passes(1)
        buf = a.save_state()
        assert not a.resume()
    assert reseal(buf).tobytes() == buf.tobytes()  # the test's checksum is the library's

    secs, n, nnz = sections(buf, g.n, c.max_iterations)
    assert n >= 2 and nnz >= 1
    bad = {}
    x = buf.copy()
    x[secs["cols"][0]] ^= 1  # one flipped bit: checksum mismatch
    bad["bit flip"] = x
    bad["truncated"] = buf[:-8].copy()
    bad["not a checkpoint"] = np.zeros_like(buf)
    x = buf.copy()
    x[secs["cols"][0]:secs["cols"][0] + 4] = np.array([n], dtype=np.int32).view(np.uint8)
    bad["column out of range (device check)"] = reseal(x)
    x = buf.copy()
    x[secs["w"][0]:secs["w"][0] + 4] = np.array([0], dtype=np.uint32).view(np.uint8)
    bad["zero weight (device check)"] = reseal(x)
    x = buf.copy()
    x[secs["C"][0]:secs["C"][0] + 4] = np.array([n], dtype=np.int32).view(np.uint8)
    bad["dendrogram id out of range"] = reseal(x)
    x = buf.copy()
    o0 = secs["off"][0]
    x[o0 + 8:o0 + 16] = np.array([nnz + 1], dtype=np.int64).view(np.uint8)
    bad["row offsets"] = reseal(x)
    x = buf.copy()
    x[secs["K"][0]:secs["K"][0] + 8] = np.array([-1], dtype=np.int64).view(np.uint8)
    bad["negative vertex weight"] = reseal(x)
    x = buf.copy()
    kv = x[secs["K"][0]:secs["K"][0] + 16].view(np.int64).copy()
    kv[0] += 1
    x[secs["K"][0]:secs["K"][0] + 16] = kv.view(np.uint8)
    bad["vertex weights off 2m"] = reseal(x)

    with lv.Louvain(lv.DeviceCSR.from_host(g), c) as b:
        for why, blob in bad.items():
            assert status_of(lambda: b.load_state(blob)) == E_INVAL, why
            assert status_of(lambda: b.resume()) == E_STATE, why
        # the context still works after every refusal
        assert_same_as_oracle(b.run().result(), ref)
        b.load_state(buf)
        assert not b.resume()
        assert_same_as_oracle(b.result(), ref)

    # another graph with the same sizes, another seed of the schedule
    g2 = gg.rmat(12, 16, seed=8)
    with lv.Louvain(lv.DeviceCSR.from_host(g2), c) as d:
        assert status_of(lambda: d.load_state(buf)) == E_INVAL
    with lv.Louvain(lv.DeviceCSR.from_host(g), cfg(schedule_seed=99)) as d:
        assert status_of(lambda: d.load_state(buf)) == E_INVAL
    with lv.Louvain(lv.DeviceCSR.from_host(g), cfg(table_window=4096)) as d:  # no effect on results: accepted
        d.load_state(buf)
        assert not d.resume()
        assert_same_as_oracle(d.result(), ref)

    # batched contexts have no pass-level control
    union, vo = gg.concat([g, gg.ring_of_cliques(4, 5)])
    with lv.LouvainBatch(lv.DeviceCSR.from_host(union), vo) as bb:
        assert status_of(lambda: lv.louvain_run_passes(bb.ctx, 1)) == E_INVAL
        assert status_of(lambda: lv.louvain_load_state(bb.ctx, buf)) == E_INVAL
