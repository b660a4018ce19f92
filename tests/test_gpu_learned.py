"""GPU tests of the learned vertex-activity predictor: the tensor-core MLP
kernels against the CPU oracle (oracle/mlp.py), training, trace recording,
and the learned-skip run against the plain method (|dQ| <= 1e-3, zero-move
final sweeps, and the work it saves)."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2501_19004_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2501_19004_gb300 import louvain as lv  # noqa: E402


def _features(rng, n):
    X = np.empty((n, 8), dtype=np.float32)
    X[:, 0] = rng.uniform(0, 1, n)
    X[:, 1] = rng.uniform(0, 1, n)
    X[:, 2] = rng.uniform(-1, 1, n)
    X[:, 3] = rng.integers(0, 2, n)
    X[:, 4] = rng.uniform(0, 1, n)
    X[:, 5] = rng.uniform(0, 1, n)
    X[:, 6] = rng.uniform(0, 0.2, n)
    X[:, 7] = rng.uniform(0, 1, n)
    return X


@pytest.mark.parametrize("n", [1, 15, 16, 17, 1000, 4099])
def test_forward_matches_oracle(n):
    rng = np.random.default_rng(n)
    p = omlp.init_params(7)
    p[256:288] = rng.normal(0, 0.2, 32)
    p[1312:1344] = rng.normal(0, 0.2, 32)
    p[-1] = -0.3
    X = _features(rng, n)
    got = lv.louvain_mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    want, _ = omlp.forward(p, X, bf16=True)
    # fp32 vs exact accumulation of bf16 products, plus at most a one-ulp
    # bf16 flip of a hidden unit: well inside 1e-2 (1 + |logit|)
    assert np.all(np.abs(got - want) <= 1e-2 * (1 + np.abs(want))), np.max(np.abs(got - want))


def _gradient_bound(p, X, Y, rel, band):
    """Element-wise bound on |GPU gradient - oracle gradient| for the
    predictor's definition (include/louvain.h), derived term by term.

    Every gradient element is a sum over the rows of terms t_s (dl h2 for
    w3, h1 bf(dz2) for W2, ...).  The device forms each term from the same
    bf16 operands as the oracle except where an fp32 pre-image and the
    oracle's fp64 one fall on either side of a bf16 rounding boundary: then
    an operand moves by one bf16 ulp, at most 2^-7 of it, so a term with two
    rounded operands moves by less than 2^-6 of itself; fp32 accumulation of
    N terms adds at most about (16 + 8 + N/128) 2^-24 of the magnitude sum,
    far below that.  A bf16 flip of a hidden unit also moves its row's logit
    and so dl; that changes the terms of a single row by a few per cent at
    most, covered by 0.1 max_s |t_s|.  A ReLU mask whose pre-activation lies
    within `band` of zero (relative to the magnitude of its own sum) may
    differ between fp32 and fp64: such terms are counted in full.  So
      |g_gpu - g_oracle| <= rel * sum_s |t_s| + 0.1 max_s |t_s|
                            + sum over uncertain masks |t_s| + 1e-9,
    with rel = 2^-6 against the bf16 definition."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    n = X.shape[0]
    P = omlp.unpack(p)
    logit, c = omlp.forward(p, X, True)
    ad = np.abs((1 / (1 + np.exp(-logit)) - Y) / n)
    unc1 = np.abs(c["z1"]) <= band * (np.abs(c["xb"]) @ np.abs(c["W1"]) + np.abs(P["b1"]))
    z2abs = np.abs(c["h1"]) @ np.abs(c["W2"]) + np.abs(P["b2"])
    unc2 = np.abs(c["z2"]) <= band * z2abs
    dz2 = ad[:, None] * np.abs(c["w3"])[None, :]
    dz2m = dz2 * ((c["z2"] > 0) | unc2)
    dz2b = omlp.bf16_round(dz2m)
    dh1 = dz2b @ np.abs(c["W2"]).T
    dz1 = dh1 * ((c["z1"] > 0) | unc1)
    dz1b = omlp.bf16_round(dz1)
    h2a, h1a, xa = np.abs(c["h2"]), np.abs(c["h1"]), np.abs(c["xb"])
    M = {"b3": ad.sum(), "w3": h2a.T @ ad, "b2": dz2m.sum(0), "W2": h1a.T @ dz2b, "b1": dz1.sum(0),
         "W1": xa.T @ dz1b}
    T = {"b3": ad.max(), "w3": (h2a * ad[:, None]).max(0), "b2": dz2m.max(0),
         "W2": (h1a[:, :, None] * dz2b[:, None, :]).max(0), "b1": dz1.max(0),
         "W1": (xa[:, :, None] * dz1b[:, None, :]).max(0)}
    U = {"b3": 0.0, "w3": (band * z2abs * unc2).T @ ad, "b2": (dz2 * unc2).sum(0), "W2": h1a.T @ (dz2b * unc2),
         "b1": (dh1 * unc1).sum(0), "W1": xa.T @ (dz1b * unc1)}
    return rel * omlp.pack(M) + 0.1 * omlp.pack(T) + omlp.pack(U) + 1e-9


def _grad_case(n):
    rng = np.random.default_rng(100 + n)
    p = omlp.init_params(11)
    p[256:288] = rng.normal(0, 0.2, 32)
    p[1312:1344] = rng.normal(0, 0.2, 32)
    X = _features(rng, n)
    Y = (rng.random(n) < 0.35).astype(np.float32)
    g, loss = lv.louvain_mlp_gradient(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(),
                                      torch.from_numpy(Y).cuda())
    return p, X, Y, g.cpu().numpy().astype(np.float64), loss


@pytest.mark.parametrize("n", [16, 128, 129, 5000])
def test_gradient_matches_oracle_elementwise(n):
    """Every gradient element against the oracle's bf16 definition, within
    the bound derived in _gradient_bound (rel = 2^-6)."""
    p, X, Y, g, loss = _grad_case(n)
    want, wloss = omlp.gradient(p, X, Y, bf16=True)
    assert abs(loss - wloss) <= 1e-3 * (1 + wloss)
    bound = _gradient_bound(p, X, Y, rel=2.0 ** -6, band=1e-5)
    bad = np.nonzero(np.abs(g - want) > bound)[0]
    assert bad.size == 0, [(int(k), g[k], want[k], bound[k]) for k in bad[:8]]
    # the bound is tight enough to matter: most elements exceed it in size,
    # so a sign or index mistake in them could not pass
    nz = np.abs(want) > 0
    assert np.mean(np.abs(want[nz]) > bound[nz]) > 0.5


@pytest.mark.parametrize("n", [129, 5000])
def test_gradient_near_the_fp64_gradient_elementwise(n):
    """Every gradient element against the plain fp64 gradient of the same
    network (inputs and weights taken on the bf16 grid, then no rounding of
    activations or deltas), at a looser bound.  What remains different is the
    rounding of h1, h2, dz2 and dz1 (2^-9 of each value); a rounded hidden
    unit also moves the logit and so dl, by several per cent of a row's
    terms where p is close to y, and moves ReLU masks near zero.  Hence
    rel = 2^-2 and masks within 2^-4 of zero counted as uncertain."""
    p, X, Y, g, _ = _grad_case(n)
    pr = p.astype(np.float64).copy()
    for k in ("W1", "W2", "w3"):
        a, b, _ = omlp._SL[k]
        pr[a:b] = omlp.bf16_round(pr[a:b])
    want, _ = omlp.gradient(pr, omlp.bf16_round(X), Y, bf16=False)
    bound = _gradient_bound(p, X, Y, rel=2.0 ** -2, band=2.0 ** -4)
    bad = np.nonzero(np.abs(g - want) > bound)[0]
    assert bad.size == 0, [(int(k), g[k], want[k], bound[k]) for k in bad[:8]]


def test_training_fits_a_separable_rule():
    rng = np.random.default_rng(5)
    n = 20000
    X = _features(rng, n)
    Y = ((X[:, 2] > 0.1) & (X[:, 7] > 0.3)).astype(np.float32)  # moves when the margin is positive
    p = torch.from_numpy(omlp.init_params(1)).cuda()
    losses = lv.louvain_mlp_train(p, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=25, batch=1024,
                                  lr=3e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0], losses
    logit = lv.louvain_mlp_forward(p, torch.from_numpy(X).cuda()).cpu().numpy()
    acc = np.mean((logit > 0) == (Y > 0.5))
    assert acc > 0.95, acc


def test_gradient_and_training_are_reproducible():
    """Per-block partial gradients are summed in block order: two gradients,
    and two training runs with the same seed, agree bit for bit."""
    rng = np.random.default_rng(9)
    n = 50000
    X = torch.from_numpy(_features(rng, n)).cuda()
    Y = torch.from_numpy((rng.random(n) < 0.3).astype(np.float32)).cuda()
    p0 = torch.from_numpy(omlp.init_params(3)).cuda()
    g1, l1 = lv.louvain_mlp_gradient(p0, X, Y)
    g2, l2 = lv.louvain_mlp_gradient(p0, X, Y)
    assert torch.equal(g1, g2) and l1 == l2
    runs = []
    for _ in range(2):
        p = p0.clone()
        losses = lv.louvain_mlp_train(p, X, Y, epochs=3, batch=4096, lr=3e-3, seed=7)
        runs.append((p.cpu().numpy(), losses))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def _traces(g, cap=400000, rate=1.0):
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(trace_capacity=cap, trace_rate=rate)) as ctx:
        ctx.run()
        res = ctx.result()
        X, Y = lv.louvain_traces(ctx.ctx, cap)
    return X, Y, res


def test_traces_are_reproducible():
    """Recorded features depend only on the schedule: two runs give the same
    (canonically ordered) traces, also with concurrent bin kernels."""
    g = gg.rmat(14, 16, seed=21)
    X1, Y1, _ = _traces(g)
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(trace_capacity=400000, trace_rate=1.0)) as ctx:
        ctx.set_schedule(dict(concurrent=1))
        ctx.run()
        X2, Y2 = lv.louvain_traces(ctx.ctx, 400000)
    assert X1.shape[0] > 1000
    assert np.array_equal(X1, X2) and np.array_equal(Y1, Y2)


def test_trace_recording_does_not_change_the_run():
    g = gg.rmat(13, 16, seed=3)
    X, Y, res = _traces(g)
    ref = oracle.louvain(g)
    assert np.array_equal(res.membership, ref.membership)
    assert X.shape[0] > 1000 and X.shape[1] == 8
    assert set(np.unique(Y)) <= {0.0, 1.0}
    assert np.all(X[:, 0] >= 0) and np.all(np.abs(X[:, 2]) <= 1) and np.all((X[:, 7] >= 0) & (X[:, 7] <= 1))


def _trained_model():
    X, Y = [], []
    for sc, seed in ((14, 101), (15, 102)):
        x, y, _ = _traces(gg.rmat(sc, 16, seed=seed))
        X.append(x)
        Y.append(y)
    X = np.concatenate(X)
    Y = np.concatenate(Y)
    p = torch.from_numpy(omlp.init_params(0)).cuda()
    lv.louvain_mlp_train(p, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=8, batch=4096, lr=3e-3)
    return p.cpu().numpy(), float(Y.mean())


def test_learned_skip_run():
    model, pos_rate = _trained_model()
    g = gg.rmat(15, 16, seed=13)
    plain = lv.run(lv.DeviceCSR.from_host(g), lv.Config())
    ref = oracle.louvain(g)
    assert np.array_equal(plain.membership, ref.membership)
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(mode=lv.MODE_LEARNED, model=model,
                                                         skip_threshold=0.5)) as ctx:
        ctx.run()
        res = ctx.result()
        st = ctx.stats()
    # the learned run is a valid partition whose modularity the oracle confirms
    q, num, den = oracle.modularity(g, res.membership)
    assert (num, den) == (res.q_num, res.q_den)
    assert abs(res.modularity - plain.modularity) <= 1e-3, (res.modularity, plain.modularity)
    # every pass ends with a full plain sweep phase
    for learned_it, fallback_it, last_moves in st["learned_passes"]:
        assert fallback_it >= 1
    assert st["skipped"] > 0
    # the zero-move fallback: every pass's last plain iteration made no move
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(mode=lv.MODE_LEARNED, model=model, skip_threshold=0.5,
                                                         learned_fallback=1)) as ctx:
        ctx.run()
        st1 = ctx.stats()
        r1 = ctx.result()
    for learned_it, fallback_it, last_moves in st1["learned_passes"]:
        assert last_moves == 0 or fallback_it == 20
    assert oracle.modularity(g, r1.membership)[1:] == (r1.q_num, r1.q_den)


@pytest.mark.parametrize("schedule", [dict(), dict(concurrent=1)])
def test_stored_predictor_run_rmat22(schedule):
    """The learned form with the stored model and its settings on R-MAT 22
    (hubs of degree above 32768 in both passes, completion steps): a valid
    partition whose exact Q the oracle confirms, within 1e-3 of plain, and
    repeated runs that agree bit for bit."""
    from paper_2501_19004_gb300 import predictor
    g = gg.rmat(22, 16, seed=7)
    dg = lv.DeviceCSR.from_host(g)
    plain = lv.run(dg)
    with lv.Louvain(dg, predictor.default_config()) as ctx:
        ctx.set_schedule(schedule)
        a = ctx.run().result()
        b = ctx.run().result()
        st = ctx.stats()
    assert np.array_equal(a.membership, b.membership) and (a.q_num, a.q_den) == (b.q_num, b.q_den)
    assert st["skipped"] > 0
    assert oracle.modularity(g, a.membership)[1:] == (a.q_num, a.q_den)
    assert abs(a.modularity - plain.modularity) <= 1e-3, (a.modularity, plain.modularity)


def test_untrained_threshold_zero_is_plain_plus_sweeps():
    g = gg.rmat(13, 16, seed=9)
    p = np.zeros(omlp.N_PARAMS, dtype=np.float32)  # logit 0 -> p = 0.5 >= threshold 0.25: nothing skipped
    with lv.Louvain(lv.DeviceCSR.from_host(g), lv.Config(mode=lv.MODE_LEARNED, model=p, skip_threshold=0.25)) as ctx:
        ctx.run()
        st = ctx.stats()
        res = ctx.result()
    assert st["skipped"] == 0
    plain = lv.run(g)
    assert abs(res.modularity - plain.modularity) <= 1e-3


def test_trained_predictor_gains_rmat24():
    """What the stored predictor gains over the plain form on R-MAT scale 24
    (seed 7), at the settings it was trained for.  In the first pass the
    moving phase ends after its second iteration, so what the predictor skips
    there is evaluated again by the completion step; the gain shows from the
    second pass on, whose iterations 1-3 re-evaluate mostly settled hubs.
    Asserted: fewer vertex evaluations over the run, less event-timed
    local-moving time summed over the passes after the first, whole runs no
    more than 5% slower, and a modularity within 1e-3 of the plain result."""
    from paper_2501_19004_gb300 import predictor
    model = predictor.load_default()
    assert model is not None
    g = gg.rmat(24, 16, seed=7)
    dg = lv.DeviceCSR.from_host(g)

    def best(cfg):
        with lv.Louvain(dg, cfg) as ctx:
            ctx.set_schedule(dict(concurrent=1))
            ctx.run()
            runs = []
            for _ in range(3):
                ctx.run()
                runs.append(ctx.stats())
            res = ctx.result()
        later = min(sum(p["move_ms"] for p in st["per_pass"][1:]) for st in runs)
        return min(st["run_ms"] for st in runs), later, runs[-1], res

    t_plain, later_plain, st_plain, plain = best(lv.Config())
    t_learned, later_learned, st_learned, learned = best(predictor.default_config(model))
    assert st_learned["skipped"] > 0
    assert st_learned["evaluated"] < st_plain["evaluated"]
    assert abs(learned.modularity - plain.modularity) <= 1e-3, (learned.modularity, plain.modularity)
    assert later_learned < later_plain, (later_learned, later_plain)
    assert t_learned <= 1.05 * t_plain, (t_learned, t_plain)
