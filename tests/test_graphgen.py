"""The seeded input generators (the input recipe of the benchmark and the
parity tests).  They hold none of the method's arithmetic; what they must
guarantee is checked here: valid symmetric CSR, results independent of the
thread count, the batched union equal to the single graphs, and the
structure each recipe states."""
import hashlib
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2501_19004_gb300 import graphgen as gg  # noqa: E402


def check_csr(g, weighted):
    off, col = g.offsets, g.cols
    assert off[0] == 0 and off[-1] == g.nnz == col.shape[0]
    assert np.all(np.diff(off) >= 0)
    assert col.min(initial=0) >= 0 and col.max(initial=-1) < g.n
    row = np.repeat(np.arange(g.n), np.diff(off))
    assert not np.any(row == col), "self-loop"
    # rows sorted and deduplicated
    same_row = row[1:] == row[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    # symmetric, with equal weights both ways
    key = row.astype(np.int64) * g.n + col
    rkey = col.astype(np.int64) * g.n + row
    order, rorder = np.argsort(key), np.argsort(rkey)
    assert np.array_equal(key[order], rkey[rorder])
    if weighted:
        assert g.weights is not None and g.weights.min() >= 1
        assert np.array_equal(g.weights[order], g.weights[rorder])
    else:
        assert g.weights is None


def test_generators_give_valid_symmetric_csr():
    check_csr(gg.rmat(11, 16, seed=7), False)
    check_csr(gg.rmat(10, 8, seed=3, weight_range=(1, 5)), True)
    check_csr(gg.grid(40, 0.02, seed=2), True)
    check_csr(gg.sbm(800, 100, 0.1, 0.01, seed=1), False)
    check_csr(gg.sbm(6000, 50, 0.2, 0.001, seed=2), False)  # geometric skipping
    check_csr(gg.ring_of_cliques(4, 5), False)
    check_csr(gg.batched_sbm(3), False)


def _digest_script():
    return ("import hashlib, sys; sys.path.insert(0, %r)\n"
            "from paper_2501_19004_gb300 import graphgen as gg\n"
            "h = hashlib.sha256()\n"
            "for g in (gg.rmat(13, 16, seed=5), gg.grid(96, 0.02, seed=4), gg.sbm(9000, 50, 0.2, 0.002, seed=6),\n"
            "          gg.batched_sbm_union(12)[0]):\n"
            "    h.update(g.offsets.tobytes()); h.update(g.cols.tobytes())\n"
            "    h.update(g.weights.tobytes() if g.weights is not None else b'-')\n"
            "print(gg.num_threads(), h.hexdigest())\n" % ROOT)


def test_results_do_not_depend_on_the_thread_count():
    out = []
    for t in ("1", "3"):
        r = subprocess.run([sys.executable, "-c", _digest_script()], capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, OMP_NUM_THREADS=t))
        assert r.returncode == 0, r.stderr[-1000:]
        nthreads, digest = r.stdout.split()
        assert nthreads == t
        out.append(digest)
    assert out[0] == out[1]


def test_batched_union_equals_the_single_graphs():
    union, vo = gg.batched_sbm_union(10, first=5)
    ref, rvo = gg.concat([gg.batched_sbm(k) for k in range(5, 15)])
    assert np.array_equal(vo, rvo)
    assert np.array_equal(union.offsets, ref.offsets) and np.array_equal(union.cols, ref.cols)


def test_grid_structure():
    side = 30
    g = gg.grid(side, 0.0, seed=1)  # no long-range pairs: the plain 4-neighbour grid
    assert g.n == side * side and g.nnz == 4 * side * (side - 1)
    deg = np.diff(g.offsets)
    assert deg.max() == 4 and deg.min() == 2 and np.sum(deg == 2) == 4  # corners
    assert g.weights.min() >= 1 and g.weights.max() <= 8
    h = gg.grid(side, 0.02, seed=1)
    extra = (h.nnz - g.nnz) // 2
    assert 0 < extra <= int(round(0.02 * 2 * side * (side - 1))) + 1  # deduplicated long-range pairs


def test_sbm_edge_counts_match_the_planted_probabilities():
    """Direct draws and geometric skipping both give Binomial edge counts
    (within 5 standard deviations) inside and between the blocks."""
    n, block, p_in, p_out = 6000, 100, 0.08, 0.002
    for direct in (True, False):
        g = gg.sbm(n, block, p_in, p_out, seed=9, direct=direct)
        row = np.repeat(np.arange(n), np.diff(g.offsets))
        inside = np.sum(row // block == g.cols // block) // 2
        between = g.nnz // 2 - inside
        pairs_in = (n // block) * block * (block - 1) // 2
        pairs_out = n * (n - 1) // 2 - pairs_in
        for got, pairs, p in ((inside, pairs_in, p_in), (between, pairs_out, p_out)):
            mean, sd = pairs * p, np.sqrt(pairs * p * (1 - p))
            assert abs(got - mean) <= 5 * sd, (direct, got, mean, sd)


def test_rmat_is_skewed_and_seeded():
    a, b = gg.rmat(14, 16, seed=7), gg.rmat(14, 16, seed=7)
    assert np.array_equal(a.cols, b.cols)
    c = gg.rmat(14, 16, seed=8)
    assert not (a.nnz == c.nnz and np.array_equal(a.cols, c.cols))
    deg = np.diff(a.offsets)
    assert deg.max() > 20 * deg[deg > 0].mean()  # heavy-tailed degrees
    assert np.sum(deg == 0) > 0                  # isolated vertices, as the recipe states
