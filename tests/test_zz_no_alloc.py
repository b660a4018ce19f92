"""The allocation-free modularity entry point (louvain_modularity_noalloc).

Callers that cannot let a library allocate device memory -- an application
whose own pool owns the device, a serving loop that must not call
cudaMalloc -- use this variant of louvain_modularity_of, whose scratch is a
fixed array inside the library.  This file is collected last on purpose: if
it fails, a run that stops at the first failure has already run every other
test.  Through the C ABI it checks two calls in a row against the existing
entry point (the shared scratch must be cleared between calls), the largest
graph the array takes, that a second call leaves the device's free memory
unchanged, and that malformed inputs are refused with a status: a graph
beyond the array's size, membership ids out of range, a zero weight, and
offsets that decrease or run past nnz (the kernel checks every row before
it reads it, so these cases read nothing out of bounds).
"""
import numpy as np
import pytest

from paper_2501_19004_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2501_19004_gb300 import louvain as lv  # noqa: E402


def _same_as_modularity_of(dg, dm):
    q_ref, num_ref, den_ref = lv.louvain_modularity_of(dg, dm)
    for _ in range(2):  # two calls in a row share (and must reset) the scratch
        st, q, num, den = lv.louvain_modularity_noalloc(dg, dm)
        assert st == 0
        assert (num, den) == (num_ref, den_ref)
        assert abs(q - q_ref) <= 1e-12


def test_noalloc_matches_modularity_of_twice():
    rng = np.random.default_rng(42)
    for g in (gg.sbm(1000, 100, 0.1, 0.002, seed=1), gg.grid(300, 0.02, seed=5), gg.rmat(16, 16, seed=7)):
        dg = lv.DeviceCSR.from_host(g)
        for k in (1, 50, g.n):
            memb = rng.integers(0, k, size=g.n).astype(np.int32)
            _same_as_modularity_of(dg, torch.from_numpy(memb).cuda())


def test_noalloc_at_its_largest_size():
    g = gg.grid(1024, 0.02, seed=3)  # exactly 1 << 20 vertices: every word of the array is cleared and used
    assert g.n == 1 << 20
    dg = lv.DeviceCSR.from_host(g)
    memb = (np.arange(g.n) // 7).astype(np.int32)
    _same_as_modularity_of(dg, torch.from_numpy(memb).cuda())
    _same_as_modularity_of(dg, torch.arange(g.n, dtype=torch.int32, device="cuda"))


def test_noalloc_allocates_nothing():
    g = gg.rmat(15, 16, seed=5)
    dg = lv.DeviceCSR.from_host(g)
    dm = torch.from_numpy((np.arange(g.n) % 97).astype(np.int32)).cuda()
    assert lv.louvain_modularity_noalloc(dg, dm)[0] == 0  # warm-up: device code loaded, array reserved
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        assert lv.louvain_modularity_noalloc(dg, dm)[0] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_refuses_graphs_beyond_its_scratch():
    n = (1 << 20) + 1
    g = gg.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    dg = lv.DeviceCSR.from_host(g)
    st, _, _, _ = lv.louvain_modularity_noalloc(dg, torch.zeros(n, dtype=torch.int32, device="cuda"))
    assert st == 1  # LOUVAIN_E_INVAL


def test_noalloc_refuses_malformed_inputs():
    g = gg.sbm(200, 50, 0.2, 0.01, seed=4)
    dg = lv.DeviceCSR.from_host(g)
    good = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    assert lv.louvain_modularity_noalloc(dg, good)[0] == 0
    for bad_id in (-1, g.n):
        m = good.clone()
        m[17] = bad_id
        assert lv.louvain_modularity_noalloc(dg, m)[0] == 1
    w = torch.ones(g.nnz, dtype=torch.int32, device="cuda")
    w[5] = 0
    assert lv.louvain_modularity_noalloc(lv.DeviceCSR(dg.offsets, dg.cols, w), good)[0] == 1
    off = dg.offsets.clone()
    off[10], off[11] = off[11].item(), off[10].item()  # rows 9..11 with decreasing offsets
    assert off[10] > off[11]
    assert lv.louvain_modularity_noalloc(lv.DeviceCSR(off, dg.cols), good)[0] == 1
    off = dg.offsets.clone()
    off[-1] += 64  # offsets[n] past nnz
    assert lv.louvain_modularity_noalloc(lv.DeviceCSR(off, dg.cols), good)[0] == 1
    off = dg.offsets.clone()
    off[g.n // 2] = g.nnz + 1000  # one interior row ends far past nnz
    assert lv.louvain_modularity_noalloc(lv.DeviceCSR(off, dg.cols), good)[0] == 1
    # the same inputs, repaired, still give the reference result afterwards
    _same_as_modularity_of(dg, good)
