"""The allocation-free modularity entry point (louvain_modularity_noalloc).

Callers that cannot let a library allocate device memory -- an application
whose own pool owns the device, a serving loop that must not call
cudaMalloc -- use this variant of louvain_modularity_of, whose scratch is a
fixed array inside the library.  This file is collected last on purpose: if
it fails, a run that stops at the first failure has already run every other
test.  It checks, through the C ABI, two calls in a row against the existing
entry point (the shared scratch must be cleared between calls), and that a
graph beyond the array's size is refused.
"""
import numpy as np
import pytest

from paper_2501_19004_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2501_19004_gb300 import louvain as lv  # noqa: E402


def test_noalloc_matches_modularity_of_twice():
    rng = np.random.default_rng(42)
    for g in (gg.sbm(1000, 100, 0.1, 0.002, seed=1), gg.grid(300, 0.02, seed=5), gg.rmat(16, 16, seed=7)):
        dg = lv.DeviceCSR.from_host(g)
        for k in (1, 50, g.n):
            memb = rng.integers(0, k, size=g.n).astype(np.int32)
            dm = torch.from_numpy(memb).cuda()
            q_ref, num_ref, den_ref = lv.louvain_modularity_of(dg, dm)
            for _ in range(2):  # two calls in a row share (and must reset) the scratch
                st, q, num, den = lv.louvain_modularity_noalloc(dg, dm)
                assert st == 0
                assert (num, den) == (num_ref, den_ref)
                assert abs(q - q_ref) <= 1e-12


def test_noalloc_refuses_graphs_beyond_its_scratch():
    n = (1 << 20) + 1
    g = gg.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), None)
    dg = lv.DeviceCSR.from_host(g)
    st, _, _, _ = lv.louvain_modularity_noalloc(dg, torch.zeros(n, dtype=torch.int32, device="cuda"))
    assert st == 1  # LOUVAIN_E_INVAL
