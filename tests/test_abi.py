"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/louvain.h declares.  No compute call is made (no GPU needed)."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "louvain.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(louvain_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2501_19004_gb300 import build
    build.build()
    from paper_2501_19004_gb300 import louvain as lv
    return lv.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("louvain_create", "louvain_run", "louvain_modularity", "louvain_memberships", "louvain_destroy",
                 "louvain_stats", "louvain_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_config_defaults_are_the_papers(lib):
    from paper_2501_19004_gb300 import louvain as lv
    c = lv.louvain_config_default()
    assert (c.max_passes, c.max_iterations, c.pickless_period, c.buckets) == (10, 20, 4, 4)
    assert (c.tolerance, c.tolerance_drop, c.aggregation_tolerance) == (0.01, 10.0, 0.8)
    assert lv.louvain_model_size() == 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1
    assert "sm_103a" in lv.louvain_version()


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2501_19004_gb300 import louvain as lv
    with pytest.raises(RuntimeError):
        lv.load(str(tmp_path / "missing.so"))


def test_config_struct_layout_matches_the_header(lib):
    """The binding's louvain_config has the C struct's size: the library's
    louvain_config_default zeroes sizeof(louvain_config) bytes, which must
    end exactly where the binding's struct ends."""
    import ctypes
    from paper_2501_19004_gb300 import louvain as lv
    n = ctypes.sizeof(lv.LouvainConfig)
    buf = (ctypes.c_uint8 * (n + 64))(*([0xAB] * (n + 64)))
    lib.louvain_config_default(ctypes.cast(buf, ctypes.POINTER(lv.LouvainConfig)))
    assert all(b == 0xAB for b in buf[n:]), "the library writes past the binding's struct"
    assert buf[n - 1] != 0xAB, "the binding's struct is longer than the library's"
    c = lv.LouvainConfig.from_buffer(buf)
    assert (c.asynchronous, c.table_window, c.learned_fallback, c.trace_capacity) == (0, 0, 0, 0)
    assert c.max_passes == 10 and c.buckets == 4


def test_binding_has_every_declared_function():
    """The Python binding keeps the C ABI's names: one wrapper per function."""
    from paper_2501_19004_gb300 import louvain as lv
    missing = [n for n in declared_functions() if not hasattr(lv, n)]
    assert not missing, missing
