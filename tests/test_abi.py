"""The C ABI library loads and exports every entry point include/knng.h
declares; host-only entry points work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "knng.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const\s+char\s*\*)\s*(knng_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_7852_gb300 import _build, binding
    _build.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_1307_7852_gb300 import binding
    assert set(declared()) <= set(binding.SIGNATURES)


def test_status_strings(lib):
    from paper_1307_7852_gb300 import binding
    L = binding.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, 7):
        assert L.knng_status_string(code)


def test_leaf_layout_matches_oracle(lib):
    from paper_1307_7852_gb300 import binding
    for n, g in [(10000, 64), (1000000, 256), (1000000, 512), (12345, 37), (5, 8), (301, 150)]:
        off = binding.knng_leaf_offsets(n, g)
        assert binding.knng_leaf_count(n, g) == oracle.leaf_count(n, g) == len(off) - 1
        assert off[0] == 0 and off[-1] == n
    X = np.zeros((777, 1), dtype=np.float32)
    np.testing.assert_array_equal(binding.knng_leaf_offsets(777, 20), oracle.partition(X, 0, 0, 20)[1])


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_1307_7852_gb300 import binding
    h = ctypes.c_void_p()
    assert binding.lib().knng_create(ctypes.byref(h), 0) != 0
    with pytest.raises(binding.KnngError):
        binding.Handle(0)
