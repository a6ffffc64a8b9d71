"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point that
include/nnsort.h declares (no compute calls here). CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nnsort.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nnsort_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1907_08817_gb300 import build as b
    return b.build()


def test_library_exports_every_declared_entry_point(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_header(libpath):
    from paper_1907_08817_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()
    L = _lib.lib()
    assert L.nnsort_version() == 10000
    assert L.nnsort_strerror(-2) == b"NaN key"


def test_struct_layouts_match_header(libpath):
    """Defaults written by the library land in the fields the binding reads."""
    from paper_1907_08817_gb300 import _lib
    L = _lib.lib()
    o = _lib.SortOpts()
    L.nnsort_default_sort_opts(ctypes.byref(o))
    assert (o.m, o.eps, o.tau, o.precision, o.bucket_log2, o.no_sync) == (1.25, 3, 1024, 0, 0, 0)
    assert o.d_slots is None and o.d_fate is None
    t = _lib.TrainOpts()
    L.nnsort_default_train_opts(ctypes.byref(t))
    assert (t.layers, t.h1, t.h2, t.sample_n, t.steps, t.batch, t.seed) == (1, 32, 0, 10000, 100, 0, 0)
    assert abs(t.lr - 1e-2) < 1e-9 and abs(t.beta2 - 0.999) < 1e-7


def test_workspace_sizing_is_host_logic(libpath):
    from paper_1907_08817_gb300 import _lib
    L = _lib.lib()
    small = L.nnsort_workspace_bytes(1000, 0, 0, None)
    big = L.nnsort_workspace_bytes(10_000_000, 0, 0, None)
    kv = L.nnsort_workspace_bytes(10_000_000, 3, 1, None)
    assert 0 < small < big < kv
    assert L.nnsort_workspace_bytes(10, 9, 0, None) == 0  # bad dtype
