"""Host-side checks of the C ABI: the library builds, loads without a GPU, and exports every function
include/rbs.h declares; the Python binding's structures match the header's field order."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rbs_[a-z_0-9]+)\s*\(", text)))


def struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = [b for b, nm in re.findall(r"typedef struct \{([^{}]*?)\}\s*(\w+);", text, flags=re.S) if nm == name][0]
    return re.findall(r"\b([a-z_]+)\s*(?:\[[A-Z_0-9]+\])?\s*;", body)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs
    return rbs.load()


def test_every_declared_function_is_exported(lib):
    from paper_1606_07428_gb300 import rbs
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(rbs.EXPORTS) == names


def test_binding_structs_follow_header():
    from paper_1606_07428_gb300 import rbs
    assert [f for f, _ in rbs.rbs_options._fields_] == struct_fields("rbs_options")
    assert [f for f, _ in rbs.rbs_stats._fields_] == struct_fields("rbs_stats")


def test_default_options_without_gpu(lib):
    from paper_1606_07428_gb300 import rbs
    o = rbs.rbs_default_options()
    assert o.precision == rbs.RBS_PREC_FP64 and o.restart == 50 and o.preconditioner == 1
    assert o.near_delta == 1.0 and o.p_up_factor == 2 and o.p_self_factor == 2 and o.viscosity == 1.0


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    from paper_1606_07428_gb300 import rbs
    assert lib.rbs_create(None, None) == rbs.RBS_EINVAL
    bad = rbs.rbs_default_options()
    bad.restart = 0
    h = ctypes.c_void_p()
    assert lib.rbs_create(ctypes.byref(bad), ctypes.byref(h)) == rbs.RBS_EINVAL
    assert lib.rbs_set_geometry(None, 1, None, None, None, None, None, None) == rbs.RBS_EINVAL
    assert lib.rbs_mobility_solve(None, None, None, 1e-8, None, None, None, None) == rbs.RBS_EINVAL
    assert lib.rbs_total_nodes(None) == 0
    assert lib.rbs_last_error(None) == b"null context"
