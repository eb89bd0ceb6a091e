"""The C-ABI library loads and exports every entry point its header declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dwos.h")


@pytest.fixture(scope="module")
def libdwos():
    from paper_2405_12964_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dwos_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["dwos_create", "dwos_set_boundary", "dwos_eval", "dwos_vjp", "dwos_grad_l2", "dwos_walk_records"]:
        assert n in names


def test_library_exports_every_declared_symbol(libdwos):
    for name in declared_functions():
        assert hasattr(libdwos, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2405_12964_gb300 import dwos
    assert set(declared_functions()) == set(dwos.exported_symbols())


def test_default_options_and_null_context_errors(libdwos):
    from paper_2405_12964_gb300 import dwos
    L = dwos.lib()
    o = dwos.Options()
    L.dwos_default_options(ctypes.byref(o))
    assert abs(o.eps - 1e-3) < 1e-9 and abs(o.h - 1e-2) < 1e-9
    assert (o.K, o.B, o.max_steps, o.seed, o.check_inside) == (1, 8, 16384, 0x12964, 1)
    assert L.dwos_set_options(None, ctypes.byref(o)) == 1
    assert L.dwos_eval(None, 0, None, 1, None, None, None, None, 0) == 1
    assert L.dwos_last_error(None)


def test_record_layouts_match_the_header():
    from paper_2405_12964_gb300 import dwos
    assert dwos.RECORD_DTYPE.itemsize == 32
    assert dwos.DEBUG_DTYPE.itemsize == 48
    assert ctypes.sizeof(dwos.Options) == 56
    # the library's defaults land in the binding's fields (same layout on both sides)
    o = dwos.Options()
    dwos.lib().dwos_default_options(ctypes.byref(o))
    assert o.K == 1 and o.B == 8 and o.seed == 0x12964 and o.check_inside == 1
    assert o.traversal == -1 and o.dudn_estimator == 0 and o.block_size == 0


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2405_12964_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "liboracle" not in src, f
