"""The C ABI: the library builds for sm_103a, loads, and exports every function include/lgf.h declares.
No compute call is made here (no GPU on the CPU runner)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(lgf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_13213_gb300.build import build_library
    path = build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lgf_table_create", "lgf_table_destroy", "lgf_poisson_solve", "lgf_heat_apply",
                     "lgf_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} missing from liblgf.so"


def test_host_only_calls(lib):
    lib.lgf_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lgf_version()
    lib.lgf_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.lgf_last_error(), bytes)


def test_binding_rejects_bad_arguments_without_touching_the_gpu(lib):
    import paper_2010_13213_gb300.lgf as L
    with pytest.raises(L.LgfError) as e:
        L.lgf_table_create(12, (1, 1, 1))
    assert e.value.status == L.LGF_E_UNSUPPORTED
    with pytest.raises(L.LgfError) as e:
        L.lgf_table_create(16, (1, -1, 1))
    assert e.value.status == L.LGF_E_INVALID_ARG
    mesh = L.Mesh([[[0, 0, 0], [0, 0, 0]]], 16, 1.0)
    with pytest.raises(L.LgfError) as e:
        L.lgf_heat_apply(None, mesh, 1, 1, 2, L.LGF_F64, 0.1)
    assert e.value.status == L.LGF_E_MESH  # duplicate block
