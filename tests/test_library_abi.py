"""libtgms loads and exports every entry point declared in include/tgms.h
(CPU only: no call that needs a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tgms.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_07220_gb300 import build, tgms
    if not os.path.exists(tgms.LIB_PATH):
        build.build_library()
    return tgms.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tg_setup", "tg_solve", "tg_destroy", "tg_strerror", "tg_default_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1807_07220_gb300 import tgms
    assert set(declared_functions()) <= set(tgms.SIGNATURES)


def test_host_only_calls(lib):
    from paper_1807_07220_gb300 import tgms
    o = tgms.default_options()
    assert abs(o.eta - 0.2) < 1e-15 and o.m1 == 1 and o.m2 == 1
    assert o.precision == 0 and o.coarse_space == 0 and o.pointer_mode == tgms.PTR_DEVICE
    for code in [0] + list(tgms.ERRORS):
        assert isinstance(tgms.tg_strerror(code), str) and tgms.tg_strerror(code)
    assert lib.tg_default_options(None) == -1
    assert o.learned_k == 4 and o.learned_max_iter == 0 and not o.net and not o.face_profiles


def test_network_shape_matches_the_oracle_layout(lib):
    """tg_mlp_shape (host-only) agrees with the parameter layout of the oracle."""
    from oracle.learned import input_shape, param_layout
    from paper_1807_07220_gb300 import tgms
    for b, k, hidden in ((16, 4, 512), (8, 4, 64), (2, 1, 3)):
        R, C = input_shape(b)
        _, total = param_layout(b, k, hidden)
        assert tgms.tg_mlp_shape(b, k, hidden) == (R * C, k * b, total)
    assert lib.tg_mlp_shape(17, 4, 8, None, None, None) == -1
    assert lib.tg_mlp_shape(16, 9, 8, None, None, None) == -1


def test_structs_match_header_layout():
    """The ctypes mirrors have the field order of the C structs."""
    from paper_1807_07220_gb300 import tgms
    text = open(HEADER).read()
    for struct in (tgms.tg_grid, tgms.tg_options, tgms.tg_report):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct.__name__, struct.__name__), text, re.S)
        fields = re.findall(r"\b(?:const\s+)?(?:int|double|float|tg_mlp)\s*\*?\s*(?:const\s*\*\s*)?([A-Za-z_][^;]*);",
                            re.sub(r"/\*.*?\*/", "", body.group(1), flags=re.S))
        names = [re.sub(r"\[.*\]", "", x).strip() for f in fields for x in f.split(",")]
        assert names == [f for f, _ in struct._fields_], struct.__name__
