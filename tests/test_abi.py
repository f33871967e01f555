"""The C-ABI library builds, loads and exports every entry point that
include/gs.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import buildlib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gs.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = buildlib.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    names = set(declared_symbols())
    bound = set(gs.SIGNATURES) | set(gs.EXTRA_SIGNATURES)
    assert names <= bound, names - bound
    gs.lib()  # loads with every signature set


def test_struct_layouts_match_the_header():
    # sizes the C compiler gives these structs on LP64 targets
    assert ctypes.sizeof(gs.GraphDesc) == 72
    assert ctypes.sizeof(gs.QueryDesc) == 48
    assert ctypes.sizeof(gs.MatchOpts) == 48
    assert ctypes.sizeof(gs.ResultDesc) == 48
    assert ctypes.sizeof(gs.ServeOpts) == 24
