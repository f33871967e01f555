"""The C-ABI library builds, loads and exports every entry point that
include/gs.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import buildlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


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


def test_struct_layouts_match_the_header(tmp_path):
    """Sizes and field offsets of the binding's structs equal what the C
    compiler gives the header's structs."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    pairs = [("gs_graph_desc", gs.GraphDesc), ("gs_query", gs.QueryDesc), ("gs_match_opts", gs.MatchOpts),
             ("gs_result", gs.ResultDesc), ("gs_serve_opts", gs.ServeOpts), ("gs_khop_opts", gs.KhopOpts),
             ("gs_cgraph_info", gs.CGraphInfo), ("gs_tuning", gs.Tuning)]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gs.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for cname, py in pairs:
        assert int(got[f"{cname} size"]) == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert int(got[f"{cname} {f[0]}"]) == getattr(py, f[0]).offset, (cname, f[0])


def test_binding_helpers():
    """Host-side marshalling of the binding: projection masks, refinement
    flags, the query pack (same flat arrays as a plain concatenation) and the
    lazy per-query row views of a batch result."""
    import numpy as np
    from paper_1807_08804_gb300 import inputs as I
    assert gs.project_mask(None) == 0 and gs.project_mask([0, 2]) == 5 and gs.project_mask(6) == 6
    assert gs.GS_REFINE_LOW(1) == 1 << 8 and gs.GS_REFINE_LOW(300) == (300 & 0xFF) << 8
    g = I.make_graph(2000, 12000, seed=5)
    qs = I.make_walk_queries(g, 40, 3, 7, seed=6)
    pack = gs._QueryPack(qs)
    for i, f in enumerate(("vtype", "vbind", "esrc", "edst", "erel")):
        want = np.concatenate([np.asarray(getattr(q, f), np.uint32) for q in qs] + [np.zeros(1, np.uint32)])
        np.testing.assert_array_equal(pack.flat[i], want)
    assert [int(d["k"]) for d in pack.desc] == [q.k for q in qs]
    big = np.arange(30, dtype=np.uint32)
    r = gs.MatchResult._view(4, 9, big, 6, 18, 4, 3, True, 0)
    np.testing.assert_array_equal(r.rows, big[6:18].reshape(4, 3))
    assert r.count == 4 and r.truncated and "count=4" in repr(r)
