"""The C-ABI library builds, loads and exports every entry point include/hsaw.h declares.

No compute call is made here (these tests run without a GPU)."""
import ctypes
import os
import re

import paper_1702_05854_gb300 as hs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hsaw.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsaw_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for must in ("hsaw_graph_from_edges", "hsaw_graph_from_csr", "hsaw_solve", "hsaw_sample", "hsaw_histogram",
                 "hsaw_greedy", "hsaw_coverage", "hsaw_stop_constants", "hsaw_check", "hsaw_last_error"):
        assert must in syms


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(hs.build.build())
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(hs.SIGNATURES)


def test_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(hs.build.ARCH)
