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


# ------------------------------------------------------------------ declarations vs binding
_SCALAR = {"int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64, "int32_t": ctypes.c_int32,
           "uint32_t": ctypes.c_uint32, "int": ctypes.c_int, "double": ctypes.c_double, "size_t": ctypes.c_size_t,
           "hsaw_mode": ctypes.c_int, "hsaw_sampling": ctypes.c_int}
_OPAQUE = {"hsaw_graph", "hsaw_walks", "hsaw_server", "hsaw_alloc_fn", "hsaw_free_fn"}


def _strip_comments(text):
    return re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", text, flags=re.S))


def declarations():
    """name -> list of parameter type strings, from every HSAW_API prototype."""
    text = _strip_comments(open(HEADER).read())
    out = {}
    for m in re.finditer(r"HSAW_API\s+[\w\s\*]+?\b(hsaw_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = [p.strip() for p in m.group(2).split(",") if p.strip()]
        if params == ["void"]:
            params = []
        out[m.group(1)] = [re.sub(r"\s*\b\w+$", "", p) if not p.endswith("*") else p for p in params]
    return out


def _kind(ctype):
    """'ptr' for pointers and opaque handles, else the ctypes scalar class."""
    if ctype in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(ctype, type) and issubclass(ctype, ctypes._Pointer)):
        return "ptr"
    return ctype


def test_binding_signatures_match_declarations():
    decl = declarations()
    assert len(decl) == len(declared_symbols())
    for name, params in decl.items():
        args = hs.SIGNATURES[name][1]
        assert len(args) == len(params), (name, params, args)
        for p, a in zip(params, args):
            base = p.replace("const", "").strip()
            if "*" in base or base in _OPAQUE:
                assert _kind(a) == "ptr", (name, p, a)
            else:
                want = _SCALAR[base]
                assert ctypes.sizeof(a) == ctypes.sizeof(want), (name, p, a)
                assert (a(-1).value < 0) == (want(-1).value < 0) or want is ctypes.c_double, (name, p, a)


def _struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    text = _strip_comments(open(HEADER).read())
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = re.sub(r"\[\d+\]", "", decl).strip()  # arrays: keep the name
        if not decl:
            continue
        first, *more = decl.split(",")
        fields.append(re.findall(r"\w+", first)[-1])
        fields += [m.strip(" *") for m in more]
    return fields


def test_structs_match_declarations():
    for cname, pyc in (("hsaw_query", hs.hsaw_query), ("hsaw_result", hs.hsaw_result),
                       ("hsaw_profile", hs.hsaw_profile)):
        assert _struct_fields(cname) == [f for f, _ in pyc._fields_], cname


def test_set_allocator_checks_its_arguments():
    """Installing a scratch allocator needs both callbacks (or neither); the registration
    itself makes no device call."""
    lib = hs.load()
    fa = hs._ALLOC_FN(lambda nbytes, stream, ctx: None)
    fr = hs._FREE_FN(lambda ptr, stream, ctx: None)
    as_ptr = lambda f: ctypes.cast(f, ctypes.c_void_p)  # noqa: E731
    assert lib.hsaw_set_allocator(as_ptr(fa), None, None) == -1
    assert lib.hsaw_set_allocator(None, as_ptr(fr), None) == -1
    assert lib.hsaw_set_allocator(as_ptr(fa), as_ptr(fr), None) == 0
    assert lib.hsaw_set_allocator(None, None, None) == 0
