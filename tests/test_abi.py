"""The C-ABI library builds, loads and exports every entry point declared in
include/bang.h; argument checks that need no GPU behave as documented."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2401_11324_gb300 as bang
from paper_2401_11324_gb300 import build as bbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|const char \*)\s*(bang_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    bbuild.build()
    return bang.lib()


def test_header_declares_the_api():
    assert {"bang_create", "bang_load_pq", "bang_register_graph", "bang_register_vectors",
            "bang_search", "bang_destroy", "bang_last_error"} <= declared_symbols()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", bbuild.LIB], text=True)
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = declared_symbols() - exported
    assert not missing, missing
    for name in declared_symbols():
        assert hasattr(lib, name)


def test_built_for_sm_103a(lib):
    out = subprocess.check_output(["cuobjdump", "--list-elf", bbuild.LIB], text=True)
    assert "sm_103a" in out


def test_null_and_range_checks_without_gpu(lib):
    ids = (ctypes.c_uint32 * 4)()
    dist = (ctypes.c_float * 4)()
    q = (ctypes.c_float * 4)()
    assert lib.bang_search(None, q, 1, 1, 1, None, ids, dist, None) == bang.BANG_EINVAL
    assert b"NULL" in lib.bang_last_error()
    assert lib.bang_destroy(None) == bang.BANG_OK
    assert lib.bang_create(0, None) == bang.BANG_EINVAL
    assert lib.bang_load_pq(None, 4, 2, None, None, 1) == bang.BANG_EINVAL


def _header_fields(struct):
    """(name, is_pointer, array_length) of each field of a struct in bang.h, in order."""
    src = open(os.path.join(ROOT, "include", "bang.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct, struct), src, re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        for item in decl.split(","):                # "uint32_t k_max, L_max"
            f = re.search(r"(\*?) ?(\w+)(?:\[(\w+)\])?$", item.strip())
            assert f, decl
            out.append((f.group(2), f.group(1) == "*", f.group(3)))
    return out


@pytest.mark.parametrize("struct", ["bang_search_params", "bang_server_config", "bang_autotune_opts",
                                    "bang_autotune_result", "bang_link_probe"])
def test_binding_structs_follow_the_header(struct):
    # the ctypes mirrors of the C structs: same fields, same order, pointers
    # where the header has pointers (a missing or misplaced field would shift
    # every later one)
    want = _header_fields(struct)
    got = getattr(bang, struct)._fields_
    assert [n for n, _, _ in want] == [f[0] for f in got]
    for (name, ptr, _), (_, ctype) in zip(want, got):
        if ptr:
            assert ctype in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(ctype, "contents"), name
        else:
            assert ctype not in (ctypes.c_void_p,), name


def test_host_alloc_aligned_zeroed_and_freed(lib):
    # bang_host_alloc needs no GPU: an anonymous mapping aligned to the
    # transparent-huge-page size, zero-filled; freed once, refused twice
    import numpy as np
    thp = 2 << 20
    try:
        thp = int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except (OSError, ValueError):
        pass
    p = ctypes.c_void_p()
    assert lib.bang_host_alloc(5 << 20, ctypes.byref(p)) == bang.BANG_OK
    assert p.value % thp == 0
    view = np.ctypeslib.as_array((ctypes.c_uint8 * (5 << 20)).from_address(p.value))
    assert not view.any()
    view[:] = 3
    del view
    assert lib.bang_host_free(p) == bang.BANG_OK
    assert lib.bang_host_free(p) == bang.BANG_EINVAL
    assert lib.bang_host_free(None) == bang.BANG_OK
    assert lib.bang_host_alloc(0, ctypes.byref(p)) == bang.BANG_EINVAL
    a = bang.host_empty((300, 7), np.float32)
    assert a.shape == (300, 7) and a.dtype == np.float32 and not a.any()
