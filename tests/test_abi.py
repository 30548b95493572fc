"""The C-ABI library builds, loads without a GPU and exports every symbol the
public header declares; the product path and the oracle stay separate."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from conftest import ROOT

HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for mt in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(dfa_\w+)\s*\(", src, flags=re.M):
            if "typedef" not in mt.group(0) and "#define" not in mt.group(0):
                names.append(mt.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dfa_build", "dfa_free", "dfa_count", "dfa_find", "dfa_find_status",
                     "dfa_strerror", "dfa_find_workspace_bytes", "dfa_find_host"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1506_08612_gb300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", so], stdout=subprocess.PIPE, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert set(declared_functions()) <= exported


def test_library_host_only_calls():
    """Calls that need no device: argument checks, sizes, strings."""
    import paper_1506_08612_gb300 as dd
    lib = dd._lib
    assert lib.dfa_strerror(dd.DFA_OK) == b"ok"
    assert b"sm_103a" in lib.dfa_version()
    assert lib.dfa_find_workspace_bytes(-1, None) == -1
    assert lib.dfa_find_workspace_bytes(0, None) == 16
    cfg = dd.dfa_config(threads=256, chunk=64)
    assert lib.dfa_find_workspace_bytes(256 * 64 * 10 + 1, ctypes.byref(cfg)) == 8 * (2 + 11)
    h = ctypes.c_void_p()
    assert lib.dfa_build(b"ACGN", 4, ctypes.byref(h)) == dd.DFA_EINVAL
    assert lib.dfa_build(b"ACGT", 0, ctypes.byref(h)) == dd.DFA_EINVAL
    assert lib.dfa_build(b"A" * 65, 65, ctypes.byref(h)) == dd.DFA_EINVAL
    assert lib.dfa_build(None, 4, ctypes.byref(h)) == dd.DFA_EINVAL
    assert lib.dfa_count(None, 10, None, None, None, None) == dd.DFA_EINVAL
    assert lib.dfa_find(None, 10, None, None, 0, None, None, 0, None, None) == dd.DFA_EINVAL
    assert lib.dfa_host_stage_bytes(100, 0) == -1
    lib.dfa_free(None)
    assert lib.dfa_pattern_length(None) == -1


def test_product_does_not_import_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_1506_08612_gb300; "
            "print('oracle' in sys.modules)" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], stdout=subprocess.PIPE, text=True, check=True)
    assert out.stdout.strip() == "False"


def test_sources_share_nothing_with_oracle():
    pkg = os.path.join(ROOT, "paper_1506_08612_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "oracle.c" not in src and "liboracle" not in src, f
    osrc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "#include \"" not in osrc          # the oracle includes no project header


def test_oracle_lib_builds():
    import oracle
    assert os.path.exists(oracle.build())


def test_workspace_covers_every_default_row_length():
    """With no configuration the workspace must hold the staged two-pass
    find of every pattern length: below m = 8 layout 1 with 1024-byte rows
    staging up to 16 u16 end offsets a row, from m = 8 the relaxed layout
    with 768-byte rows keeping a u64 stage mask a row; one tile is 512 rows;
    per tile a u64 total (and 16 u32 walker-warp totals for layout 1), per
    row a u16 count."""
    import paper_1506_08612_gb300 as dd
    n = 3_200_000_000
    need = 0
    for row_bytes, per_row, per_tile in ((1024, 32, 64), (768, 8, 0)):
        tiles = -(-n // (512 * row_bytes))
        need = max(need, 8 * (2 + tiles) + tiles * per_tile + tiles * 512 * (2 + per_row))
    assert dd._lib.dfa_find_workspace_bytes(n, None) >= need


def test_binding_rejects_bad_buffers_before_the_library():
    """The binding hands the library flat ``data_ptr()`` arrays, so it turns
    host tensors where device buffers belong (and device ones where host
    buffers belong), wrong element types, strided views and mismatched list
    lengths into Python errors before any call; the table is never touched."""
    import torch

    import paper_1506_08612_gb300 as dd
    text = torch.zeros(100, dtype=torch.uint8)
    i64 = torch.zeros(4, dtype=torch.int64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_count(text, None, i64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_find(text, None, i64, i64, text)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_find_noalloc(b"ACGT", None, None, i64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_multi_count([text], None, i64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_multi_locate(text, None, [1], i64, text)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_find_status(text, i64, 4)
    # host-buffer calls: element type, layout, list lengths, device stage
    with pytest.raises(TypeError, match="torch.uint8"):
        dd.dfa_find_host(torch.zeros(8, dtype=torch.int32), None, None, text, 1 << 20)
    with pytest.raises(TypeError, match="torch.int64"):
        dd.dfa_find_host(text, None, torch.zeros(8, dtype=torch.int32), text, 1 << 20)
    with pytest.raises(ValueError, match="contiguous"):
        dd.dfa_find_host(text[::2], None, None, text, 1 << 20)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dd.dfa_find_host(text, None, i64, text, 1 << 20)
    with pytest.raises(ValueError, match="2 position buffers for 1 tables"):
        dd.dfa_find_host_multi(text, [None], [i64, i64], text, 1 << 20)
    with pytest.raises(ValueError, match="CPU tensor"):
        dd.dfa_find_host(b"ACGT", None, None, text, 1 << 20)
