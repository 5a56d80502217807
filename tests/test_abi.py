"""CPU checks of the C ABI: the shared library builds, loads, and exports every
function include/ckks.h declares (no compute call needs a GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "ckks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ckks_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2312_04356_gb300 import build
    so = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    syms = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    names = declared()
    assert len(names) > 50
    missing = [n for n in names if n not in syms]
    assert not missing, missing
    from paper_2312_04356_gb300 import ckks
    lib = ckks.lib()
    for n in names:
        assert hasattr(lib, n)
    # the binding wraps every declared entry point under the same name
    assert set(names) <= set(ckks.exported_symbols())


def test_oracle_and_library_share_no_code():
    """neither side imports, includes or loads the other"""
    import glob
    for f in glob.glob(os.path.join(ROOT, "paper_2312_04356_gb300", "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
            text = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
            assert "libckks_ref" not in text and "ckks_ref.c" not in text, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".c")):
            text = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2312_04356_gb300", text, flags=re.M), f
            assert "libckks_gb300" not in text and "#include" not in text.replace("#include <", ""), f


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_is_plain_c(lang, std):
    """include/ckks.h compiles on its own as pedantic C99 and as C++17 (no torch or CUDA
    types in the signatures; checked for syntax only, nothing is written)"""
    cc = "gcc" if lang == "c" else "g++"
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                        os.path.join(ROOT, "include", "ckks.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_argument_counts_match_the_header():
    """every ctypes signature of the binding has as many arguments as the C declaration"""
    from paper_2312_04356_gb300 import ckks
    src = open(os.path.join(ROOT, "include", "ckks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"^\s*(?:int|const char\*)\s+(ckks_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.M | re.S)
    assert len(decls) == len(declared())
    bad = []
    for name, params in decls:
        params = " ".join(params.split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        if name in ckks._SIGS and len(ckks._SIGS[name]) != n:
            bad.append((name, n, len(ckks._SIGS[name])))
    assert not bad, bad


def _kind_c(param):
    if "*" in param:
        return "ptr"
    t = param.strip().rsplit(" ", 1)[0].replace("const ", "").strip()
    return {"int": "i32", "int32_t": "i32", "double": "f64", "uint64_t": "u64", "int64_t": "i64",
            "ckks_alloc_fn": "ptr", "ckks_free_fn": "ptr"}.get(t, t)


def _kind_py(t):
    import ctypes
    if t is ctypes.c_void_p or t is ctypes.c_char_p or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int: "i32", ctypes.c_double: "f64", ctypes.c_uint64: "u64", ctypes.c_int64: "i64"}.get(t, str(t))


def test_binding_argument_types_match_the_header():
    """pointer, int, double and 64-bit integer positions agree between each C declaration
    and its ctypes signature (a swapped int / double would pass garbage, not fail)"""
    from paper_2312_04356_gb300 import ckks
    src = open(os.path.join(ROOT, "include", "ckks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"^\s*(?:int|const char\*)\s+(ckks_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.M | re.S)
    bad = []
    for name, params in decls:
        params = " ".join(params.split())
        ps = [] if params in ("", "void") else params.split(",")
        for i, (p, t) in enumerate(zip(ps, ckks._SIGS.get(name, []))):
            if _kind_c(p) != _kind_py(t):
                bad.append((name, i, p.strip(), _kind_c(p), _kind_py(t)))
    assert not bad, bad
