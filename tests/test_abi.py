"""The C ABI library builds, loads and exports every function include/mm.h
declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w \*]*?\b(mm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1912_13282_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "mm_rbffd_weights" in names and "mm_knn_stencils" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1912_13282_gb300 import binding
    assert sorted(binding.EXPORTS) == sorted(declared_functions())


def test_binding_constants_match_the_header():
    """Every integer #define of include/mm.h that the binding mirrors (same
    name, with or without the MM_ prefix) has the same value there."""
    from paper_1912_13282_gb300 import binding
    text = open(os.path.join(ROOT, "include", "mm.h")).read()
    defines = dict((k, int(v)) for k, v in re.findall(r"^#define\s+(MM_\w+)\s+\(?(-?\d+)\)?", text, flags=re.M))
    checked = 0
    for name, value in defines.items():
        for alias in (name, name[3:]):
            if hasattr(binding, alias):
                assert getattr(binding, alias) == value, (name, alias)
                checked += 1
                break
    assert checked >= 20 and "MM_OPT_WIDE" in defines and binding.OPT_WIDE == defines["MM_OPT_WIDE"]
