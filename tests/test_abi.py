"""The C-ABI library builds, loads without a GPU and exports every symbol the
header declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(msa_\w+)\s*\(", text, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    from paper_1704_00878_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1704_00878_gb300 import binding
    assert set(declared_functions()) <= set(binding._SIGS)


def test_oracle_builds_and_is_separate():
    import oracle
    p = oracle.build()
    assert os.path.exists(p)
    src = open(os.path.join(ROOT, "oracle", "msa_oracle.c")).read()
    assert "msa.h" not in src and "paper_1704_00878_gb300" not in src
