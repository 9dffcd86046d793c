"""The C ABI library builds for sm_103a and exports every function that
include/warplda.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(warplda_\w+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    from paper_1510_08628_gb300 import _build, warplda
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"warplda_init", "warplda_sweep", "warplda_counts", "warplda_loglik"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared functions
    assert set(warplda._SIGS) == names


def test_binding_raises_without_context():
    from paper_1510_08628_gb300 import warplda
    lib = warplda.load()
    assert lib.warplda_sweep(None, 1) == warplda.EINVAL
    assert b"context" in lib.warplda_last_error()


def test_error_codes_match_the_header():
    """The binding's error constants are the header's WARPLDA_* codes."""
    from paper_1510_08628_gb300 import warplda
    src = open(os.path.join(ROOT, "include", "warplda.h")).read()
    codes = {m.group(1): int(m.group(2))
             for m in re.finditer(r"#define WARPLDA_(OK|E[A-Z]+) \(?(-?\d+)\)?", src)}
    assert {"OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEDOUT", "ESTATE", "EIO", "EBUSY", "EINTERNAL"} <= set(codes)
    for name, value in codes.items():
        assert getattr(warplda, name) == value, name
    assert len(set(codes.values())) == len(codes)
