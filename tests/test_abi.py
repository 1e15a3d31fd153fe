"""The C-ABI library loads and exports every entry point that include/line.h
declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "line.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^LINE_API [^;(]*?\b(line_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2604_09419_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name


def test_binding_mirrors_header():
    from paper_2604_09419_gb300 import build as B
    B.build()
    from paper_2604_09419_gb300 import line as L
    assert sorted(L.EXPORTED) == _declared()


def test_struct_layouts_match_header():
    """The ctypes mirrors of the option structs have the C sizes (x86-64/aarch64 LP64)."""
    from paper_2604_09419_gb300 import build as B
    B.build()
    from paper_2604_09419_gb300 import line as L
    assert ctypes.sizeof(L.GraphDesc) == 40
    assert ctypes.sizeof(L.LR) == 32
    assert ctypes.sizeof(L.TrainOpts) == 64
    assert ctypes.sizeof(L.Stats) == 56
    o = L.train_opts_default()
    assert o.batch == 4096 and o.alpha_neg == 1.0 and o.mode == L.MODE_BATCHED
