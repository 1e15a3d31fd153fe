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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the option structs have the sizes and field
    offsets that a C compiler gives the header's structs."""
    import shutil
    import subprocess
    from paper_2604_09419_gb300 import build as B
    B.build()
    from paper_2604_09419_gb300 import line as L
    mirrors = {"line_graph_desc": L.GraphDesc, "line_lr": L.LR, "line_train_opts": L.TrainOpts,
               "line_stats": L.Stats, "line_tune_opts": L.TuneOpts}
    # the C names of the mirrored fields (the binding renames C's "lambda")
    cname = {"lambda_": "lambda"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "line.h"', "int main(void) {"]
    for cs, py in mirrors.items():
        lines.append(f'  printf("{cs} %zu\\n", sizeof({cs}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cs}.{f} %zu\\n", offsetof({cs}, {cname.get(f, f)}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    gcc = shutil.which("gcc") or shutil.which("cc")
    assert gcc, "a C compiler is needed to read the header's layouts"
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    for cs, py in mirrors.items():
        assert int(got[cs]) == ctypes.sizeof(py), cs
        for f, _ in py._fields_:
            assert int(got[f"{cs}.{f}"]) == getattr(py, f).offset, (cs, f)
    o = L.train_opts_default()
    assert o.batch == 4096 and o.alpha_neg == 1.0 and o.mode == L.MODE_BATCHED and o.graph == 1
