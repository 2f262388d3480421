"""C-ABI library checks that need no GPU: it loads, and it exports exactly the
entry points include/tc.h declares (and the Python binding names them)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", text))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("tc_build_csr", "tc_count", "tc_count_batch", "tc_submit", "tc_poll"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2309_09064_gb300 as tc
    path = tc.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (tc_[a-z0-9_]+)$", out, flags=re.M))
    assert declared_functions() == exported
    assert set(tc.EXPORTED) == exported
    for name in exported:
        assert callable(getattr(tc, name))


def test_binding_raises_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2309_09064_gb300 as tc
    with pytest.raises(tc.TcError):
        tc.tc_create(0)


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2309_09064_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text and "liboracle" not in text, f


def test_build_entry_point():
    import __graft_entry__
    __graft_entry__.build()


def test_struct_layouts_match_the_header(tmp_path):
    """Offsets and sizes of tc_options / tc_tuning / tc_stats as gcc lays them
    out from include/tc.h equal those of the ctypes mirrors in the binding."""
    import ctypes
    import paper_2309_09064_gb300 as tc
    structs = {"tc_options": tc.tc_options, "tc_tuning": tc.tc_tuning, "tc_stats": tc.tc_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_every_declaration_is_documented():
    """Each entry point of include/tc.h is preceded by its own comment (arguments, layout, ownership, errors)."""
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    decls = list(re.finditer(r"^(?:tc_status|const char \*|void|int)\s*\*?\s*(tc_[a-z0-9_]+)\s*\(", text, flags=re.M))
    assert len(decls) >= 20
    undocumented = [m.group(1) for m in decls if not text[:m.start()].rstrip().endswith("*/")]
    assert undocumented == []


def test_every_declaration_cites_the_paper_or_says_it_has_no_counterpart():
    """The comment of each entry point names the passage of the paper that defines
    the operation (a section or an algorithm), or states that the paper has none."""
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    decls = list(re.finditer(r"^(?:tc_status|const char \*|void|int)\s*\*?\s*(tc_[a-z0-9_]+)\s*\(", text, flags=re.M))
    missing = []
    for m in decls:
        head = text[:m.start()].rstrip()
        comment = head[head.rfind("/*"):]
        if not re.search(r"Sec\. [IVX]+|Algorithm [1-4]|no counterpart in\s+(?:\*\s*)?the\s+(?:\*\s*)?paper",
                         comment, flags=re.I):
            missing.append(m.group(1))
    assert missing == []
