"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/gx.h declares, and the Python binding mirrors them;
the struct layouts the binding uses match the header's field order; the
product package has no CPU fallback (it never imports the oracle)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gx.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gx_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2506_11320_gb300 import build
    try:
        build.build()
    except RuntimeError as e:      # pragma: no cover - needs nvcc
        pytest.skip(str(e))
    import paper_2506_11320_gb300 as gx
    return gx


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 20
    L = built.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(built.EXPORTED)


def test_status_strings(built):
    L = built.lib()
    assert L.gx_status_string(0) == b"ok"
    assert L.gx_status_string(built.GX_ENOCONV) == b"GMRES did not converge"


def _struct_fields(name):
    src = open(HEADER).read()
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", src)
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.replace(",", " , ").split()
        names = [p for p in parts[1:] if p != ","]
        for nm in names:
            fields.append(re.sub(r"\[.*\]", "", nm))
    return fields


def test_binding_struct_layout_matches_header(built):
    assert [f for f, _ in built.Config._fields_] == _struct_fields("gx_config")
    assert [f for f, _ in built.SolveStats._fields_] == _struct_fields("gx_solve_stats")
    assert [f for f, _ in built.Diag._fields_] == _struct_fields("gx_diag")


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2506_11320_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            tree = ast.parse(open(os.path.join(pkg, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert all(not a.name.startswith("oracle") for a in node.names), f
                if isinstance(node, ast.ImportFrom):
                    assert not (node.module or "").startswith("oracle"), f
    for f in os.listdir(os.path.join(pkg, "csrc")):
        assert "gx_oracle" not in open(os.path.join(pkg, "csrc", f)).read(), f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2506_11320_gb300 as gx
    monkeypatch.setattr(gx, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gx, "_lib", None)
    with pytest.raises(RuntimeError):
        gx.lib()
