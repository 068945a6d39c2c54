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


def test_corrupt_configs_are_refused_before_any_device_work(built):
    # gx_create checks its config before it touches a device, so these run on a
    # host without a GPU: every corrupt field gives GX_EINVAL (a 3D grid beyond
    # the cell limit likewise), never a crash, and the error text names the field.
    L = built.lib()
    nan = float("nan")
    cases = [
        ("n", lambda c: c.n.__setitem__(0, 0), "n[d]"),
        ("dx", lambda c: c.dx.__setitem__(1, -0.1), "dx"),
        ("dx nan", lambda c: c.dx.__setitem__(0, nan), "dx"),
        ("dx inf", lambda c: c.dx.__setitem__(0, float("inf")), "dx"),
        ("c", lambda c: setattr(c, "c", 0.0), "c and dt"),
        ("dt nan", lambda c: setattr(c, "dt", nan), "c and dt"),
        ("dt inf", lambda c: setattr(c, "dt", float("inf")), "finite"),
        ("theta", lambda c: setattr(c, "theta", 0.3), "theta"),
        ("theta nan", lambda c: setattr(c, "theta", nan), "theta"),
        ("restart", lambda c: setattr(c, "gmres_restart", 0), "gmres_restart"),
        ("restart big", lambda c: setattr(c, "gmres_restart", 65), "gmres_restart"),
        ("maxit", lambda c: setattr(c, "gmres_maxit", 0), "gmres_maxit"),
        ("tol", lambda c: setattr(c, "gmres_tol", -1e-8), "gmres_tol"),
        ("tol nan", lambda c: setattr(c, "gmres_tol", nan), "gmres_tol"),
        ("precond", lambda c: setattr(c, "precond", 7), "precond"),
        ("smoothing", lambda c: setattr(c, "ns_j", -1), "smoothing"),
        ("lf_beta nan", lambda c: setattr(c, "lf_beta", nan), "lf_beta"),
        ("lf_beta", lambda c: setattr(c, "lf_beta", -0.5), "lf_beta"),
        ("bin_slack nan", lambda c: setattr(c, "bin_slack", nan), "bin_slack"),
        ("bc_cells", lambda c: setattr(c, "bc_cells", 3), "bc_cells"),
        ("wall", lambda c: setattr(c, "bc_wall", 1), "wall"),
        ("cells", lambda c: (c.n.__setitem__(0, 1 << 16), c.n.__setitem__(1, 1 << 16)), "2^31"),
        ("gl_gamma", lambda c: setattr(c, "gl_gamma", 1.5), "gl_gamma"),
        ("gmres_mixed", lambda c: setattr(c, "gmres_mixed", 2), "gmres_mixed"),
        ("gmres_mixed net", lambda c: (setattr(c, "gmres_mixed", 1), setattr(c, "precond", built.GX_PRECOND_NET)),
         "gmres_mixed"),
    ]
    for name, corrupt, text in cases:
        cfg = built.make_config((16, 8, 1), (0.1, 0.1, 1.0))
        corrupt(cfg)
        h = built._CTX()
        rc = L.gx_create(built.C.byref(cfg), built.C.byref(h))
        assert rc == built.GX_EINVAL, name
        assert not h.value, name
        assert text in L.gx_last_error(None).decode(), (name, L.gx_last_error(None))
    assert L.gx_create(None, None) == built.GX_EINVAL
