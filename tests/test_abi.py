"""The C-ABI library builds for sm_103a, loads, and exports what include/fmm.h declares.

No compute call is made here (no GPU): only argument checks that the library
rejects before touching the device.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:int64_t|int|void|const char\s*\*)\s*(fmm_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1203_0889_gb300 import _build
    import paper_1203_0889_gb300 as fmm
    _build.build()
    return fmm.load()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("fmm_build_tree", "fmm_evaluate", "fmm_tree_export", "fmm_tree_destroy", "fmm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_argument_errors(lib):
    import paper_1203_0889_gb300 as fmm
    assert b"sm_103a" in lib.fmm_version()
    out = C.c_void_p()
    # NULL params
    assert lib.fmm_build_tree(None, 10, None, 0, C.byref(out), None) == fmm.FMM_ERR_ARG
    assert b"params" in lib.fmm_last_error()
    bad = [fmm.Params(-1, 64, 0.5, 0, 0, 0), fmm.Params(4, 0, 0.5, 0, 0, 0), fmm.Params(4, 64, 1.5, 0, 0, 0),
           fmm.Params(4, 64, 0.5, 9, 0, 0), fmm.Params(4, 64, 0.5, 0, 256, 0), fmm.Params(21, 64, 0.5, 0, 0, 0),
           fmm.Params(4, 64, 0.0, 0, 0, 0), fmm.Params(4, 64, 0.5, 0, 0, -1),
           fmm.Params(4, 64, 0.5, 0, 0, 0, 4, 0), fmm.Params(4, 64, 0.5, 0, 0, 0, 70000, 0),
           fmm.Params(4, 64, 0.5, 0, 0, 0, 0, -3), fmm.Params(4, 64, 0.5, 0, 0, 0, 0, 5000)]
    for prm in bad:
        assert lib.fmm_build_tree(C.byref(prm), 10, C.c_void_p(8), 0, C.byref(out), None) == fmm.FMM_ERR_ARG
        assert out.value is None
    good = fmm.Params(4, 64, 0.5, 0, 0, 0)
    assert lib.fmm_build_tree(C.byref(good), -5, C.c_void_p(8), 0, C.byref(out), None) == fmm.FMM_ERR_ARG
    assert lib.fmm_build_tree(C.byref(good), 1 << 31, C.c_void_p(8), 0, C.byref(out), None) == fmm.FMM_ERR_ARG
    assert lib.fmm_build_tree(C.byref(good), 10, None, 0, C.byref(out), None) == fmm.FMM_ERR_ARG
    assert lib.fmm_build_tree(C.byref(good), 10, C.c_void_p(8), 7, C.byref(out), None) == fmm.FMM_ERR_ARG
    assert lib.fmm_build_tree(C.byref(good), 10, C.c_void_p(8), 0, None, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_evaluate(None, None, None, None, 0, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_tree_get_info(None, None) == fmm.FMM_ERR_ARG
    assert lib.fmm_status(None) == fmm.FMM_ERR_ARG
    lib.fmm_tree_destroy(None)


def test_stage_names_agree(lib):
    """Stage names of the library, the binding and the header's stage count."""
    import paper_1203_0889_gb300 as fmm
    txt = open(os.path.join(ROOT, "include", "fmm.h")).read()
    nstage = int(re.search(r"#define FMM_NUM_STAGES\s+(\d+)", txt).group(1))
    assert len(fmm.STAGE_NAMES) == nstage
    assert [lib.fmm_stage_name(i).decode() for i in range(nstage)] == list(fmm.STAGE_NAMES)
    assert lib.fmm_stage_name(nstage) == b"" and lib.fmm_stage_name(-1) == b""


def test_flag_values_match_the_header():
    """Every FMM_* flag and precision the binding exports has the header's value."""
    import paper_1203_0889_gb300 as fmm
    txt = open(os.path.join(ROOT, "include", "fmm.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define FMM_(\w+)\s+(-?\d+)", txt)}
    for name in ("OUT_FIELD", "STAGED", "TIMING", "NO_OVERLAP", "BUILD_FALLBACKS", "TASK_GRAPH", "MUTUAL",
                 "LISTS_UVWX", "PREC_FP64", "PREC_FP32_P2P", "PREC_FP32", "PREC_MIXED_TC"):
        assert defs[name] == getattr(fmm, name), name
    flags = [defs[k] for k in ("OUT_FIELD", "STAGED", "TIMING", "NO_OVERLAP", "BUILD_FALLBACKS", "TASK_GRAPH",
                               "MUTUAL", "LISTS_UVWX")]
    assert sorted(flags) == [1 << i for i in range(len(flags))]


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    import paper_1203_0889_gb300 as fmm
    monkeypatch.setattr(fmm, "_lib", None)
    monkeypatch.setattr(fmm, "_LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        fmm.load()


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the sizes and field offsets that a C
    compiler gives the structs of include/fmm.h."""
    import shutil
    import subprocess

    import paper_1203_0889_gb300 as fmm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fmm_params": fmm.Params, "fmm_tree_info": fmm.TreeInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fmm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
