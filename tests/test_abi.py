"""The C-ABI library loads and exports every function include/kpsb.h declares (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z][a-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for required in ("kp_build", "sb_solve", "kp_apply", "kp_free", "kpsb_last_error"):
        assert required in names


def test_library_exports_all_declared_symbols():
    from paper_2410_00233_gb300 import build as B
    from paper_2410_00233_gb300 import kpsb as K

    if not os.path.exists(K.LIB_PATH):
        B.build()
    L = K.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert L.kpsb_last_error() is not None


def test_binding_covers_header():
    from paper_2410_00233_gb300 import kpsb as K

    missing = [n for n in _declared() if n not in K._SIGS]
    assert not missing, missing


def test_invalid_arguments_fail_without_touching_the_gpu():
    import numpy as np

    from paper_2410_00233_gb300 import kpsb as K

    with pytest.raises(K.KpsbError) as e:
        K.kp_build(np.ones((3, 3)), 1, K.BC_ZERO, 2, K.EGKB)  # n < 2
    assert e.value.code == -1
    with pytest.raises(K.KpsbError) as e:
        K.kp_build(np.ones((3, 3)), 8, 7, 2, K.EGKB)  # unknown boundary
    assert e.value.code == -1
    with pytest.raises(K.KpsbError) as e:
        K.kp_build(np.ones((3, 3)), 8, K.BC_ZERO, 0.5, K.RSVD)  # RSVD needs a fixed rank
    assert "RSVD" in str(e.value)
    with pytest.raises(K.KpsbError):
        K.kp_build(np.ones((40, 40)), 8, K.BC_REFLEXIVE, 2, K.EGKB)  # overhang > image
    with pytest.raises(K.KpsbError) as e:
        K.kpsb_timer_stats(len(K.TIMER_NAMES) + len(K.TSVD_TIMERS))  # unknown timer category
    assert e.value.code == -1
    with pytest.raises(K.KpsbError) as e:
        K.kp_build(np.ones((3, 3)), 16385, K.BC_ZERO, 2, K.EGKB)  # n above KPSB_MAX_N
    assert e.value.code == -1
    with pytest.raises(K.KpsbError) as e:
        K.kp_dense_blur(np.ones((3, 3)), 200, K.BC_ZERO)  # explicit A limited to n <= 128
    assert e.value.code == -1
    import ctypes

    dummy = (ctypes.c_double * 4)()
    out = ctypes.c_void_p()
    assert K.lib().kp_build_dense(dummy, 200, 3.0, K.EGKB, None, ctypes.byref(out)) == -1  # n > 128
    with pytest.raises(K.KpsbError) as e:
        K.kp_build_dense(np.eye(16), 4, 2.0, K.EGKB, fp64=True)  # explicit operators: SP TSVD only
    assert e.value.code == -1


def test_binding_constants_match_the_header():
    """Every status code and enum value the binding hard-codes equals the header's."""
    from paper_2410_00233_gb300 import kpsb as K

    txt = open(os.path.join(ROOT, "include", "kpsb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    hdr = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(KPSB_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    block = re.search(r"typedef enum \{(.*?)\} kpsb_status;", txt, flags=re.S).group(1)
    status = {int(v): name for name, v in re.findall(r"KPSB_([A-Z0-9_]+)\s*=\s*(-?\d+)", block)}
    assert status == K.STATUS
    for py, c in [("BC_ZERO", "KPSB_BC_ZERO"), ("BC_REFLEXIVE", "KPSB_BC_REFLEXIVE"),
                  ("EGKB", "KPSB_EGKB"), ("RSVD", "KPSB_RSVD"), ("ANISO", "KPSB_ANISO"),
                  ("ISO", "KPSB_ISO"), ("P_FP64", "KPSB_P_FP64"), ("P_FP32", "KPSB_P_FP32"),
                  ("P_TF32X3", "KPSB_P_TF32X3"), ("P_TF32X2", "KPSB_P_TF32X2"),
                  ("P_BF16X3", "KPSB_P_BF16X3"), ("P_BF16X2", "KPSB_P_BF16X2"),
                  ("THR_EXACT", "KPSB_THR_EXACT"), ("THR_PAPER", "KPSB_THR_PAPER"),
                  ("KPSB_OK", "KPSB_OK")]:
        assert getattr(K, py) == hdr[c], py
    assert int(re.search(r"#define KPSB_MAX_N (\d+)", txt).group(1)) == 16384


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the header's structs, as a C compiler lays them out,
    equal the binding's ctypes structures (a C program built against include/kpsb.h)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2410_00233_gb300 import kpsb as K

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("kpsb_build_opts", K.BuildOpts), ("kpsb_sb_opts", K.SBOpts),
             ("kpsb_sb_stats", K.SBStats), ("kpsb_problem", K.Problem), ("kpsb_sb_job", K.SBJob),
             ("kpsb_request", K.Request), ("kpsb_srv_stats", K.SrvStats)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kpsb.h"', "int main(void) {"]
    expect = []
    for cname, cls in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            field = "lambda" if f == "lambda_" else f
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {field}));')
            expect.append(getattr(cls, f).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every entry point raises; there is no fallback path."""
    import numpy as np

    from paper_2410_00233_gb300 import kpsb as K

    monkeypatch.setattr(K, "_lib", None)
    monkeypatch.setattr(K, "LIB_PATH", str(tmp_path / "libkpsb.so"))
    with pytest.raises(RuntimeError, match="missing"):
        K.kp_build(np.ones((3, 3)) / 9, 8, K.BC_ZERO, 2, K.EGKB)
    with pytest.raises(RuntimeError, match="missing"):
        K.kpsb_kernel_launches()


def test_package_never_imports_the_oracle():
    """The product package (binding, inputs, cost model, sharding, build) has no import of
    oracle/: the oracle is test infrastructure only."""
    import ast

    pkg = os.path.join(ROOT, "paper_2410_00233_gb300")
    for f in sorted(os.listdir(pkg)):
        if not f.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, f)).read())
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (f, names)
