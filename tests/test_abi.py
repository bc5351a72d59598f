"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/viper.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(viper_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("viper_scene_create", "viper_step", "viper_skin", "viper_set_bones", "viper_get_state",
                     "viper_set_state", "viper_sync", "viper_scene_destroy", "viper_error_string"):
        assert required in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no nvcc")
def test_library_builds_and_exports_every_declared_symbol():
    from paper_1906_05260_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.viper_error_string.restype = ctypes.c_char_p
    assert lib.viper_error_string(0) == b"ok"
    assert lib.viper_error_string(-4) == b"state became non-finite"
    # every code the header defines has its own message
    codes = {}
    for line in open(os.path.join(ROOT, "include", "viper.h")):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == "#define" and parts[1].startswith("VIPER_E"):
            codes[parts[1]] = int(parts[2])
    msgs = {name: lib.viper_error_string(code) for name, code in codes.items()}
    assert all(m != b"unknown error" for m in msgs.values()), msgs
    assert len(set(msgs.values())) == len(msgs)
    assert codes["VIPER_ECONTACTS"] == -9


def test_oracle_and_library_share_no_code():
    """The oracle (test infrastructure) and the CUDA library include nothing of each other."""
    csrc = os.path.join(ROOT, "paper_1906_05260_gb300", "csrc")
    for fn in os.listdir(csrc):
        txt = open(os.path.join(csrc, fn)).read()
        assert "oracle" not in txt.lower() and "vo.h" not in txt
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".c", ".h", ".py")):
            txt = open(os.path.join(ROOT, "oracle", fn)).read()
            assert "viper.h" not in txt and "paper_1906_05260_gb300.viper" not in txt
    for fn in ("viper.py", "scenes.py", "build.py", "__init__.py"):
        txt = open(os.path.join(ROOT, "paper_1906_05260_gb300", fn)).read()
        assert "import oracle" not in txt and "from oracle" not in txt


def test_binding_constants_match_the_header():
    """The Python binding's flag, solver and profiling constants carry the
    values include/viper.h defines (the binding passes them through as ints)."""
    text = open(os.path.join(ROOT, "include", "viper.h")).read()
    defs = dict((k, int(v)) for k, v in re.findall(r"#define\s+VIPER_([A-Z0-9_]+)\s+(-?\d+)", text))
    from paper_1906_05260_gb300 import viper as V
    checked = 0
    for name, value in defs.items():
        if name.startswith(("FLAG_", "SOLVER_", "PROF_")) and hasattr(V, name):
            assert getattr(V, name) == value, name
            checked += 1
    for name in ("FLAG_CONTACTS", "FLAG_VOLUME", "FLAG_SURFACE_BENDING", "FLAG_JACOBI", "FLAG_WARM_START",
                 "FLAG_VOLUME_VECTOR", "FLAG_CONTACT_THREADS", "SOLVER_PLAIN", "SOLVER_BATCHED", "SOLVER_FRAME"):
        assert name in defs and hasattr(V, name), name
    assert checked >= 10
