"""The C-ABI library builds, loads and exports every symbol include/gp.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2412_10789_gb300 import build, gp
    build.build()
    return gp.load_library()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("gp_graph_create", "gp_ppr", "gp_hkpr", "gp_submit", "gp_poll", "gp_graph_destroy",
                 "gp_batch", "gp_power"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def _param_counts():
    """Number of parameters of every function declared in include/*.h."""
    counts = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", h)).read(), flags=re.S)
        for m in re.finditer(r"\b(gp_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
            args = m.group(2).strip()
            if "(" in args:  # a function-pointer member, not a declaration
                continue
            counts[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return counts


def test_binding_signatures_match_the_header(lib):
    counts = _param_counts()
    checked = 0
    for name, n in counts.items():
        f = getattr(lib, name)
        if f.argtypes is None:
            continue
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
        checked += 1
    assert checked >= 20


def test_status_strings_and_defaults(lib):
    from paper_2412_10789_gb300 import gp
    assert gp.gp_status_string(gp.GP_OK) == "GP_OK"
    assert "EINVAL" in gp.gp_status_string(gp.GP_EINVAL)
    cfg = gp.gp_config_default()
    assert cfg.k_max == 96 and cfg.validate_symmetry == 1 and abs(cfg.warmup_tail - 1e-2) < 1e-15


def test_null_arguments_are_rejected_without_gpu(lib):
    from paper_2412_10789_gb300 import gp
    out = ctypes.c_void_p()
    rc = lib.gp_graph_create(4, 0, None, 0, None, None, 0, None, ctypes.byref(out))
    assert rc == gp.GP_EINVAL
    assert "NULL" in gp.gp_last_error()
    assert lib.gp_ppr(None, 0, 0.2, 1e-6, gp.GP_F64, None, 1, None) == gp.GP_EINVAL
    assert lib.gp_graph_destroy(None) == gp.GP_OK


def test_coefficient_engine_is_not_the_oracle():
    # The library and the oracle share no source: no oracle file is compiled into
    # the library and the library's sources never mention the oracle module.
    csrc = os.path.join(ROOT, "paper_2412_10789_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
    for f in ("gp.py", "build.py", "__init__.py"):
        text = open(os.path.join(ROOT, "paper_2412_10789_gb300", f)).read()
        assert "import oracle" not in text and "from oracle" not in text, f
