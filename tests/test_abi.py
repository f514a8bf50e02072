"""The C ABI library loads and exports every entry point include/*.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(gs_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2410_08743_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("gs_render_forward", "gs_render_backward", "gs_pose_step", "gs_scene_load", "gs_scene_free",
                 "gs_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2410_08743_gb300 import _lib
    assert set(_lib.EXPORTED) <= _declared_functions()


def test_default_opts_and_version_without_gpu(lib):
    from paper_2410_08743_gb300 import _lib
    o = _lib.gs_default_opts()
    assert abs(o.alpha_max - 0.99) < 1e-7 and abs(o.t_min - 1e-4) < 1e-10 and o.flags == 0
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.eps2d - 0.3) < 1e-7 and abs(o.z_near - 0.2) < 1e-7
    assert "sm_103a" in _lib.gs_version()


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2410_08743_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
