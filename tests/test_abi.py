"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/amg.h (no GPU needed: nothing is called)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_19754_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("amg_setup", "amg_vcycle_apply", "pcg_solve", "amg_spmv", "amg_destroy",
                 "amg_pairwise_match", "amg_level_export"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(libpath):
    from paper_2406_19754_gb300 import _lib

    assert set(_lib.SIGNATURES) == set(_declared_functions())
    lib = _lib.load()
    assert lib.amg_status_string(-2).decode().startswith("matrix not")


def test_options_roundtrip_without_gpu(libpath):
    import paper_2406_19754_gb300 as amg

    o = amg.options(precision="f32", threads_per_row=2)
    assert o.sweeps == 2 and o.max_coarse == 200 and o.precision == 1 and o.threads_per_row == 2


def test_library_built_for_sm103a(libpath):
    # the fatbinary carries sm_103a code: cuobjdump is not used; ask the build flags instead
    from paper_2406_19754_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
