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
    # every default the library writes lands in the binding's field of that name:
    # the ctypes layout matches include/amg.h to the last member
    d = amg.options()
    assert (d.max_levels, d.stall_ratio, d.max_dense, d.tail_rows) == (30, 0.9, 8192, 1024)
    assert (d.smooth_sweeps, d.variable_cycle, d.coarse_solver) == (1, 0, 0)
    assert (d.coarse_maxit, d.coarse_tol, d.compress_columns) == (40, 1e-4, 0)
    assert (d.smooth_prolongator, d.aggregation) == (0, 0)
    assert (d.vbm_theta, d.prolongator_filter, d.stream_ring) == (0.01, 0.0, 1)
    v = amg.options(aggregation="vbm", vbm_theta=0.2, prolongator_filter=0.05)
    assert (v.aggregation, v.vbm_theta, v.prolongator_filter) == (1, 0.2, 0.05)


def test_library_built_for_sm103a(libpath):
    # the fatbinary carries sm_103a code: cuobjdump is not used; ask the build flags instead
    from paper_2406_19754_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_struct_sizes_match_the_header(tmp_path):
    """The ctypes mirrors of the option and result structs have the C sizes."""
    import ctypes as C
    import shutil
    import subprocess

    from paper_2406_19754_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text('#include "amg.h"\n#include <stdio.h>\nint main(void) {\n'
                   '  printf("%zu %zu %zu\\n", sizeof(amg_options), sizeof(pcg_options),\n'
                   '         sizeof(pcg_stats));\n  return 0;\n}\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(t) for t in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [C.sizeof(_lib.AmgOptions), C.sizeof(_lib.PcgOptions),
                   C.sizeof(_lib.PcgStats)]
