"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(bl_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1005_2594_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    declared = _declared()
    assert "bl_step" in declared and "bl_lb_init" in declared
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_1005_2594_gb300 import bloodlb
    declared = _declared()
    assert set(bloodlb.ABI_FUNCTIONS) <= declared
    for name in declared:
        if name in bloodlb.ABI_FUNCTIONS:
            assert hasattr(bloodlb, name), name


def test_struct_layouts_match_header(libpath):
    from paper_1005_2594_gb300 import bloodlb
    # 3 ints + 3 ints + 24 doubles + 2 doubles + 3 doubles + 2 ints
    assert ctypes.sizeof(bloodlb.bl_lb_params) == 6 * 4 + 29 * 8 + 2 * 4
    assert ctypes.sizeof(bloodlb.bl_particle_params) == 12 * 8 + 2 * 4


def test_build_targets_sm103a(libpath):
    from paper_1005_2594_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
