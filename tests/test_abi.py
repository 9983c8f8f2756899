"""The C-ABI library loads here (no GPU) and exports every entry point that
include/slar.h declares; no compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "slar.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:slar_status|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_29027_b300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("init_ht", "sl_step", "ht_truncate", "moments", "lomac_correct", "poisson_field"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2606_29027_b300 import slar
    assert sorted(slar.EXPORTED) == _declared()


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the sizes a C compiler gives them."""
    import subprocess
    import tempfile
    from paper_2606_29027_b300 import slar
    src = ('#include "slar.h"\n#include <stdio.h>\nint main(){printf("%zu %zu %zu\\n",'
           'sizeof(slar_config),sizeof(slar_stats),sizeof(slar_ht_view));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        with open(c, "w") as f:
            f.write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(slar.Config), ctypes.sizeof(slar.Stats),
                                     ctypes.sizeof(slar.HTView)]
