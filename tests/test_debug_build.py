"""The debug build (kernels compiled with PT_DEBUG: device-side bounds checks that
report a failing index through a status bit): it builds, its library loads and says it
is the debug build, the normal one says it is not, and the C ABI of both answers a NULL
handle alike.  Nothing here touches a GPU."""

import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2501_05520_gb300 import build as pbuild  # noqa: E402


@pytest.fixture(scope="module")
def libs():
    return pbuild.build(), pbuild.build(debug=True)


def test_debug_library_says_so(libs):
    release, debug = (ctypes.CDLL(p) for p in libs)
    assert release.pt_debug_build() == 0
    assert debug.pt_debug_build() == 1
    for L in (release, debug):
        L.pt_set_fishbone.argtypes = [ctypes.c_void_p, ctypes.c_int]
        assert L.pt_set_fishbone(None, 1) == 1  # PT_ERR_INVALID


def test_environment_selects_the_debug_library(libs):
    code = ("import paper_2501_05520_gb300 as pt; import os; "
            "print(os.path.basename(pt.LIB_PATH), pt.lib().pt_debug_build())")
    for env, want in (({"PT_DEBUG": "1"}, "libptca_debug.so 1"), ({}, "libptca.so 0")):
        e = dict(os.environ)
        e.pop("PT_DEBUG", None)
        e.update(env)
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=e, capture_output=True,
                             text=True, check=True).stdout.strip()
        assert out == want
