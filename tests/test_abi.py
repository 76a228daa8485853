"""The C-ABI library loads and exports every function include/*.h declares
(no CUDA work: only host-side argument checks are called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(lc_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def so():
    from paper_1401_4441_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lc_create", "lc_bin", "lc_forces", "lc_verlet_step", "lc_energy_virial",
                     "lc_set_state", "lc_get", "lc_destroy", "lc_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing


def test_host_side_argument_checks(so):
    so.lc_status_str.restype = ctypes.c_char_p
    assert so.lc_status_str(0) == b"ok"
    assert b"3 cells" in so.lc_status_str(2)
    box = (ctypes.c_double * 3)(10.0, 10.0, 7.4)
    h = ctypes.c_void_p()
    so.lc_create.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    assert so.lc_create(box, 2.5, 10, 1, ctypes.byref(h)) == 2     # box too small, before any CUDA call
    assert so.lc_create(box, -1.0, 10, 1, ctypes.byref(h)) == 1
    assert so.lc_create(box, 2.5, -1, 1, ctypes.byref(h)) == 1
    assert h.value is None


def test_binding_enums_match_header():
    """The Python binding's schedule, precision, array and status codes are
    the values include/lc.h gives them."""
    text = open(os.path.join(ROOT, "include", "lc.h")).read()
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(LC_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    from paper_1401_4441_gb300 import lc
    for name, v in lc.SCHED.items():
        assert vals[f"LC_SCHED_{name.upper()}"] == v
    for name, v in lc.PREC.items():
        assert vals[f"LC_PREC_{name.upper()}"] == v
    for name, v in lc.GET.items():
        assert vals[f"LC_GET_{name.upper()}"] == v
    for name, v in lc.ORDER.items():
        assert vals[f"LC_ORDER_{name.upper()}"] == v
    for v, name in lc.STATUS.items():
        assert vals[name] == v
    assert len([k for k in vals if k.startswith("LC_SCHED_")]) == len(lc.SCHED)


def test_size_limits_are_checked_on_the_host(so):
    """Sizes beyond the stated maxima are rejected before any device work:
    n >= 2^26 particles, more than 1e9 cells, an invalid 2D box."""
    h = ctypes.c_void_p()
    so.lc_create.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    box = (ctypes.c_double * 3)(100.0, 100.0, 100.0)
    assert so.lc_create(box, 2.5, 1 << 26, 1, ctypes.byref(h)) == 9
    huge = (ctypes.c_double * 3)(1.0e4, 1.0e4, 1.0e4)
    assert so.lc_create(huge, 1.0, 10, 1, ctypes.byref(h)) == 9
    so.lc_create_2d.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    small2 = (ctypes.c_double * 2)(7.4, 100.0)
    assert so.lc_create_2d(small2, 2.5, 10, 1, ctypes.byref(h)) == 2
    assert so.lc_create_2d(None, 2.5, 10, 1, ctypes.byref(h)) == 1
    assert h.value is None


def test_header_is_plain_c_and_links(so, tmp_path):
    """A C99 program that calls the boundary compiles against include/lc.h
    with warnings as errors and links against liblc.so (no C++ in the ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_lc.c"
    src.write_text("""
#include <stdint.h>
#include <stddef.h>
#include "lc.h"
int main(void) {
    const double box[3] = {12.0, 12.0, 12.0};
    lc_ctx *ctx = NULL;
    double pos[3] = {1.0, 1.0, 1.0}, u, k, w;
    int64_t np;
    if (lc_create(box, 2.5, 1, LC_PREC_MIXED, &ctx) != LC_OK) return 1;
    lc_set_state(ctx, pos, NULL, NULL, 0, NULL);
    lc_forces(ctx, LC_SCHED_ATOMIC, NULL);
    lc_verlet_step(ctx, 0.005, 2, LC_SCHED_LIST, NULL);
    lc_energy_virial(ctx, &u, &k, &w, &np, NULL);
    lc_destroy(ctx);
    return 0;
}
""")
    lib = so._name
    out = tmp_path / "use_lc"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        lib, "-o", str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
