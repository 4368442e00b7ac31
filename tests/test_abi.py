"""Host-side checks of the C ABI: the library loads, exports every entry point that
include/ib_cav.h declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ib_cav.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:ib_status|void|const char\*|int)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def api():
    from paper_2608_14310_b300 import build
    build.build()
    from paper_2608_14310_b300 import api
    return api


def test_every_declared_symbol_is_exported(api):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(api._lib, n), n
    assert set(names) <= set(api.EXPORTED)


def test_abi_version(api):
    assert api._lib.ib_abi_version() == 5


def test_null_arguments_are_rejected_without_a_device(api):
    out = C.c_void_p()
    st = api._lib.ib_setup(None, None, None, C.byref(out))
    assert st == api.IB_ERR_INVALID and not out.value
    assert "NULL" in api._lib.ib_last_error().decode()
    st = api._lib.cav_setup(None, None, None, C.byref(out))
    assert st == api.IB_ERR_INVALID
    g = api.ib_grid_desc(4, 1.0, 1.0, 0.01, 0.1)   # N below the minimum
    sd = api.ib_structure_desc(0, 1, 0, None, None, 0.0, 0.0, 0.0, 0.0)
    st = api._lib.ib_setup(C.byref(g), C.byref(sd), None, C.byref(out))
    assert st == api.IB_ERR_INVALID and "N must be" in api._lib.ib_last_error().decode()
    g = api.ib_grid_desc(16, 1.0, 1.0, 0.01, 0.1)
    sd = api.ib_structure_desc(10, 1, 1, None, None, 0.1, 0.0, 1.0, 0.0)   # markers missing
    st = api._lib.ib_setup(C.byref(g), C.byref(sd), None, C.byref(out))
    assert st == api.IB_ERR_INVALID
    # boundary conditions: an unknown value is rejected before any device work
    g = api.ib_grid_desc(16, 1.0, 1.0, 0.01, 0.1, 7)
    sd = api.ib_structure_desc(0, 1, 0, None, None, 0.0, 0.0, 0.0, 0.0)
    st = api._lib.ib_setup(C.byref(g), C.byref(sd), None, C.byref(out))
    assert st == api.IB_ERR_INVALID and "boundary" in api._lib.ib_last_error().decode()
    info = api.fgmres_info()
    d = api.fgmres_desc(1e-10, 10, 0, 0)
    st = api._lib.fgmres_solve(None, None, None, None, C.byref(d), C.byref(info), None, None)
    assert st == api.IB_ERR_INVALID


def test_grid_descriptor_layout(api):
    # the binding's struct matches the header: bc follows dt
    g = api.ib_grid_desc
    assert [f for f, _ in g._fields_] == ["N", "L", "rho", "mu", "dt", "bc"]
    assert g.bc.offset == g.dt.offset + 8
    assert api.BC == {"periodic": 0, "channel": 1}


def test_fgmres_descriptor_layout_matches_the_header(api, tmp_path):
    # fgmres_desc.loop (ABI 5) sits where the C compiler puts it
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if cc is None or not os.path.isdir(cuda_inc):
        pytest.skip("no C compiler or CUDA headers")
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ib_cav.h"\n'
                   'int main(void) { printf("%zu %zu %zu", offsetof(fgmres_desc, host_io), '
                   'offsetof(fgmres_desc, loop), sizeof(fgmres_desc)); return 0; }\n')
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc, str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    host_io, loop, size = map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split())
    d = api.fgmres_desc
    assert (d.host_io.offset, d.loop.offset, C.sizeof(d)) == (host_io, loop, size)
    assert api.LOOP == {"host": 0, "device": 1}


def test_product_path_has_no_fallback():
    # the binding refuses to import without the compiled library (checked by reading its source:
    # no other implementation is referenced)
    src = open(os.path.join(ROOT, "paper_2608_14310_b300", "api.py")).read()
    assert "oracle" not in src and "raise ImportError" in src


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header must compile as C99 (and C++), with no torch types
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "ib_cav.h"\nint main(void) { cav_desc c; ib_structure_desc d; (void)c; (void)d;'
                   ' return ib_abi_version(); }\n')
    inc = ["-I" + os.path.join(ROOT, "include")]
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if os.path.isdir(cuda_inc):
        inc.append("-I" + cuda_inc)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", *inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert "torch" not in open(os.path.join(ROOT, "include", "ib_cav.h")).read()
