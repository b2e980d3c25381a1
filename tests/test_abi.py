"""The C-ABI library builds, loads and exports every symbol include/bd.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_]*\s*\*?\s*(bd_[A-Za-z0-9_]+)\s*\(", src,
                       flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1203_6208_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("bd_plan_create", "bd_plan_destroy", "bd_build_D", "bd_apply_D",
              "bd_eig_bounds", "bd_chebyshev_sqrt", "bd_step", "bd_forces", "bd_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version(libpath):
    from paper_1203_6208_gb300 import binding
    L = binding.load(libpath)
    assert b"sm_103a" in L.bd_version()
    assert L.bd_last_error() == b""
    for n in declared_functions():
        assert hasattr(L, n)


def test_header_is_plain_c():
    """The boundary compiles as C (no C++ or torch types)."""
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = '#include "bd.h"\nint main(void){bd_params p; (void)p; return 0;}\n'
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-x", "c", "-", "-o", os.devnull], input=src, text=True,
                       capture_output=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_binding():
    """The ctypes mirrors have the sizes of the C structs."""
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1203_6208_gb300 import binding as b
    src = ('#include <stdio.h>\n#include "bd.h"\nint main(void){printf("%zu %zu %zu %zu",'
           'sizeof(bd_params),sizeof(bd_plan_info),sizeof(bd_step_stats),sizeof(bd_step_opts));'
           'return 0;}\n')
    exe = os.path.join(ROOT, "_build_sizes")
    try:
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-x", "c", "-", "-o", exe],
                       input=src, text=True, check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    finally:
        if os.path.exists(exe):
            os.remove(exe)
    assert sizes == [ctypes.sizeof(b.BdParams), ctypes.sizeof(b.BdPlanInfo),
                     ctypes.sizeof(b.BdStepStats), ctypes.sizeof(b.BdStepOpts)]


def test_mesh_fft_rejects_bad_arguments_before_any_device_call(libpath):
    """bd_mesh_fft checks its arguments on the host before it touches the
    device: NULL buffers, B outside 1..65535 and unknown precisions are
    BD_ERR_INVALID / BD_ERR_UNSUPPORTED, and so is an odd mesh size (the
    real-to-complex pass packs two real lines into one complex line)."""
    from paper_1203_6208_gb300 import binding
    L = binding.load(libpath)
    INVALID, UNSUPPORTED = 1, 8      # bd_status codes (include/bd.h)
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails its checks first
    cases = [((8, 1, 0, 0, None, fake), INVALID),
             ((8, 0, 0, 0, fake, ctypes.c_void_p(0x2000)), INVALID),
             ((8, 70000, 0, 0, fake, ctypes.c_void_p(0x2000)), UNSUPPORTED),
             ((8, 1, 7, 0, fake, ctypes.c_void_p(0x2000)), INVALID),
             ((15, 1, 0, 0, fake, ctypes.c_void_p(0x2000)), UNSUPPORTED),
             ((0, 1, 1, 1, fake, ctypes.c_void_p(0x2000)), UNSUPPORTED),
             # even sizes the radix plan refuses (prime factor 7; above 512): the
             # plan is formed before any allocation
             ((14, 1, 0, 0, fake, ctypes.c_void_p(1 << 44)), UNSUPPORTED),
             ((1024, 1, 1, 0, fake, ctypes.c_void_p(1 << 44)), UNSUPPORTED)]
    for args, want in cases:
        assert L.bd_mesh_fft(*args, None) == want, args
        assert L.bd_last_error() != b""
