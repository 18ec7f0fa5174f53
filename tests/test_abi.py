"""The C-ABI library loads and exports every symbol the public header declares (CPU only:
no compute call is made)."""
import ctypes
import subprocess

import pytest


@pytest.fixture(scope="module")
def libmod():
    from paper_1707_04333_gb300 import build_lib, fetdpic
    build_lib.build()
    return fetdpic


def test_header_symbols_exported(libmod):
    syms = libmod.declared_symbols()
    assert "fetdpic_create" in syms and "fetdpic_step" in syms and len(syms) >= 15
    L = libmod.lib()
    for s in syms:
        assert hasattr(L, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", libmod.library_path()], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(syms) <= exported


def test_kernels_target_sm103a(libmod):
    """The library embeds sm_103a device code (checked from the build command, not the binary)."""
    from paper_1707_04333_gb300 import build_lib
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-fmad=false" in build_lib.CU_SOURCES["kernels_fp64.cu"]


def test_invalid_arguments_rejected_without_gpu(libmod):
    """Argument validation happens before any device work."""
    L = libmod.lib()
    h = ctypes.c_void_p()
    assert L.fetdpic_create(ctypes.byref(h), None, 1, None) == libmod.EINVAL
    assert L.fetdpic_create(None, None, 0, None) == libmod.EINVAL
    assert L.fetdpic_step(None, 1, 0) == libmod.EINVAL
    assert L.fetdpic_sync(None) == libmod.EINVAL
    assert L.fetdpic_set_probes(None, 0, None, None, 0) == libmod.EINVAL
    assert L.fetdpic_read_probes(None, None, 0, None, None) == libmod.EINVAL
    assert L.fetdpic_solve_electrostatic(None, 0, None, None) == libmod.EINVAL
    assert L.fetdpic_set_external_profile(None, 0, None) == libmod.EINVAL
    assert L.fetdpic_set_external_amplitude(None, 0, 1.0) == libmod.EINVAL
    assert L.fetdpic_last_error(None) == b"null context"


def test_header_is_plain_c99(libmod):
    """A C program that uses only include/fetdpic.h compiles as strict C99 and links against the
    library (no C++ or CUDA types at the boundary); it runs in tests/test_gpu_c_abi.py."""
    import os
    import subprocess
    import tempfile
    from paper_1707_04333_gb300 import build_lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(build_lib.LIB)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "c_abi_roundtrip")
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                            "-I", os.path.join(root, "include"), os.path.join(root, "tests", "c_abi_roundtrip.c"),
                            "-L", libdir, "-lfetdpic", f"-Wl,-rpath,{libdir}", "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        assert os.path.exists(exe)
