"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/iblb.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(iblb_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "iblb_create" in names and "iblb_step" in names and len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_2305_18919_gb300 import binding
    lib = ctypes.CDLL(binding.lib()._name)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding's table covers the same surface
    assert set(binding.SIGNATURES) == set(declared_functions())


def test_struct_layouts_match_header():
    from paper_2305_18919_gb300 import binding
    # iblb_lattice_desc: 6 int32 + 2 doubles + 9 doubles; iblb_iface_params: 6 doubles + 2 int32
    assert ctypes.sizeof(binding.iblb_lattice_desc) == 6 * 4 + 11 * 8
    assert ctypes.sizeof(binding.iblb_iface_params) == 6 * 8 + 2 * 4


def test_invalid_descriptions_rejected_before_any_device_work():
    """Argument validation happens on the host, so it answers the same with or without a GPU."""
    from paper_2305_18919_gb300 import binding
    L = binding.lib()
    h = ctypes.c_void_p()
    for kw in (dict(nx=6), dict(tau=0.5), dict(precision=7), dict(nz=2), dict(rho0=0.0)):
        d = binding.iblb_lattice_desc()
        d.nx, d.ny, d.nz, d.precision, d.tau, d.rho0 = 8, 8, 8, 2, 1.0, 1.0
        for k, v in kw.items():
            setattr(d, k, v)
        assert L.iblb_create(ctypes.byref(d), None, ctypes.byref(h)) == binding.IBLB_EINVAL
    d = binding.iblb_lattice_desc()
    d.nx, d.ny, d.nz, d.precision, d.tau, d.rho0 = 8, 8, 8, 2, 1.0, 1.0
    d.wall_u_bottom[2] = 0.01  # wall-normal wall velocity is not a tangential wall
    assert L.iblb_create(ctypes.byref(d), None, ctypes.byref(h)) == binding.IBLB_EINVAL
    assert L.iblb_step(None, 1) == binding.IBLB_EINVAL
    assert L.iblb_last_error(None) == b"null context"


def test_no_gpu_fails_loudly():
    """Without a usable CUDA device the library reports an error; it never computes on the CPU."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2305_18919_gb300 import binding
    with pytest.raises(binding.IBLBError):
        binding.Lattice(8, 8, 8, 1.0)


def test_header_is_plain_c():
    """include/iblb.h compiles as C99 and as C++ without warnings: the ABI uses plain C types
    only (no torch or C++ types in the signatures)."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "iblb.h")
    for cc, args in (("gcc", ["-std=c99", "-x", "c"]), ("g++", ["-std=c++17", "-x", "c++"])):
        exe = shutil.which(cc)
        if exe is None:
            pytest.skip(f"{cc} not installed")
        r = subprocess.run([exe, *args, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
