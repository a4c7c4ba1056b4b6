"""The C-ABI library builds for sm_103a and exports every entry point that
include/lnf.h declares (no GPU needed: nothing is called)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:lnf_status|void|char|double|int)\s*\*?\s*(lnf_\w+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1807_03119_gb300 import builder
    return builder.build()


def exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    return {line.split()[-1] for line in out.splitlines() if " T " in line}


def test_header_declares_the_boundary():
    names = declared()
    for must in ("lnf_create", "lnf_destroy", "lnf_filter_volume", "lnf_entropy", "lnf_submit", "lnf_poll",
                 "lnf_filter_batch", "lnf_filter_multi", "lnf_filter_multi_host"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    missing = declared() - exported(libpath)
    assert not missing, f"declared in include/*.h but not exported: {sorted(missing)}"


def test_library_loads_without_gpu(libpath):
    import ctypes
    try:
        lib = ctypes.CDLL(libpath)
    except OSError as e:   # the CUDA runtime itself is missing on this machine
        pytest.skip(f"cannot dlopen: {e}")
    lib.lnf_version.restype = ctypes.c_char_p
    assert lib.lnf_version().startswith(b"lnf")


def test_oracle_builds_and_loads():
    import oracle
    oracle.build()
    assert oracle.lib() is not None


@pytest.mark.parametrize("spec", ["bogus", "output@0", "launch@x", "stage@", "resident,nope@2", "output@-1"])
def test_fault_spec_is_checked_before_any_device_call(libpath, monkeypatch, spec):
    """An LNF_FAULT list naming an unknown site or a bad count makes lnf_create
    fail with LNF_EINVAL, before it touches the device."""
    import ctypes
    try:
        lib = ctypes.CDLL(libpath)
    except OSError as e:
        pytest.skip(f"cannot dlopen: {e}")
    monkeypatch.setenv("LNF_FAULT", spec)
    h = ctypes.c_void_p()
    assert lib.lnf_create(None, ctypes.byref(h)) == 1
    assert not h.value


def test_spacing_radii_match_the_oracle(libpath):
    """lnf_spacing_radii (host code of the library, no device call) against the
    oracle's own rounding of extent / spacing, on random and half-way cases."""
    import ctypes
    import random
    import oracle
    try:
        lib = ctypes.CDLL(libpath)
    except OSError as e:
        pytest.skip(f"cannot dlopen: {e}")
    lib.lnf_spacing_radii.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    rng = random.Random(5)
    cases = [(1.5, (1.0, 3.0, 0.5)), (2.5, (1.0, 1.0, 1.0)), (0.0, (1.0, 2.0, 3.0))]
    cases += [(rng.uniform(0, 6), tuple(rng.uniform(0.3, 4.0) for _ in range(3))) for _ in range(500)]
    for extent, spacing in cases:
        out = (ctypes.c_int * 3)()
        rc = lib.lnf_spacing_radii(extent, (ctypes.c_double * 3)(*spacing), out)
        want = oracle.spacing_radii(extent, spacing)
        if max(want) > 8:
            assert rc == 1
        else:
            assert rc == 0 and tuple(out) == want, (extent, spacing)
    for bad in ((1.0, (0.0, 1.0, 1.0)), (-1.0, (1.0, 1.0, 1.0)), (float("inf"), (1.0, 1.0, 1.0))):
        assert lib.lnf_spacing_radii(bad[0], (ctypes.c_double * 3)(*bad[1]), (ctypes.c_int * 3)()) == 1
