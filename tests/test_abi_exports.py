"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/rihf.h declares (no device calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rihf.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rihf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2407_19614_gb300 import build
    path = build.LIB
    if not os.path.exists(path):
        build.build()
    return path


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rihf_setup", "rihf_scf", "rihf_gradient", "rihf_destroy", "rihf_update_geometry"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rihf_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_matches_header(libpath):
    from paper_2407_19614_gb300 import rihf as R
    lib = R.load(libpath)
    for n in _declared():
        assert hasattr(lib, n)
    assert set(R.EXPORTS) <= set(_declared())
    # host-only entry points work without a device
    assert lib.rihf_strerror(-4) == b"SCF not converged"
    o = R.default_options()
    assert o.diis_size == 8 and o.pure == 1
    assert o.cuda_graphs == 1 and o.confirm_fp64 == 0   # the struct's tail matches the header

