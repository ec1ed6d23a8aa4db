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



def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of rihf_options and rihf_shell, as a C
    compiler lays them out from include/rihf.h, against the binding's ctypes
    structures (a field added on one side only shifts everything after it)."""
    import ctypes
    from paper_2407_19614_gb300 import rihf as R
    structs = {"rihf_options": R.rihf_options, "rihf_shell": R.rihf_shell}
    lines = []
    for sname, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (sname, sname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (sname, fname, sname, fname))
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "rihf.h"\nint main(void) {\n%s\nreturn 0;\n}\n'
                   % "\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        k, v = line.rsplit(" ", 1)
        got[k] = int(v)
    for sname, cls in structs.items():
        assert got["%s size" % sname] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got["%s %s" % (sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_enums_match_the_header():
    """The matrix selectors, error codes and precision values of the binding
    against the enums of include/rihf.h."""
    from paper_2407_19614_gb300 import rihf as R
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"\b(RIHF_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    mats = {k[len("RIHF_MAT_"):]: v for k, v in enum.items() if k.startswith("RIHF_MAT_")}
    assert mats == R.MAT
    assert enum["RIHF_OK"] == 0 and enum["RIHF_ERR_STATE"] == -7
    assert enum["RIHF_PRECISION_FP64"] == 0 and enum["RIHF_PRECISION_MIXED"] == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2407_19614_gb300 import rihf as R
    monkeypatch.setattr(R, "_lib", None)
    with pytest.raises(RuntimeError, match="librihf.so not found"):
        R.load(str(tmp_path / "librihf.so"))


def test_no_cpu_fallback_without_a_device(libpath):
    """Without a usable CUDA device the setup call returns a CUDA error: the
    library has no CPU path to fall back to."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2407_19614_gb300 import rihf as R
    from paper_2407_19614_gb300 import workloads as W
    R.load(libpath)
    with pytest.raises(R.RihfError, match="CUDA"):
        R.Context(W.water_monomer(0))
