"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (CPU only: no kernel is launched)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(swe_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_1912_02457_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("swe_create_domain", "swe_set_forcing", "swe_step", "swe_read_state",
              "swe_get_info", "swe_destroy_domain"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (swe_[a-z0-9_]+)", out))
    missing = declared_functions() - exported
    assert not missing, missing


def test_binding_covers_every_symbol(built_lib):
    from paper_1912_02457_gb300 import swe
    L = swe.load(built_lib)
    assert set(swe.SIGNATURES) == declared_functions()
    assert L.swe_abi_version() == 2
    assert L.swe_status_string(-4) == b"non-finite state or time step"
    p = swe.default_params()
    assert p.g == 9.81 and p.theta_mm == 1.3 and p.frs_width == 10


def test_create_rejects_bad_descriptions(built_lib):
    """Host-side validation runs before any CUDA call."""
    import ctypes as C
    from paper_1912_02457_gb300 import swe
    L = swe.load(built_lib)
    d = swe.DomainDesc()
    p = swe.default_params()
    h = C.c_void_p()
    d.nx = 0
    assert L.swe_create_domain(C.byref(d), C.byref(p), None, C.byref(h)) == swe.ERR_INVALID_ARG
    d.nx, d.ny, d.dx, d.dy = 4, 4, 1.0, 1.0
    assert L.swe_create_domain(C.byref(d), C.byref(p), None, C.byref(h)) == swe.ERR_INVALID_ARG
    assert L.swe_step(None, 1) == swe.ERR_INVALID_ARG
    assert h.value is None


def test_binding_structs_match_the_header(tmp_path):
    """Every field of the ctypes mirrors sits where a C compiler puts it
    (gcc on include/swe.h): the parameter, description and info structs
    cross the boundary by pointer."""
    from paper_1912_02457_gb300 import swe
    structs = {"swe_params": swe.Params, "swe_domain_desc": swe.DomainDesc, "swe_info": swe.Info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "swe.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes_sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def ctypes_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)
