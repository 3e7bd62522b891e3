"""The C ABI library loads and exports every symbol the header declares (no GPU needed)."""
import ctypes
import subprocess

import paper_2306_12616_gb300 as fo
from conftest import header_symbols


def test_header_declares_the_documented_calls():
    syms = header_symbols()
    for name in ("fo_spectral_bounds", "fo_chebyshev_coeffs", "fo_density_matrix"):
        assert name in syms
    assert sorted(fo.EXPORTED_SYMBOLS) == syms


def test_library_exports_every_header_symbol(built_library):
    lib = ctypes.CDLL(built_library)
    for name in header_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built_library], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(header_symbols()) <= exported


def test_host_only_calls(built_library):
    assert fo.fo_version().startswith("fermi-gb300")
    assert fo.fo_status_string(0) == "ok"
    assert fo.fo_status_string(4) == "non-finite input"


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, measured by the C compiler."""
    from conftest import ROOT
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fermi.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", f"{ROOT}/include", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return [int(x) for x in out]


def test_struct_layouts_match_header(tmp_path):
    for cls, cname in ((fo.FoParams, "fo_params"), (fo.FoResult, "fo_result"), (fo.FoProfile, "fo_profile")):
        names = [f for f, _ in cls._fields_]
        got = _c_layout(cname, names, tmp_path)
        assert got[0] == ctypes.sizeof(cls), cname
        for f, off in zip(names, got[1:]):
            assert getattr(cls, f).offset == off, (cname, f)
