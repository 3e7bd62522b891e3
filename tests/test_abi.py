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


def test_struct_layouts_match_header():
    # fo_params: 2 ints, 2 doubles, 4 ints, 2 doubles, int, uint -> 64 bytes with padding
    assert ctypes.sizeof(fo.FoParams) == 64
    assert ctypes.sizeof(fo.FoResult) == 6 * 8 + 8 * 4
    assert ctypes.sizeof(fo.FoProfile) == 8 * 8 * 3 + 8
