"""The C-ABI library builds, loads and exports every entry point include/*.h declares (no GPU calls)."""
import ctypes
import glob
import os
import re

from paper_2107_12437_gb300 import build as B
from paper_2107_12437_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_expected_entry_points():
    names = declared_symbols()
    for n in ("pc_ctx_create", "pc_ctx_destroy", "pc_fields", "pc_fields_plane", "pc_dipoles_run", "pc_ke_fit",
              "pc_status_string", "pc_alu_peaks"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header():
    assert declared_symbols() == set(capi.SIGNATURES)


def test_status_strings_without_gpu():
    lib = capi.load()
    for s in range(8):
        assert lib.pc_status_string(s)
