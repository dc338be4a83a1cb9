"""The C-ABI library (no GPU needed): it builds in-tree for sm_103a, loads,
and exports every function that include/sibfa.h declares; the Python binding
declares a prototype for each of them and refuses to run without the library
rather than falling back to anything else."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sibfa.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sibfa_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sibfa_create", "sibfa_energy_forces", "sibfa_solve_dipoles", "sibfa_destroy",
                     "sibfa_last_error", "sibfa_cluster_elec_noalloc"):
        assert required in names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2201_00804_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_prototypes(lib_path):
    from paper_2201_00804_gb300 import sibfa
    lib = sibfa.load_library()
    missing = [n for n in declared_functions() if getattr(lib, n).argtypes is None]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2201_00804_gb300 import sibfa
    monkeypatch.setattr(sibfa, "_lib", None)
    with pytest.raises(OSError):
        sibfa.load_library(str(tmp_path / "missing.so"))
