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


def test_create_rejects_bad_arguments_on_the_host(lib_path):
    """sibfa_create checks its arguments before its first CUDA call, so each
    bad argument returns its status here without a GPU: no molecules, an
    unknown precision, a warm-start mode outside 0..6, an unsupported spline order, a grid below 8 points,
    a non-positive cutoff or Ewald exponent, a cutoff plus twice the O-H
    extent above half the box (CUTOFF), and malformed cluster batches
    (periodic, not ending at n_mol, decreasing, an empty cluster, a cluster
    above the 385-molecule bound)."""
    import numpy as np
    import synth
    import paper_2201_00804_gb300 as pkg
    mp = synth.make_cluster(2, seed=1).mp_local
    b = synth.make_box(3, 9.31, seed=1)
    per = dict(mp_local=b.mp_local, periodic=True, box=b.box, rc=2.5, grid=16, ewald_alpha=0.5)
    many = np.repeat(mp[:1], 388, axis=0)
    cases = [
        (dict(mp_local=mp[:0], periodic=False), -1),
        (dict(mp_local=mp, periodic=False, precision=7), -1),
        (dict(mp_local=mp, periodic=False, warm_start=7), -1),
        (dict(mp_local=mp, periodic=False, warm_start=-1), -1),
        (dict(per, order=4), -1),
        (dict(per, grid=(16, 16, 4)), -1),
        (dict(per, rc=0.0), -1),
        (dict(per, ewald_alpha=-1.0), -1),
        (dict(per, box=(9.31, 0.0, 9.31)), -1),
        (dict(per, rc=3.0), -4),      # 3.0 + 2 * 0.9572 > 9.31 / 2
        (dict(mp_local=b.mp_local, periodic=True, box=b.box, rc=2.5, grid=16, cluster_start=[0, 10, 27]), -1),
        (dict(mp_local=mp, periodic=False, cluster_start=[0, 1, 1]), -1),
        (dict(mp_local=mp, periodic=False, cluster_start=[0, 2, 1]), -1),
        (dict(mp_local=np.repeat(mp[:1], 3, axis=0), periodic=False, cluster_start=[0, 2, 2, 3]), -1),
        (dict(mp_local=many, periodic=False, cluster_start=[0, 386, 388]), -1),
    ]
    for kw, status in cases:
        kw = dict(kw)
        with pytest.raises(pkg.SibfaError) as ei:
            pkg.sibfa_create(synth.PARAMS, kw.pop("mp_local"), **kw)
        assert ei.value.status == status, (kw, ei.value)
    # the per-call entry points reject a NULL context before touching it
    lib = pkg.sibfa.load_library()
    assert lib.sibfa_energy_forces(None, None, None, None, None, None) == -1
    assert lib.sibfa_last_stats(None, None, None) == -1
    lib.sibfa_destroy(None)
