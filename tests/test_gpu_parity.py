"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, in the FP64 path (tight) and the mixed path (energy
relative error <= 1e-6, force RMS relative error <= 1e-5, induced-dipole RMS
error <= 1e-6 D)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (FP64_E_REL, FP64_F_RMS_REL, FP64_MU_RMS_D, MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D,
                      compare, run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


_cache = {}


def _ref(key, system, opts):
    if key not in _cache:
        _cache[key] = oracle.evaluate(system, opts, tol_D=1e-11)
    return _cache[key]


def _cases():
    return {
        "cluster8": (synth.make_cluster(8, seed=31), None),
        "cluster2": (synth.make_cluster(2, seed=32), None),
        "water216": synth.make_config("water216"),
        # 512 waters with rc 5 A: three cells per side (cells of rc + 2.6 A of
        # site extents + 0.4 A of list skin), exercises the cell list
        "water512": (synth.make_box(8, 24.83, seed=33), {"rc": 5.0, "grid": 32, "order": 5, "ewald": 0.6}),
        # dipoles of any direction and quadrupoles with off-diagonal entries in
        # every local frame: the full rotation and its torques
        "cluster8_general": (synth.with_general_multipoles(synth.make_cluster(8, seed=31), seed=34), None),
        "water216_general": (synth.with_general_multipoles(synth.make_config("water216")[0], seed=35),
                             synth.make_config("water216")[1]),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_path_matches_oracle(name):
    import paper_2201_00804_gb300 as pkg
    s, o = CASES[name]
    ref = _ref(name, s, o)
    gpu = run_gpu(s, o, pkg.PREC_FP64, 1e-11)
    compare(gpu, ref, FP64_E_REL, FP64_F_RMS_REL, FP64_MU_RMS_D)


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_path_matches_oracle(name):
    import paper_2201_00804_gb300 as pkg
    s, o = CASES[name]
    ref = _ref(name, s, o)
    gpu = run_gpu(s, o, pkg.PREC_MIXED, 1e-8)
    compare(gpu, ref, MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D)


def test_host_and_device_pointers_agree():
    import paper_2201_00804_gb300 as pkg
    s, o = CASES["water216"]
    # FP64 path: only the order of the grid atomics can differ between runs
    a = run_gpu(s, o, pkg.PREC_FP64, 1e-10, device=True)
    for host in (False, "pinned"):   # pageable (staged) and page-locked host buffers
        b = run_gpu(s, o, pkg.PREC_FP64, 1e-10, device=host)
        assert a["terms"]["total"] == pytest.approx(b["terms"]["total"], rel=1e-11)
        np.testing.assert_allclose(a["forces"], b["forces"], rtol=0, atol=1e-8)
        np.testing.assert_allclose(a["mu"], b["mu"], rtol=0, atol=1e-9)


def test_single_molecule_has_no_intermolecular_energy():
    import paper_2201_00804_gb300 as pkg
    s = synth.make_cluster(1, seed=5)
    gpu = run_gpu(s, None, pkg.PREC_FP64, 1e-10)
    for k, v in gpu["terms"].items():
        assert abs(v) < 1e-12, (k, v)
    assert np.abs(gpu["forces"]).max() < 1e-12


def test_results_are_deterministic():
    import paper_2201_00804_gb300 as pkg
    s, o = CASES["water216"]
    a = run_gpu(s, o, pkg.PREC_FP64, 1e-10)
    b = run_gpu(s, o, pkg.PREC_FP64, 1e-10)
    assert a["terms"]["total"] == pytest.approx(b["terms"]["total"], rel=1e-13)


def test_solver_limit_reports_not_converged():
    """A solve stopped by pcg_max_iter returns NOT_CONVERGED (status -3) from
    the device-side loop, and the statistics show the one iteration done."""
    import paper_2201_00804_gb300 as pkg
    s, o = _cases()["water216"]
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=1e-12, pcg_max_iter=1, precision=pkg.PREC_FP64,
                           warm_start=False)
    F = np.zeros(s.n_mol * 9)
    try:
        with pytest.raises(pkg.SibfaError) as ei:
            pkg.sibfa_energy_forces(ctx, s.pos.reshape(-1), F)
        assert ei.value.status == -3
        it, _ = pkg.sibfa_last_stats(ctx)
        assert it == 1
    finally:
        pkg.sibfa_destroy(ctx)
