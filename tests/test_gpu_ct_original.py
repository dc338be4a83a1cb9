"""The original many-body charge transfer (run option ct_original; CT
section: the acceptor atoms' potentials V(a) kept in e1, e2 and the
denominator, and V*(a) without the donor molecule) through the C ABI
against the oracle's `ct_original` evaluation: every term, forces and
induced dipoles, FP64 and mixed paths, on gas-phase clusters (workload and
general multipoles) and periodic boxes (all-pairs and cell-list lists); the
virial is refused with it."""
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


CASES = {
    "cluster8": lambda: (synth.make_cluster(8, seed=31), None),
    "cluster8_general": lambda: (synth.with_general_multipoles(synth.make_cluster(8, seed=31), seed=34), None),
    "water216": lambda: synth.make_config("water216"),
    "water512": lambda: (synth.make_box(8, 24.83, seed=33), {"rc": 5.0, "grid": 32, "order": 5, "ewald": 0.6}),
}
_ref = {}


def _oracle(name):
    if name not in _ref:
        s, o = CASES[name]()
        _ref[name] = (s, o, oracle.evaluate(s, dict(o or {}, ct_original=True), tol_D=1e-11))
    return _ref[name]


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_path_matches_oracle(name):
    import paper_2201_00804_gb300 as pkg
    s, o, ref = _oracle(name)
    gpu = run_gpu(s, o, pkg.PREC_FP64, 1e-11, ct_original=True)
    compare(gpu, ref, FP64_E_REL, FP64_F_RMS_REL, FP64_MU_RMS_D)
    # the original form differs from the reduced one
    red = run_gpu(s, o, pkg.PREC_FP64, 1e-11)
    assert abs(red["terms"]["ct"] - gpu["terms"]["ct"]) > 1e-6 * abs(gpu["terms"]["ct"])


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_path_matches_oracle(name):
    import paper_2201_00804_gb300 as pkg
    s, o, ref = _oracle(name)
    gpu = run_gpu(s, o, pkg.PREC_MIXED, 1e-8, ct_original=True)
    compare(gpu, ref, MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D)


def test_virial_is_refused():
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], precision=pkg.PREC_FP64, ct_original=True)
    try:
        pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError, match="INVALID|virial"):
            pkg.sibfa_energy_forces(ctx, pos, torch.zeros_like(pos), virial=np.zeros((3, 3)))
    finally:
        pkg.sibfa_destroy(ctx)
