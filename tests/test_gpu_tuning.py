"""The short-range schedule tuning (resident blocks per SM, and whether the
short-range kernels finish before the polarization solve): after its
warm-up and timed evaluations a context has fixed one of the candidates,
every candidate was timed, and the choice changes the scheduling only:
energies and forces equal those of a context with the tuning off."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


def _ctx(pkg, s, o, tune):
    old = os.environ.get("SIBFA_TUNE")
    os.environ["SIBFA_TUNE"] = "1" if tune else "0"
    try:
        return pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                                ewald_alpha=o["ewald"], pcg_tol_D=1e-10, precision=pkg.PREC_FP64, warm_start=False)
    finally:
        if old is None:
            del os.environ["SIBFA_TUNE"]
        else:
            os.environ["SIBFA_TUNE"] = old


def test_tuning_fixes_a_shape_and_leaves_results_unchanged():
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    a, b = _ctx(pkg, s, o, True), _ctx(pkg, s, o, False)
    try:
        Fa, Fb = torch.zeros_like(pos), torch.zeros_like(pos)
        for _ in range(14):   # 2 warm-up + 5 candidates x 2 timed, each read at the next call
            ea = pkg.sibfa_energy_forces(a, pos, Fa)
        blocks, done = pkg.sibfa_tuned_shape(a)
        assert done and blocks in (0, 2, 3)
        b2, join, done2, ms = pkg.sibfa_tuned_schedule(a)
        assert (b2, done2) == (blocks, done) and join in (False, True)
        assert all(t > 0 for t in ms)                       # every candidate was timed
        assert pkg.sibfa_tuned_schedule(b)[:3] == (3, False, True)
        eb = pkg.sibfa_energy_forces(b, pos, Fb)
        assert pkg.sibfa_tuned_shape(b) == (3, True)      # tuning off: the fixed periodic shape
        torch.cuda.synchronize()
        for k in ea:
            assert ea[k] == pytest.approx(eb[k], rel=1e-12, abs=1e-10), k
        assert np.abs((Fa - Fb).cpu().numpy()).max() < 1e-9
    finally:
        pkg.sibfa_destroy(a)
        pkg.sibfa_destroy(b)
