"""Long-range dispersion beyond the cutoff (run option disp_tail): through
the C ABI, the 216-water box with and without it differs in the dispersion
energy and the total by the oracle's homogeneous-fluid tail (its closed form
by the incomplete gamma function, against the library's quadrature), in
the virial by the same value on the diagonal, and not at all in the
forces."""
import numpy as np
import pytest

import synth
from oracle import terms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_disp_tail_energy_virial_forces(precision):
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    prec = pkg.PREC_FP64 if precision == "fp64" else pkg.PREC_MIXED
    out = {}
    for tail in (False, True):
        ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                               ewald_alpha=o["ewald"], pcg_tol_D=1e-10, precision=prec, warm_start=False,
                               disp_tail=tail)
        try:
            pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
            F = torch.zeros_like(pos)
            W = np.zeros((3, 3))
            e = pkg.sibfa_energy_forces(ctx, pos, F, virial=W)
            torch.cuda.synchronize()
            out[tail] = (e, F.cpu().numpy(), W)
        finally:
            pkg.sibfa_destroy(ctx)
    ref = terms.disp_tail(s.n_mol, float(np.prod(s.box)), o["rc"], synth.PARAMS)
    (e0, F0, W0), (e1, F1, W1) = out[False], out[True]
    assert abs((e1["disp"] - e0["disp"]) - ref) < 1e-9 * abs(ref) + 1e-9, (e1["disp"] - e0["disp"], ref)
    # the totals of two mixed-precision runs also differ by the order of the FP32 grid atomics
    assert abs((e1["total"] - e0["total"]) - ref) < (1e-9 * abs(ref) if precision == "fp64" else
                                                     1e-7 * abs(e0["total"])) + 1e-9
    np.testing.assert_allclose(W1 - W0, ref * np.eye(3),
                               atol=(1e-9 * abs(ref) if precision == "fp64" else 1e-7 * np.abs(W0).max()) + 1e-9)
    # the same arithmetic with and without the tail: forces equal up to the order of the grid atomics
    assert np.abs(F1 - F0).max() <= (1e-9 if precision == "fp64" else 1e-5) * np.abs(F0).max()
