"""The 32,000-water box (98.6 A, rc 9 A, SPME 108^3) at full size, where the
FP64 oracle does not fit in host memory: properties that hold at any size.
(1) The mixed path in the benchmark's configuration against the FP64 GPU
path (which matches the oracle to ~1e-12 on the 4096-water box): total
energy relative error <= 1e-6, force RMS relative error <= 1e-5 over all
atoms, induced-dipole RMS error <= 1e-6 D.  (2) FP64 forces equal minus the
central finite-difference gradient of the FP64 energy on sampled atoms."""
import numpy as np
import pytest

import synth
from gpu_util import MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D, TERMS, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def box():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()
    return synth.make_config("water32000")


def test_mixed_against_fp64_path(box):
    import paper_2201_00804_gb300 as pkg
    s, o = box
    ref = run_gpu(s, o, pkg.PREC_FP64, 1e-10)
    gpu = run_gpu(s, o, pkg.PREC_MIXED, o["pcg_tol"])
    rt, gt = ref["terms"], gpu["terms"]
    scale = sum(abs(rt[k]) for k in TERMS)
    for k in TERMS:
        assert abs(gt[k] - rt[k]) < MIXED_E_REL * scale, (k, gt[k], rt[k])
    assert abs(gt["total"] - rt["total"]) < MIXED_E_REL * abs(rt["total"])
    ferr = np.sqrt(np.mean((gpu["forces"] - ref["forces"]) ** 2) / np.mean(ref["forces"] ** 2))
    assert ferr < MIXED_F_RMS_REL, ferr
    dmu = (gpu["mu"] - ref["mu"]).reshape(-1, 3) * 4.80321
    assert np.sqrt((dmu ** 2).sum(-1).mean()) < MIXED_MU_RMS_D


def _points(pos):
    """O, H1, H2, the two O-H midpoints and the two lone pairs of every
    molecule (lone pairs from the O frame: bisector z, x toward H1)."""
    P = synth.PARAMS
    O, H1, H2 = pos[:, 0], pos[:, 1], pos[:, 2]
    u1 = (H1 - O) / np.linalg.norm(H1 - O, axis=-1, keepdims=True)
    u2 = (H2 - O) / np.linalg.norm(H2 - O, axis=-1, keepdims=True)
    z = u1 + u2
    z /= np.linalg.norm(z, axis=-1, keepdims=True)
    x = (H1 - O) - ((H1 - O) * z).sum(-1, keepdims=True) * z
    x /= np.linalg.norm(x, axis=-1, keepdims=True)
    y = np.cross(z, x)
    t = np.radians(P["lp_half_deg"])
    d = P["d_lp"]
    lp1 = O + d * (-np.cos(t) * z + np.sin(t) * y)
    lp2 = O + d * (-np.cos(t) * z - np.sin(t) * y)
    return np.stack([O, H1, H2, 0.5 * (O + H1), 0.5 * (O + H2), lp1, lp2], 1)


def _clear_of_cutoff(pts, box, m, rc, margin):
    """No point pair of molecule m with another molecule lies within margin
    of rc: every cutoff of the method (site pairs, bond midpoints, lone pairs,
    the charge-transfer O-O distance) is a distance between these points, so
    a small displacement cannot move a term across its cutoff."""
    d = pts[None, :, None, :, :] - pts[m][None, None, :, None, :]      # (1, M, 7, 7, 3)
    d -= box * np.round(d / box)
    r = np.linalg.norm(d, axis=-1)[0]
    r[m] = 0.0
    return not np.any(np.abs(r - rc) < margin)


def test_fp64_forces_are_minus_the_energy_gradient(box):
    """Central differences with h = 1e-5 A on atoms of molecules clear of the
    (hard) cutoff shell; the FP64 energy is deterministic to ~1e-12 kcal/mol,
    so the difference quotient is exact to far below the tolerance."""
    import paper_2201_00804_gb300 as pkg
    s, o = box
    pts = _points(s.pos)
    rng = np.random.default_rng(32000)
    mols = []
    for m in rng.permutation(s.n_mol)[:64]:
        if _clear_of_cutoff(pts, s.box, m, o["rc"], 1e-4):
            mols.append(m)
            if len(mols) == 2:
                break
    assert len(mols) == 2
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=1e-12, pcg_max_iter=400, precision=pkg.PREC_FP64,
                           warm_start=False)
    try:
        x0 = np.ascontiguousarray(s.pos.reshape(-1))
        F = np.zeros_like(x0)
        pkg.sibfa_energy_forces(ctx, x0, F)
        h = 1e-5
        for m, atom in zip(mols, (0, 1)):
            for c in range(3):
                k = (m * 3 + atom) * 3 + c
                xp, xm = x0.copy(), x0.copy()
                xp[k] += h
                xm[k] -= h
                ep = pkg.sibfa_energy_forces(ctx, xp)["total"]
                em = pkg.sibfa_energy_forces(ctx, xm)["total"]
                fd = -(ep - em) / (2 * h)
                assert abs(fd - F[k]) <= 2e-4 * max(1.0, abs(F[k])), (k, fd, F[k])
    finally:
        pkg.sibfa_destroy(ctx)
