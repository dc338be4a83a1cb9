"""Helpers shared by the GPU tests: run the CUDA library through the C ABI and
compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np

import synth

# Tolerances of the mixed-precision path against the FP64 oracle (the
# workloads' bounds: total energy relative error, force RMS relative error,
# induced-dipole RMS error; each term is held to the energy bound relative to
# the sum of the term magnitudes)
MIXED_E_REL = 1e-6
MIXED_F_RMS_REL = 1e-5
MIXED_MU_RMS_D = 1e-6
# FP64 path
FP64_E_REL = 1e-9
FP64_F_RMS_REL = 1e-8
FP64_MU_RMS_D = 1e-8

TERMS = ("elec", "pen", "rep", "disp", "xdisp", "pol", "ct")


def run_gpu(system, opts, precision, tol_D, device=True, params=None, max_iter=300, **create_kw):
    import torch
    import paper_2201_00804_gb300 as pkg

    P = synth.PARAMS if params is None else params
    periodic = system.box is not None
    kw = {}
    if periodic:
        kw = dict(box=system.box, rc=opts["rc"], grid=opts["grid"], ewald_alpha=opts["ewald"])
    ctx = pkg.sibfa_create(P, system.mp_local, periodic=periodic, pcg_tol_D=tol_D, precision=precision,
                           pcg_max_iter=max_iter, warm_start=False, **kw, **create_kw)
    try:
        if device == "pinned":   # page-locked host memory, copied without staging
            pos = torch.tensor(system.pos.reshape(-1), dtype=torch.float64).pin_memory()
            F = torch.zeros_like(pos).pin_memory()
            mu = torch.zeros_like(pos).pin_memory()
        elif device:
            pos = torch.tensor(system.pos.reshape(-1), dtype=torch.float64, device="cuda")
            F = torch.zeros_like(pos)
            mu = torch.zeros_like(pos)
        else:
            pos = np.ascontiguousarray(system.pos.reshape(-1))
            F = np.zeros_like(pos)
            mu = np.zeros_like(pos)
        e = pkg.sibfa_energy_forces(ctx, pos, F)
        it, res = pkg.sibfa_last_stats(ctx)
        pkg.sibfa_solve_dipoles(ctx, pos, mu, tol_D)
        if device:
            torch.cuda.synchronize()
            F = F.cpu().numpy()
            mu = mu.cpu().numpy()
        return {"terms": e, "forces": F.reshape(-1, 3, 3), "mu": mu.reshape(-1, 3, 3), "iters": it, "resid": res}
    finally:
        pkg.sibfa_destroy(ctx)


def compare(gpu, ref, e_rel, f_rel, mu_d):
    """Returns a dict of errors and asserts the tolerances: each term's error
    relative to the sum of the term magnitudes (the per-term statement), the
    total's error relative to |total|, the force RMS error relative to the
    force RMS, and the induced-dipole RMS error in Debye."""
    rt, gt = ref["terms"], gpu["terms"]
    scale = sum(abs(rt[k]) for k in TERMS)
    errs = {k: abs(gt[k] - rt[k]) / scale for k in TERMS}
    errs["total"] = abs(gt["total"] - rt["total"]) / max(abs(rt["total"]), 1e-300)
    Fr = ref["forces"].reshape(-1)
    Fg = gpu["forces"].reshape(-1)
    errs["force_rms_rel"] = float(np.sqrt(np.mean((Fg - Fr) ** 2) / np.mean(Fr ** 2)))
    dmu = (gpu["mu"] - ref["mu"]).reshape(-1, 3) * 4.80321
    errs["mu_rms_D"] = float(np.sqrt((dmu ** 2).sum(-1).mean()))
    msg = f"errors {errs}\n gpu {gt}\n ref {rt}"
    for k in TERMS:
        assert errs[k] < e_rel, msg
    assert errs["total"] < e_rel, msg
    assert errs["force_rms_rel"] < f_rel, msg
    assert errs["mu_rms_D"] < mu_d, msg
    return errs
