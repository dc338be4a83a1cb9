"""Batched gas-phase clusters (one context, one launch per kernel): every
cluster's terms, total, forces and induced dipoles match the oracle on that
cluster alone; the batch result of a cluster matches the same cluster
evaluated on its own.

Mixed path: each term and the total within 1e-6 of the cluster's energy
scale (the sum of its term magnitudes, or 1 kcal/mol for the weakest
clusters: FP32 site-pair energies of a few kcal/mol leave absolute errors of
~1e-7 kcal/mol whatever the cluster's total), force RMS relative error <= 1e-5,
dipole RMS error <= 1e-6 D, for the workloads' multipoles and for general
ones (dipoles of any direction and full quadrupoles on every site); the
total of the whole batch within 1e-6 of itself.  A single random cluster's
total is a difference of terms and can lie arbitrarily close to zero (0.85
kcal/mol from terms of 40 kcal/mol for a 12-water cluster here), so its
error is measured on the energy scale rather than relative to the total.
The FP32 inputs set the scale of that error, not the arithmetic: rounding
the O-O displacements and site offsets to 24 bits moves the exact energy of
a 25-water cluster with general multipoles by 2e-6 to 1e-5 kcal/mol (force
times displacement error), about 1e-7 of its energy scale.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FP64_E_REL, FP64_F_RMS_REL, FP64_MU_RMS_D, MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D

pytestmark = pytest.mark.gpu

TERMS = ("elec", "pen", "rep", "disp", "xdisp", "pol", "ct")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


def _batch_run(allsys, start, precision, tol):
    import paper_2201_00804_gb300 as pkg
    ctx = pkg.sibfa_create(synth.PARAMS, allsys.mp_local, periodic=False, pcg_tol_D=tol, precision=precision,
                           warm_start=False, cluster_start=start)
    try:
        F = np.zeros(allsys.n_mol * 9)
        mu = np.zeros(allsys.n_mol * 9)
        tot = pkg.sibfa_energy_forces(ctx, allsys.pos.reshape(-1), F)
        per = pkg.sibfa_cluster_terms(ctx, len(start) - 1)
        pkg.sibfa_solve_dipoles(ctx, allsys.pos.reshape(-1), mu, tol)
    finally:
        pkg.sibfa_destroy(ctx)
    return tot, per, F.reshape(-1, 3, 3), mu.reshape(-1, 3, 3)


def _batch(general):
    allsys, start, parts = synth.make_cluster_batch(24, seed=41)
    if general:
        parts = [synth.with_general_multipoles(c, seed=100 + k) for k, c in enumerate(parts)]
        allsys = synth.System(pos=allsys.pos, mp_local=np.concatenate([c.mp_local for c in parts]), box=None)
    return allsys, start, parts


@pytest.mark.parametrize("general", [False, True], ids=["workload", "general"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_batch_matches_oracle(precision, general):
    import paper_2201_00804_gb300 as pkg
    allsys, start, parts = _batch(general)
    prec = pkg.PREC_FP64 if precision == "fp64" else pkg.PREC_MIXED
    tot, per, F, mu = _batch_run(allsys, start, prec, 1e-10 if precision == "fp64" else 1e-8)
    e_tol = FP64_E_REL if precision == "fp64" else MIXED_E_REL
    f_tol = FP64_F_RMS_REL if precision == "fp64" else MIXED_F_RMS_REL
    mu_tol = FP64_MU_RMS_D if precision == "fp64" else MIXED_MU_RMS_D
    sums = {k: 0.0 for k in TERMS}
    worst, ref_total = 0.0, 0.0
    for c, cl in enumerate(parts):
        ref = oracle.evaluate(cl, None, tol_D=1e-11)
        mag = sum(abs(ref["terms"][k]) for k in TERMS)
        if precision == "mixed":
            mag = max(mag, 1.0)
        for k in TERMS:
            assert abs(per[c][k] - ref["terms"][k]) <= e_tol * mag, (c, k, per[c][k], ref["terms"][k])
            sums[k] += per[c][k]
        rel = abs(per[c]["total"] - ref["terms"]["total"]) / mag
        worst = max(worst, rel)
        assert rel <= e_tol, (c, cl.n_mol, per[c]["total"], ref["terms"]["total"], rel)
        ref_total += ref["terms"]["total"]
        fr = ref["forces"]
        fg = F[start[c]:start[c + 1]]
        rms = np.sqrt(np.mean((fg - fr) ** 2)) / np.sqrt(np.mean(fr ** 2))
        assert rms <= f_tol, (c, rms)
        dmu = (mu[start[c]:start[c + 1]] - ref["mu"]).reshape(-1, 3) * 4.80321
        assert np.sqrt((dmu ** 2).sum(-1).mean()) <= mu_tol, c
    for k in TERMS:
        assert tot[k] == pytest.approx(sums[k], rel=1e-12, abs=1e-9)
    assert abs(tot["total"] - ref_total) <= e_tol * abs(ref_total), (tot["total"], ref_total)
    print(f"worst per-cluster total error on the energy scale ({precision}, general={general}): {worst:.2e}")


def test_cluster_alone_equals_in_batch():
    import paper_2201_00804_gb300 as pkg
    allsys, start, parts = synth.make_cluster_batch(16, seed=42)
    _, per, F, _ = _batch_run(allsys, start, pkg.PREC_FP64, 1e-10)
    for c in (0, 7, 15):
        cl = parts[c]
        ctx = pkg.sibfa_create(synth.PARAMS, cl.mp_local, periodic=False, pcg_tol_D=1e-10, precision=pkg.PREC_FP64,
                               warm_start=False)
        try:
            Fa = np.zeros(cl.n_mol * 9)
            ea = pkg.sibfa_energy_forces(ctx, cl.pos.reshape(-1), Fa)
        finally:
            pkg.sibfa_destroy(ctx)
        mag = sum(abs(ea[k]) for k in TERMS)
        for k in TERMS:
            assert abs(per[c][k] - ea[k]) <= 1e-9 * mag
        assert np.abs(F[start[c]:start[c + 1]].reshape(-1) - Fa).max() <= 1e-8 * np.abs(Fa).max()


def test_full_4096_cluster_batch_sampled_against_oracle():
    """The 4096-cluster workload as the benchmark runs it (one context, mixed
    precision, PCG 1e-8 D here so that the dipole bound is not the solver's):
    64 seeded clusters of the batch against the oracle on each of them."""
    import torch
    import paper_2201_00804_gb300 as pkg
    allsys, start, parts = synth.make_cluster_batch(4096, seed=4)
    ctx = pkg.sibfa_create(synth.PARAMS, allsys.mp_local, periodic=False, pcg_tol_D=1e-8,
                           precision=pkg.PREC_MIXED, warm_start=False, cluster_start=start)
    try:
        pos = torch.tensor(allsys.pos.reshape(-1), dtype=torch.float64, device="cuda")
        F = torch.zeros_like(pos)
        mu = torch.zeros_like(pos)
        pkg.sibfa_energy_forces(ctx, pos, F)
        per = pkg.sibfa_cluster_terms(ctx, len(start) - 1)
        pkg.sibfa_solve_dipoles(ctx, pos, mu, 1e-8)
        torch.cuda.synchronize()
        F = F.cpu().numpy().reshape(-1, 3, 3)
        mu = mu.cpu().numpy().reshape(-1, 3, 3)
    finally:
        pkg.sibfa_destroy(ctx)
    sample = np.sort(np.random.default_rng(4096).choice(4096, 64, replace=False))
    got_total, ref_total = 0.0, 0.0
    for c in sample:
        ref = oracle.evaluate(parts[c], None, tol_D=1e-11)
        mag = max(1.0, sum(abs(ref["terms"][k]) for k in TERMS))
        for k in TERMS + ("total",):
            assert abs(per[c][k] - ref["terms"][k]) <= MIXED_E_REL * mag, (c, k, per[c][k], ref["terms"][k])
        got_total += per[c]["total"]
        ref_total += ref["terms"]["total"]
        fr, fg = ref["forces"], F[start[c]:start[c + 1]]
        assert np.sqrt(np.mean((fg - fr) ** 2) / np.mean(fr ** 2)) <= MIXED_F_RMS_REL, c
        dmu = (mu[start[c]:start[c + 1]] - ref["mu"]).reshape(-1, 3) * 4.80321
        assert np.sqrt((dmu ** 2).sum(-1).mean()) <= MIXED_MU_RMS_D, c
    # the sampled clusters' total energy
    assert abs(got_total - ref_total) <= MIXED_E_REL * abs(ref_total), (got_total, ref_total)
