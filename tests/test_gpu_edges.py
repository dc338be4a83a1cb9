"""GPU parity on edge shapes, through the C ABI against the FP64 oracle:

- a non-cubic orthorhombic box (504 waters, 21.73 x 24.83 x 27.94 A) with
  SPME grids of 27 x 32 x 35 points: per-axis cell counts, strides and
  grid sizes, odd transforms without a Nyquist plane on two axes; energies,
  forces, dipoles and the virial in both precisions;
- a gas-phase batch of clusters of 1, 385, 1, 6 and 1 molecules: molecules
  with no partner at all beside a cluster at the 385-molecule bound, where
  every molecule fills all 384 neighbour slots;
- a charge-transfer denominator ae + V - ah pushed below zero for every
  lone pair (ah above ae + |V|) returns CT_DENOM, as the oracle's smallest
  denominator says it must."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (FP64_E_REL, FP64_F_RMS_REL, FP64_MU_RMS_D, MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D,
                      TERMS, compare, run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


ORTHO = (synth.make_ortho_box((7, 8, 9), (21.73, 24.83, 27.94), seed=51),
         {"rc": 5.5, "grid": (27, 32, 35), "order": 5, "ewald": 0.55})
_ref = {}


def ortho_ref(virial=False):
    if virial not in _ref:
        s, o = ORTHO
        _ref[virial] = oracle.evaluate(s, o, tol_D=1e-11, virial=virial)
    return _ref[virial]


def test_orthorhombic_odd_grid_fp64_matches_oracle():
    import paper_2201_00804_gb300 as pkg
    s, o = ORTHO
    compare(run_gpu(s, o, pkg.PREC_FP64, 1e-11), ortho_ref(), FP64_E_REL, FP64_F_RMS_REL, FP64_MU_RMS_D)


def test_orthorhombic_odd_grid_mixed_matches_oracle():
    import paper_2201_00804_gb300 as pkg
    s, o = ORTHO
    compare(run_gpu(s, o, pkg.PREC_MIXED, 1e-8), ortho_ref(), MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D)


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-8), ("mixed", 2e-5)])
def test_orthorhombic_odd_grid_virial_matches_oracle(precision, rel):
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = ORTHO
    ref = ortho_ref(virial=True)["virial"]
    prec = pkg.PREC_FP64 if precision == "fp64" else pkg.PREC_MIXED
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=1e-11 if precision == "fp64" else 1e-8,
                           precision=prec, warm_start=False)
    try:
        pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
        W = np.zeros((3, 3))
        pkg.sibfa_energy_forces(ctx, pos, torch.zeros_like(pos), virial=W)
        torch.cuda.synchronize()
    finally:
        pkg.sibfa_destroy(ctx)
    err = np.abs(W - ref).max() / np.abs(ref).max()
    assert err < rel, (err, W, ref)


def test_single_molecules_beside_largest_cluster():
    import paper_2201_00804_gb300 as pkg
    sizes = [1, 385, 1, 6, 1]
    allsys, start, parts = synth.make_cluster_sizes(sizes, seed=53)
    ctx = pkg.sibfa_create(synth.PARAMS, allsys.mp_local, periodic=False, pcg_tol_D=1e-10,
                           precision=pkg.PREC_FP64, warm_start=False, cluster_start=start)
    try:
        F = np.zeros(allsys.n_mol * 9)
        tot = pkg.sibfa_energy_forces(ctx, allsys.pos.reshape(-1), F)
        per = pkg.sibfa_cluster_terms(ctx, len(sizes))
    finally:
        pkg.sibfa_destroy(ctx)
    F = F.reshape(-1, 3, 3)
    for c, n in enumerate(sizes):
        if n == 1:
            assert all(abs(per[c][k]) < 1e-12 for k in TERMS), per[c]
            assert np.abs(F[start[c]:start[c + 1]]).max() < 1e-12
    # the six-molecule cluster against the oracle
    ref = oracle.evaluate(parts[3], None, tol_D=1e-11)
    mag = sum(abs(ref["terms"][k]) for k in TERMS)
    for k in TERMS:
        assert abs(per[3][k] - ref["terms"][k]) <= FP64_E_REL * mag, (k, per[3][k], ref["terms"][k])
    fr, fg = ref["forces"], F[start[3]:start[4]]
    assert np.sqrt(np.mean((fg - fr) ** 2) / np.mean(fr ** 2)) <= FP64_F_RMS_REL
    # the 385-molecule cluster in the batch = the same cluster alone
    big = parts[1]
    ctx = pkg.sibfa_create(synth.PARAMS, big.mp_local, periodic=False, pcg_tol_D=1e-10, precision=pkg.PREC_FP64,
                           warm_start=False)
    try:
        Fa = np.zeros(big.n_mol * 9)
        ea = pkg.sibfa_energy_forces(ctx, big.pos.reshape(-1), Fa)
    finally:
        pkg.sibfa_destroy(ctx)
    mag = sum(abs(ea[k]) for k in TERMS)
    for k in TERMS:
        assert abs(per[1][k] - ea[k]) <= 1e-9 * mag, (k, per[1][k], ea[k])
        assert tot[k] == pytest.approx(sum(per[c][k] for c in range(len(sizes))), rel=1e-12, abs=1e-9)
    assert np.abs(F[start[1]:start[2]].reshape(-1) - Fa).max() <= 1e-8 * np.abs(Fa).max()


def test_negative_ct_denominator_returns_ct_denom():
    import paper_2201_00804_gb300 as pkg
    s = synth.make_cluster(8, seed=31)
    P = dict(synth.PARAMS, ct_ah=2000.0)
    assert oracle.evaluate(s, None, P=P, forces=False, tol_D=1e-8)["min_ct_denominator"] < 0
    with pytest.raises(pkg.SibfaError) as ei:
        run_gpu(s, None, pkg.PREC_FP64, 1e-8, params=P)
    assert ei.value.status == -5
