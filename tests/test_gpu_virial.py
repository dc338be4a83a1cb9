"""GPU virial W_ab = -dE/d eps_ab (affine strain of atoms and cell) through the
C ABI against the oracle's (which is pinned by strain finite differences):
FP64 path to 1e-8 and mixed path to 2e-5 of max |W|.  Also: in the gas phase
the GPU's W equals sum F_a x_b of its own forces; a cluster batch returns the
sum over its clusters; requesting the virial changes neither energies nor
forces."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FP64_W_REL = 1e-8
MIXED_W_REL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


CASES = {
    "cluster8": (synth.make_cluster(8, seed=31), None),
    "water216": synth.make_config("water216"),
    "water512": (synth.make_box(8, 24.83, seed=33), {"rc": 5.5, "grid": 32, "order": 5, "ewald": 0.55}),
}
_ref = {}


def ref_virial(name):
    if name not in _ref:
        s, o = CASES[name]
        _ref[name] = oracle.evaluate(s, o, tol_D=1e-11, virial=True)["virial"]
    return _ref[name]


def run(system, opts, precision, tol_D, virial=True, cluster_start=None):
    import torch
    import paper_2201_00804_gb300 as pkg
    periodic = system.box is not None
    kw = {}
    if periodic:
        kw = dict(box=system.box, rc=opts["rc"], grid=opts["grid"], ewald_alpha=opts["ewald"])
    if cluster_start is not None:
        kw["cluster_start"] = cluster_start
    ctx = pkg.sibfa_create(synth.PARAMS, system.mp_local, periodic=periodic, pcg_tol_D=tol_D, precision=precision,
                           warm_start=False, **kw)
    try:
        pos = torch.tensor(system.pos.reshape(-1), dtype=torch.float64, device="cuda")
        F = torch.zeros_like(pos)
        W = np.zeros((3, 3)) if virial else None
        e = pkg.sibfa_energy_forces(ctx, pos, F, virial=W)
        torch.cuda.synchronize()
        return e, F.cpu().numpy().reshape(-1, 3, 3), W
    finally:
        pkg.sibfa_destroy(ctx)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_virial_matches_oracle(name):
    import paper_2201_00804_gb300 as pkg
    s, o = CASES[name]
    ref = ref_virial(name)
    _, _, W = run(s, o, pkg.PREC_FP64, 1e-11)
    err = np.abs(W - ref).max() / np.abs(ref).max()
    assert err < FP64_W_REL, (err, W, ref)


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_virial_matches_oracle(name):
    import paper_2201_00804_gb300 as pkg
    s, o = CASES[name]
    ref = ref_virial(name)
    _, _, W = run(s, o, pkg.PREC_MIXED, 1e-8)
    err = np.abs(W - ref).max() / np.abs(ref).max()
    assert err < MIXED_W_REL, (err, W, ref)


def test_gas_phase_virial_is_sum_of_force_times_position():
    import paper_2201_00804_gb300 as pkg
    s = synth.make_cluster(12, seed=41)
    _, F, W = run(s, None, pkg.PREC_FP64, 1e-11)
    ref = np.einsum("mka,mkb->ab", F, s.pos)
    assert np.abs(W - ref).max() < 1e-10 * np.abs(ref).max()


def test_cluster_batch_virial_is_sum_over_clusters():
    import paper_2201_00804_gb300 as pkg
    batch, start, parts = synth.make_cluster_batch(5, seed=43, n_min=2, n_max=9)
    _, _, W = run(batch, None, pkg.PREC_FP64, 1e-11, cluster_start=start)
    ref = sum(run(c, None, pkg.PREC_FP64, 1e-11)[2] for c in parts)
    assert np.abs(W - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["cluster8", "water216"])
def test_virial_request_leaves_energy_and_forces(name):
    import paper_2201_00804_gb300 as pkg
    s, o = CASES[name]
    for prec, rel in ((pkg.PREC_FP64, 1e-12), (pkg.PREC_MIXED, 1e-6)):
        e0, F0, _ = run(s, o, prec, 1e-10, virial=False)
        e1, F1, _ = run(s, o, prec, 1e-10, virial=True)
        for k in e0:
            assert e1[k] == pytest.approx(e0[k], rel=rel, abs=rel), k
        assert np.abs(F1 - F0).max() <= rel * np.abs(F0).max()
