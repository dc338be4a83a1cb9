"""Constant-pressure support: a periodic context whose box changes through
sibfa_energy_forces(box=...) gives the energies, forces and virial of a
context created with that box (FP64 and mixed paths, with the dispersion
tail on, on the all-pairs 216-water box and the cell-list 512-water box),
and changing back restores the first box's results; a box needing more
cells than the context allocated, or too small for the cutoff, is refused
and leaves the box unchanged; the configurational pressure from the virial,
-tr(W)/(3V) = dE/dV under isotropic scaling, matches a central difference
of the energy over box changes; a short Berendsen run moves the volume with
every evaluation succeeding."""
import numpy as np
import pytest

import synth
from gpu_util import TERMS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


def _ctx(pkg, s, o, box, prec, tail=True):
    return pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=np.asarray(box, dtype=np.float64),
                            rc=o["rc"], grid=o["grid"], ewald_alpha=o["ewald"], pcg_tol_D=1e-10, precision=prec,
                            warm_start=False, disp_tail=tail)


def _eval(pkg, ctx, pos, box=None):
    import torch
    F = torch.zeros_like(pos)
    W = np.zeros((3, 3))
    e = pkg.sibfa_energy_forces(ctx, pos, F, box=box, virial=W)
    torch.cuda.synchronize()
    return e, F.cpu().numpy(), W


CASES = {
    "water216": lambda: synth.make_config("water216"),
    # 512 waters with rc 5 A: three cells per side, the cell list
    "water512": lambda: (synth.make_box(8, 24.83, seed=33), {"rc": 5.0, "grid": 32, "order": 5, "ewald": 0.6}),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_box_change_equals_a_fresh_context(name, precision):
    import torch
    import paper_2201_00804_gb300 as pkg
    prec = pkg.PREC_FP64 if precision == "fp64" else pkg.PREC_MIXED
    s, o = CASES[name]()
    box0 = np.asarray(s.box, dtype=np.float64)
    scale = 0.995                      # compression keeps the cell grid within its capacity
    box1 = box0 * scale
    pos0 = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    pos1 = pos0 * scale
    a = _ctx(pkg, s, o, box0, prec)
    b = _ctx(pkg, s, o, box1, prec)
    try:
        ea0, Fa0, Wa0 = _eval(pkg, a, pos0)
        ea1, Fa1, Wa1 = _eval(pkg, a, pos1, box=box1)          # the box changes here
        eb1, Fb1, Wb1 = _eval(pkg, b, pos1)
        ea2, Fa2, Wa2 = _eval(pkg, a, pos0, box=box0)          # and back
    finally:
        pkg.sibfa_destroy(a)
        pkg.sibfa_destroy(b)
    e_tol, f_tol, w_tol = (1e-10, 1e-8, 1e-8) if precision == "fp64" else (2e-7, 2e-6, 2e-5)
    mag = sum(abs(eb1[k]) for k in TERMS)
    for k in TERMS + ("total",):
        assert abs(ea1[k] - eb1[k]) <= e_tol * mag, (k, ea1[k], eb1[k])
        assert abs(ea2[k] - ea0[k]) <= e_tol * mag, (k, ea2[k], ea0[k])
    assert abs(ea1["disp"] - ea0["disp"]) > 1e-6 * mag     # the box change is not a no-op
    fs = np.abs(Fb1).max()
    assert np.abs(Fa1 - Fb1).max() <= f_tol * fs
    assert np.abs(Fa2 - Fa0).max() <= f_tol * fs
    ws = np.abs(Wb1).max()
    assert np.abs(Wa1 - Wb1).max() <= w_tol * ws
    assert np.abs(Wa2 - Wa0).max() <= w_tol * ws


def test_refused_boxes_leave_the_box_unchanged():
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = CASES["water512"]()
    box0 = np.asarray(s.box, dtype=np.float64)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = _ctx(pkg, s, o, box0, pkg.PREC_FP64)
    try:
        e0, F0, W0 = _eval(pkg, ctx, pos)
        # 4 cells per side (64) where the context holds 27
        with pytest.raises(RuntimeError, match="INVALID|cells"):
            _eval(pkg, ctx, pos * 1.3, box=box0 * 1.3)
        # rc 5 + 1.91 over half the box
        with pytest.raises(RuntimeError, match="CUTOFF|half"):
            _eval(pkg, ctx, pos * 0.5, box=box0 * 0.5)
        e1, F1, W1 = _eval(pkg, ctx, pos)
    finally:
        pkg.sibfa_destroy(ctx)
    for k in TERMS:
        assert abs(e1[k] - e0[k]) <= 1e-10 * sum(abs(e0[t]) for t in TERMS)
    assert np.abs(F1 - F0).max() <= 1e-9 * np.abs(F0).max()


def test_virial_pressure_is_the_volume_derivative():
    """Under x -> (1 + e) x and L -> (1 + e) L, dE/de = -tr(W): central
    difference of the FP64 energy over two box changes of one context (a
    step small enough that no point pair crosses the hard cutoff)."""
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = CASES["water216"]()
    box0 = np.asarray(s.box, dtype=np.float64)
    pos0 = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = _ctx(pkg, s, o, box0, pkg.PREC_FP64)
    try:
        _, _, W = _eval(pkg, ctx, pos0)
        h = 1e-8
        ep, _, _ = _eval(pkg, ctx, pos0 * (1 + h), box=box0 * (1 + h))
        em, _, _ = _eval(pkg, ctx, pos0 * (1 - h), box=box0 * (1 - h))
    finally:
        pkg.sibfa_destroy(ctx)
    dEde = (ep["total"] - em["total"]) / (2 * h)
    assert abs(dEde + np.trace(W)) <= 1e-3 * abs(np.trace(W)), (dEde, -np.trace(W))


def test_short_berendsen_run_changes_the_volume():
    """Velocity Verlet with a Berendsen barostat applied every 5 steps
    through box changes (the bench's constant-pressure driver): every call
    succeeds and the volume moves."""
    import torch
    import paper_2201_00804_gb300 as pkg
    import bench
    s, o = synth.make_config("water216")
    box = np.asarray(s.box, dtype=np.float64)
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=1e-6, precision=pkg.PREC_MIXED, warm_start=4,
                           disp_tail=True)
    try:
        pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
        vel = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=3).reshape(-1), dtype=torch.float64,
                           device="cuda")
        masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
        pkg.sibfa_minimize(ctx, pos, 20, 0.01)
        out = bench.berendsen_npt(pkg, ctx, pos, vel, masses, box, n_steps=60, every=5, dt_fs=0.5)
    finally:
        pkg.sibfa_destroy(ctx)
    vols = out["volumes"]
    assert len(vols) == 12 and all(np.isfinite(vols))
    assert abs(vols[-1] - vols[0]) > 1e-6 * vols[0]
    assert np.isfinite(out["pressure_bar"]).all()
