"""The device velocity-Verlet driver (sibfa_md_steps) against a host
integration of the same trajectory: two 0.5 fs steps of the 216-water box,
FP64 path.  The host side takes the intermolecular forces from
sibfa_energy_forces on a second context and the intramolecular support
forces as central finite differences of the energy the header defines
(k_bond (r - r0)^2 per O-H bond + k_angle (theta - theta0)^2 per angle), and
converts (kcal/mol/A)/amu to A/fs^2 from the unit definitions.  Positions,
velocities and the reported energy terms of the last step must agree."""
import math

import numpy as np
import pytest

import synth
from gpu_util import TERMS

pytestmark = pytest.mark.gpu

KB, R0, KA, TH0_DEG = 529.6, 0.9572, 34.05, 104.52
DT_FS = 0.5
# 1 kcal/mol/A per amu: 4184 J/mol / (1e-3 kg/mol) / 1e-10 m, in A/fs^2
ACC = 4184.0 / 1e-3 / 1e-10 * 1e10 * 1e-30


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


def intra_energy(x):
    """Per-molecule support energy; x (M, 3, 3)."""
    a, b = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    ra, rb = np.linalg.norm(a, axis=-1), np.linalg.norm(b, axis=-1)
    th = np.arccos(np.clip((a * b).sum(-1) / (ra * rb), -1.0, 1.0))
    return KB * ((ra - R0) ** 2 + (rb - R0) ** 2) + KA * (th - math.radians(TH0_DEG)) ** 2


def intra_forces(x, h=1e-5):
    """-dE/dx by central differences; molecules are independent, so one
    coordinate is displaced in every molecule at once."""
    F = np.zeros_like(x)
    for k in range(3):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[:, k, c] += h
            xm[:, k, c] -= h
            F[:, k, c] = -(intra_energy(xp) - intra_energy(xm)) / (2 * h)
    return F


def _ctx(pkg, s, o):
    return pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                            ewald_alpha=o["ewald"], pcg_tol_D=1e-11, precision=pkg.PREC_FP64, warm_start=0,
                            md_k_bond=KB, md_r0=R0, md_k_angle=KA, md_theta0_deg=TH0_DEG)


def test_velocity_verlet_matches_host_integration():
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    M = s.n_mol
    m = s.masses()                                     # (M, 3) amu
    v0 = synth.maxwell_velocities(s, 300.0, seed=11)   # (M, 3, 3) A/fs
    ctx_f = _ctx(pkg, s, o)
    try:
        def inter(x):
            xd = torch.tensor(x.reshape(-1), dtype=torch.float64, device="cuda")
            F = torch.zeros_like(xd)
            e = pkg.sibfa_energy_forces(ctx_f, xd, F)
            torch.cuda.synchronize()
            return F.cpu().numpy().reshape(M, 3, 3), e

        x, v = s.pos.copy(), v0.copy()
        F = inter(x)[0] + intra_forces(x)
        for _ in range(2):
            v = v + 0.5 * DT_FS * ACC * F / m[:, :, None]
            x = x + DT_FS * v
            Fi, e_host = inter(x)
            F = Fi + intra_forces(x)
            v = v + 0.5 * DT_FS * ACC * F / m[:, :, None]
    finally:
        pkg.sibfa_destroy(ctx_f)

    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(v0.reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(m.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = _ctx(pkg, s, o)
    try:
        e_dev = pkg.sibfa_md_steps(ctx, pos, vel, masses, DT_FS, 2)
        torch.cuda.synchronize()
    finally:
        pkg.sibfa_destroy(ctx)
    xd = pos.cpu().numpy().reshape(M, 3, 3)
    vd = vel.cpu().numpy().reshape(M, 3, 3)
    moved = np.abs(x - s.pos).max()
    assert moved > 1e-3                                 # the step did move the atoms
    assert np.abs(xd - x).max() < 1e-9, np.abs(xd - x).max()
    assert np.abs(vd - v).max() < 1e-7 * np.abs(v).max(), np.abs(vd - v).max()
    mag = sum(abs(e_host[k]) for k in TERMS)
    for k in TERMS:
        assert abs(e_dev[k] - e_host[k]) <= 1e-9 * mag, (k, e_dev[k], e_host[k])


def test_nve_stays_stable_with_bounded_drift():
    """The 216-water box as the MD workloads run it (mixed precision, PCG
    1e-6 D, quartic-extrapolation start): 20 capped relaxation steps, 100
    velocity-rescaled steps at 300 K, then 240 NVE steps of 0.5 fs: no error
    status (in particular no charge-transfer denominator reaching zero, no
    atom leaving its molecule), the total energy (kinetic + intermolecular +
    support) drifts by less than 0.02 kcal/mol per atom, and the temperature
    stays bounded (the random lattice is still relaxing into the liquid, so
    it rises above 300 K in NVE; a collapse would run away)."""
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=1e-6, precision=pkg.PREC_MIXED, warm_start=5,
                           md_k_bond=KB, md_r0=R0, md_k_angle=KA, md_theta0_deg=TH0_DEG)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=21).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    m3 = masses.repeat_interleave(3)
    ndof = vel.numel() - 3
    kb, conv = 0.0019872041, 4.184e-4

    def kinetic():
        return 0.5 * float((m3 * vel * vel).sum()) / conv

    try:
        pkg.sibfa_minimize(ctx, pos, 20, 0.01)
        for _ in range(20):
            pkg.sibfa_md_steps(ctx, pos, vel, masses, DT_FS, 5)
            vel.mul_(math.sqrt(300.0 / (2.0 * kinetic() / (ndof * kb))))
        totals, temps = [], []
        for _ in range(24):
            e = pkg.sibfa_md_steps(ctx, pos, vel, masses, DT_FS, 10)
            x = pos.cpu().numpy().reshape(-1, 3, 3)
            totals.append(kinetic() + e["total"] + float(intra_energy(x).sum()))
            temps.append(2.0 * kinetic() / (ndof * kb))
    finally:
        pkg.sibfa_destroy(ctx)
    drift = abs(totals[-1] - totals[0]) / s.n_atoms
    assert drift < 0.02, (drift, totals[0], totals[-1])
    assert 200.0 < min(temps) and max(temps) < 1500.0, temps


@pytest.mark.parametrize("name,n_nve", [("water4096", 1000), ("water32000", 500)])
def test_workload_nve_runs_reach_their_lengths(name, n_nve):
    """The MD workloads' own lengths at 0.5 fs (1000 NVE steps of the
    4096-water box, 500 of the 32,000-water box) after the bench's
    preparation shortened (20 capped relaxation steps, 200 velocity-rescaled
    steps at 300 K): every chunk returns without an error status, the total
    energy drifts by less than 0.02 kcal/mol per atom and the temperature
    stays bounded."""
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config(name)
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=o["pcg_tol"], precision=pkg.PREC_MIXED, warm_start=5,
                           md_k_bond=KB, md_r0=R0, md_k_angle=KA, md_theta0_deg=TH0_DEG)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=22).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    m3 = masses.repeat_interleave(3)
    ndof = vel.numel() - 3
    kb, conv = 0.0019872041, 4.184e-4

    def kinetic():
        return 0.5 * float((m3 * vel * vel).sum()) / conv

    try:
        pkg.sibfa_minimize(ctx, pos, 20, 0.01)
        for _ in range(40):
            pkg.sibfa_md_steps(ctx, pos, vel, masses, DT_FS, 5)
            vel.mul_(math.sqrt(300.0 / (2.0 * kinetic() / (ndof * kb))))
        totals, temps = [], []
        for _ in range(n_nve // 50):
            e = pkg.sibfa_md_steps(ctx, pos, vel, masses, DT_FS, 50)
            x = pos.cpu().numpy().reshape(-1, 3, 3)
            totals.append(kinetic() + e["total"] + float(intra_energy(x).sum()))
            temps.append(2.0 * kinetic() / (ndof * kb))
    finally:
        pkg.sibfa_destroy(ctx)
    assert len(totals) * 50 == n_nve
    drift = abs(totals[-1] - totals[0]) / s.n_atoms
    assert drift < 0.02, (drift, totals[0], totals[-1])
    assert 200.0 < min(temps) and max(temps) < 1500.0, temps


KUB, RUB = 38.25, 1.5326


def intra_energy_mm3(x):
    """The anharmonic support potential of the header (MM3-style bond and
    angle factors, Urey-Bradley H-H term), per molecule."""
    a, b = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    ra, rb = np.linalg.norm(a, axis=-1), np.linalg.norm(b, axis=-1)
    th = np.arccos(np.clip((a * b).sum(-1) / (ra * rb), -1.0, 1.0))

    def bond(dr):
        return KB * dr ** 2 * (1 - 2.55 * dr + (7.0 / 12.0) * 2.55 ** 2 * dr ** 2)

    dth = th - math.radians(TH0_DEG)
    D = np.degrees(dth)
    ang = KA * dth ** 2 * (1 - 0.014 * D + 5.6e-5 * D ** 2 - 7e-7 * D ** 3 + 9e-10 * D ** 4)
    rhh = np.linalg.norm(x[:, 1] - x[:, 2], axis=-1)
    return bond(ra - R0) + bond(rb - R0) + ang + KUB * (rhh - RUB) ** 2


def intra_forces_mm3(x, h=1e-5):
    F = np.zeros_like(x)
    for k in range(3):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[:, k, c] += h
            xm[:, k, c] -= h
            F[:, k, c] = -(intra_energy_mm3(xp) - intra_energy_mm3(xm)) / (2 * h)
    return F


def test_beeman_with_anharmonic_support_matches_host_integration():
    """Beeman steps (the paper's integrator) with the anharmonic bond/angle
    factors and the Urey-Bradley term against a host integration of the
    same recurrences, with the library's intermolecular forces and
    central-difference support forces from the header's definition."""
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    M = s.n_mol
    m = s.masses()
    v0 = synth.maxwell_velocities(s, 300.0, seed=12)
    ctx_f = _ctx(pkg, s, o)
    try:
        def inter(x):
            xd = torch.tensor(x.reshape(-1), dtype=torch.float64, device="cuda")
            F = torch.zeros_like(xd)
            e = pkg.sibfa_energy_forces(ctx_f, xd, F)
            torch.cuda.synchronize()
            return F.cpu().numpy().reshape(M, 3, 3), e

        dt = 1.0
        x, v = s.pos.copy(), v0.copy()
        a = ACC * (inter(x)[0] + intra_forces_mm3(x)) / m[:, :, None]
        a_prev = a.copy()
        for _ in range(2):
            x = x + v * dt + (4 * a - a_prev) * dt * dt / 6
            Fi, e_host = inter(x)
            a_new = ACC * (Fi + intra_forces_mm3(x)) / m[:, :, None]
            v = v + (2 * a_new + 5 * a - a_prev) * dt / 6
            a_prev, a = a, a_new
    finally:
        pkg.sibfa_destroy(ctx_f)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(v0.reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(m.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=1e-11, precision=pkg.PREC_FP64, warm_start=0,
                           md_k_bond=KB, md_r0=R0, md_k_angle=KA, md_theta0_deg=TH0_DEG, md_integrator="beeman",
                           md_anharmonic=True, md_k_ub=KUB, md_r_ub=RUB)
    try:
        pkg.sibfa_md_steps(ctx, pos, vel, masses, 1.0, 2)
        torch.cuda.synchronize()
    finally:
        pkg.sibfa_destroy(ctx)
    xd = pos.cpu().numpy().reshape(M, 3, 3)
    vd = vel.cpu().numpy().reshape(M, 3, 3)
    assert np.abs(x - s.pos).max() > 1e-3
    assert np.abs(xd - x).max() < 1e-9, np.abs(xd - x).max()
    assert np.abs(vd - v).max() < 1e-7 * np.abs(v).max(), np.abs(vd - v).max()


@pytest.mark.parametrize("case", ["water512_cells", "water216_all_pairs"])
def test_neighbour_list_reuse_matches_a_fresh_build(case):
    """Along 40 MD steps the periodic neighbour list is rebuilt only when an
    O has moved by half the list skin; in between its entries are refreshed.
    Energies, forces and dipoles at the final positions equal those of a
    fresh context, which builds its list from scratch (FP64, rounding only):
    the cell-list path (512 waters, three cells per side) and the all-pairs
    path (216 waters)."""
    import torch
    import paper_2201_00804_gb300 as pkg
    if case == "water512_cells":
        s = synth.make_box(8, 24.83, seed=33)
        o = {"rc": 5.0, "grid": 32, "order": 5, "ewald": 0.6}
    else:
        s, o = synth.make_config("water216")

    def ctx_():
        return pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                                ewald_alpha=o["ewald"], pcg_tol_D=1e-11, precision=pkg.PREC_FP64, warm_start=0,
                                md_k_bond=KB, md_r0=R0, md_k_angle=KA, md_theta0_deg=TH0_DEG)

    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(synth.maxwell_velocities(s, 600.0, seed=13).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    res = []
    a = ctx_()
    try:
        pkg.sibfa_md_steps(a, pos, vel, masses, 0.5, 40)
        F = torch.zeros_like(pos)
        mu = torch.zeros_like(pos)
        res.append((pkg.sibfa_energy_forces(a, pos, F), F.clone()))
        pkg.sibfa_solve_dipoles(a, pos, mu, 1e-11)
        res[-1] += (mu.clone(),)
    finally:
        pkg.sibfa_destroy(a)
    b = ctx_()
    try:
        F = torch.zeros_like(pos)
        mu = torch.zeros_like(pos)
        res.append((pkg.sibfa_energy_forces(b, pos, F), F.clone()))
        pkg.sibfa_solve_dipoles(b, pos, mu, 1e-11)
        res[-1] += (mu.clone(),)
    finally:
        pkg.sibfa_destroy(b)
    torch.cuda.synchronize()
    (ea, Fa, ma), (eb, Fb, mb) = res
    assert float((pos.view(-1, 3, 3)[:, 0] - torch.tensor(s.pos[:, 0], device="cuda")).norm(dim=-1).max()) > 0.05
    mag = sum(abs(eb[k]) for k in TERMS)
    for k in TERMS:
        assert abs(ea[k] - eb[k]) <= 1e-10 * mag, (k, ea[k], eb[k])
    assert float((Fa - Fb).abs().max()) <= 1e-8 * float(Fb.abs().max())
    assert float((ma - mb).abs().max()) <= 1e-9
