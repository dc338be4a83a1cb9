"""PCG initial guesses along an MD trajectory (216-water box, FP64 path,
tolerance 1e-10 D): the direct-field guess (0), the previous dipoles (1)
and the cubic, quartic and quintic extrapolations through the last four,
five and six full evaluations (4, 5, 6) all converge to the same energies,
forces and dipoles; the extrapolations need no more iterations than the
previous dipoles once their history is full; a dipole-only solve in
between does not enter that history."""
import numpy as np
import pytest

import synth
from gpu_util import TERMS

pytestmark = pytest.mark.gpu

N_STEPS = 12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


def _ctx(pkg, s, o, warm):
    return pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                            ewald_alpha=o["ewald"], pcg_tol_D=1e-10, precision=pkg.PREC_FP64, warm_start=warm)


def test_guesses_converge_to_the_same_solution():
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    # a short NVE trajectory (0.5 fs steps) from a context of its own
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=7).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    md = _ctx(pkg, s, o, 1)
    snaps = []
    try:
        for _ in range(N_STEPS):
            pkg.sibfa_md_steps(md, pos, vel, masses, 0.5, 1)
            snaps.append(pos.clone())
    finally:
        pkg.sibfa_destroy(md)
    res = {}
    for warm in (0, 1, 4, 5, 6):
        ctx = _ctx(pkg, s, o, warm)
        out = []
        try:
            for k, x in enumerate(snaps):
                F = torch.zeros_like(x)
                e = pkg.sibfa_energy_forces(ctx, x, F)
                it = pkg.sibfa_last_stats(ctx)[0]
                if k == N_STEPS // 2:
                    # a dipole-only solve at other positions between two steps
                    mu = torch.zeros_like(x)
                    pkg.sibfa_solve_dipoles(ctx, snaps[0], mu, 1e-10)
                torch.cuda.synchronize()
                out.append((e, F.cpu().numpy(), it))
        finally:
            pkg.sibfa_destroy(ctx)
        res[warm] = out
    for k in range(N_STEPS):
        e0, F0, _ = res[0][k]
        mag = sum(abs(e0[t]) for t in TERMS)
        for warm in (1, 4, 5, 6):
            e, F, _ = res[warm][k]
            for t in TERMS:
                assert abs(e[t] - e0[t]) <= 1e-9 * mag, (warm, k, t, e[t], e0[t])
            assert np.abs(F - F0).max() <= 1e-7 * np.abs(F0).max(), (warm, k)
    it1 = sum(r[2] for r in res[1][6:])
    for warm in (4, 5, 6):
        itw = sum(r[2] for r in res[warm][6:])
        assert itw <= it1, (warm, [r[2] for r in res[1]], [r[2] for r in res[warm]])


def test_minimize_then_md_matches_a_fresh_context():
    """sibfa_minimize leaves no dipoles in the extrapolation history: MD steps
    after a relaxation take the same PCG iterations and give the same energies
    and positions as a fresh context started from the relaxed positions.  (The
    first evaluation of each MD call sequence differs only in its guess, the
    relaxation's last dipoles or the direct field, and is not counted: the
    iterations compared are those of each call's last evaluation.)"""
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    v0 = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=9).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    a = _ctx(pkg, s, o, 4)
    try:
        pkg.sibfa_minimize(a, pos, 5, 0.01)
        relaxed = pos.clone()
        pa, va = relaxed.clone(), v0.clone()
        ea, ita = [], []
        for _ in range(3):
            ea.append(pkg.sibfa_md_steps(a, pa, va, masses, 0.5, 1))
            ita.append(pkg.sibfa_last_stats(a)[0])
    finally:
        pkg.sibfa_destroy(a)
    b = _ctx(pkg, s, o, 4)
    try:
        pb, vb = relaxed.clone(), v0.clone()
        eb, itb = [], []
        for _ in range(3):
            eb.append(pkg.sibfa_md_steps(b, pb, vb, masses, 0.5, 1))
            itb.append(pkg.sibfa_last_stats(b)[0])
    finally:
        pkg.sibfa_destroy(b)
    assert ita == itb, (ita, itb)
    for x, y in zip(ea, eb):
        for t in TERMS:
            assert abs(x[t] - y[t]) <= 1e-9 * max(1.0, abs(y[t])), (t, x[t], y[t])
    assert float((pa - pb).abs().max()) <= 1e-10


def test_mixed_path_with_extrapolated_guess_matches_oracle_along_trajectory():
    """The mixed path as the MD workloads run it (quartic extrapolation of the
    last five solutions as the PCG start) meets the mixed-precision bounds
    against the oracle at later points of a trajectory, where the guess
    comes from the history and not from the direct field."""
    import torch
    import oracle
    import paper_2201_00804_gb300 as pkg
    from gpu_util import MIXED_E_REL, MIXED_F_RMS_REL, compare
    s, o = synth.make_config("water216")
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=11).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                           ewald_alpha=o["ewald"], pcg_tol_D=o["pcg_tol"], precision=pkg.PREC_MIXED, warm_start=5)
    try:
        for step in range(1, 9):
            pkg.sibfa_md_steps(ctx, pos, vel, masses, 0.5, 1)
            if step in (6, 8):
                # the same positions through the same context: its guess is the
                # extrapolation of the trajectory's last five solutions
                x = pos.clone()
                F = torch.zeros_like(x)
                mu = torch.zeros_like(x)
                e = pkg.sibfa_energy_forces(ctx, x, F)
                it = pkg.sibfa_last_stats(ctx)[0]
                pkg.sibfa_solve_dipoles(ctx, x, mu, o["pcg_tol"])
                torch.cuda.synchronize()
                snap = synth.System(pos=x.cpu().numpy().reshape(-1, 3, 3), mp_local=s.mp_local, box=s.box)
                ref = oracle.evaluate(snap, o, tol_D=1e-11)
                gpu = {"terms": e, "forces": F.cpu().numpy().reshape(-1, 3, 3), "mu": mu.cpu().numpy().reshape(-1, 3, 3)}
                # the workload's dipole tolerance (1e-8 D here) bounds the dipole error
                compare(gpu, ref, MIXED_E_REL, MIXED_F_RMS_REL, 1e-6)
                assert it < 30, it
    finally:
        pkg.sibfa_destroy(ctx)


@pytest.mark.parametrize("warm", [2, 3, 4, 5, 6])
def test_extrapolation_of_a_constant_history_is_the_solution(warm):
    """At fixed positions every stored solution is the same vector, and the
    extrapolation coefficients (-1)^(j+1) C(n, j) of each order sum to one:
    once the history holds n solutions, the initial guess is the converged
    solution itself and the solve stops before its first iteration."""
    import torch
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    ctx = _ctx(pkg, s, o, warm)
    try:
        pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
        F = torch.zeros_like(pos)
        its = []
        for _ in range(warm + 2):
            pkg.sibfa_energy_forces(ctx, pos, F)
            its.append(pkg.sibfa_last_stats(ctx)[0])
    finally:
        pkg.sibfa_destroy(ctx)
    assert its[0] > 5, its                 # the first solve starts from the direct field
    assert its[warm + 1] == 0, its          # history full: the guess is the answer
