"""Oracle pins for the dispersion beyond the cutoff (homogeneous-fluid tail
correction):

- without damping (all gamma_n -> 0) each C_n term integrates to the
  elementary r^(3-n) / (n - 3) power, written out here;
- for molecules placed uniformly at random (pair distribution exactly 1 in
  expectation) the dispersion between two cutoffs, summed pair by pair with
  the oracle's own truncated sum, equals the difference of the tail values at
  the two cutoffs within its sampling error;
- the virial of the tail is the tail energy on the diagonal (the tail scales
  as 1/V at fixed cutoff).
"""
import math

import numpy as np
import torch

import oracle
import synth
from oracle import core, terms
from synth import PARAMS


def test_undamped_limit_is_the_power_law_integral():
    P = dict(PARAMS, gamma6=1e-9, gamma8=1e-9, gamma10=1e-9)
    N, V, rc = 100, 3000.0, 9.0
    rv = [P["rvdw_disp_o"], P["rvdw_disp_h"], P["rvdw_disp_h"], P["rvdw_disp_lp"], P["rvdw_disp_lp"]]
    beta = [P["beta_o"], P["beta_h"], P["beta_h"]]
    n = P["n_lp"]
    ref = 0.0
    for u in range(5):
        for v in range(5):
            pref = (-beta[u] * beta[v] if u < 3 and v < 3 else
                    (-n * n / 4 if u >= 3 and v >= 3 else -P["disp_delta"] / 2))
            k = 2 * math.sqrt(rv[u] * rv[v])
            # int_rc^inf r^2 C_n (k / r)^n dr = C_n k^n rc^(3-n) / (n - 3)
            ref += pref * (P["c6"] * k ** 6 * rc ** -3 / 3 + P["c8"] * k ** 8 * rc ** -5 / 5
                           + P["c10"] * k ** 10 * rc ** -7 / 7)
    ref *= 2 * math.pi * N * (N - 1) / V
    got = terms.disp_tail(N, V, rc, P)
    assert abs(got - ref) < 1e-7 * abs(ref), (got, ref)


def _uniform_fluid(n, L, seed):
    rng = np.random.default_rng(seed)
    body = synth.water._water_body()
    pos = np.stack([body @ synth.random_rotation(rng).T + rng.uniform(0, L, 3) for _ in range(n)])
    return synth.System(pos=pos, mp_local=np.zeros((n, 5, 10)), box=np.array([L] * 3))


def test_shell_sum_of_a_uniform_fluid_matches_tail_difference():
    n, L, rc1, rc2 = 1200, 50.0, 6.0, 12.0
    s = _uniform_fluid(n, L, seed=61)
    S = core.build_sites(torch.tensor(s.pos), torch.tensor(s.mp_local), PARAMS)
    i, j, sh = terms.mol_pairs(s.pos[:, 0], s.box, rc2 + 2.6)
    e = {rc1: 0.0, rc2: 0.0}
    for a in range(0, i.size, 8192):
        sl = slice(a, a + 8192)
        for rc in (rc1, rc2):
            ed, _ = terms.disp_pairs(S, i[sl], j[sl], torch.tensor(sh[sl]), PARAMS, rc)
            e[rc] += float(ed)
    shell = e[rc2] - e[rc1]
    V = L ** 3
    ref = terms.disp_tail(n, V, rc1, PARAMS) - terms.disp_tail(n, V, rc2, PARAMS)
    # ~1e6 point pairs in the shell: the sampling error is a few tenths of a percent
    assert abs(shell - ref) < 0.02 * abs(ref), (shell, ref)


def test_tail_enters_energy_and_virial():
    s, o = synth.make_config("water216")
    o = dict(o)
    base = oracle.evaluate(s, o, forces=False, tol_D=1e-8)
    o["disp_tail"] = True
    with_tail = oracle.evaluate(s, o, forces=False, tol_D=1e-8)
    tail = terms.disp_tail(s.n_mol, float(np.prod(s.box)), o["rc"], PARAMS)
    assert tail < 0
    assert abs(with_tail["terms"]["disp"] - base["terms"]["disp"] - tail) < 1e-9 * abs(tail)
    small = synth.make_box(2, 13.0, seed=62, jitter=0.2)
    os_ = {"rc": 3.5, "grid": 12, "order": 5, "ewald": 0.9}
    w0 = oracle.evaluate(small, os_, virial=True, tol_D=1e-10)["virial"]
    w1 = oracle.evaluate(small, dict(os_, disp_tail=True), virial=True, tol_D=1e-10)["virial"]
    t = terms.disp_tail(small.n_mol, 13.0 ** 3, 3.5, PARAMS)
    np.testing.assert_allclose(w1 - w0, t * np.eye(3), atol=1e-9 * abs(t))
