"""Oracle pins for the short-range terms: penetration limits, charge-transfer
sign, scaling and decay, repulsion sign and decay, the C6 tail of the
dispersion and its asymptotic coefficient in closed form."""
import numpy as np

import oracle
import synth
from synth import PARAMS


def _dimer_at(scale, seed=2):
    s = synth.make_dimer(2.91, seed=seed)
    d = s.pos[1, 0] - s.pos[0, 0]
    pos = s.pos.copy()
    pos[1] += (scale - 1.0) * d
    return synth.System(pos=pos, mp_local=s.mp_local, box=None)


def _terms(s, **upd):
    P = dict(PARAMS)
    P.update(upd)
    return oracle.evaluate(s, None, forces=False, P=P, tol_D=1e-11)["terms"]


def test_penetration_vanishes_for_large_b():
    s = synth.make_cluster(3, seed=1)
    t = _terms(s, b_o=1e4, b_h=1e4)
    assert abs(t["pen"]) < 1e-10


def test_penetration_zero_b_turns_charges_into_nuclei():
    """b = 0: every atom charge acts as its nuclear charge Z in all
    charge-involving terms; dipole/quadrupole terms are unchanged."""
    s = synth.make_cluster(3, seed=1)
    t0 = _terms(s, b_o=0.0, b_h=0.0)
    mp = s.mp_local.copy()
    mp[:, 0, 0] = PARAMS["z_o"]
    mp[:, 1:3, 0] = PARAMS["z_h"]
    tz = _terms(synth.System(pos=s.pos, mp_local=mp, box=None))
    assert abs((t0["elec"] + t0["pen"]) - tz["elec"]) < 1e-9 * abs(tz["elec"])


def test_ct_sign_scaling_and_decay():
    s = _dimer_at(1.0)
    t1 = _terms(s)
    assert t1["ct"] < 0
    t2 = _terms(s, ct_t=2 * PARAMS["ct_t"], ct_m=2 * PARAMS["ct_m"])
    assert abs(t2["ct"] - 4 * t1["ct"]) < 1e-9 * abs(t1["ct"])
    far = _terms(_dimer_at(3.0))
    assert abs(far["ct"]) < 1e-3 * abs(t1["ct"])
    c = synth.make_cluster(6, seed=8)
    assert _terms(c)["ct"] < 0


def test_repulsion_positive_and_decaying():
    vals = [_terms(_dimer_at(s))["rep"] for s in (0.95, 1.0, 1.1, 1.3)]
    assert all(v > 0 for v in vals)
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_dispersion_c6_tail():
    # far apart the damping exponent d -> -1 and every pair type decays as 1/r^6
    e1 = _terms(_dimer_at(1000 / 2.91))["disp"]
    e2 = _terms(_dimer_at(2000 / 2.91))["disp"]
    assert e1 < 0 and e2 < 0
    assert abs(e2 / e1 * 64.0 - 1.0) < 0.01
    x = _terms(_dimer_at(1.0))["xdisp"]
    assert x > 0


def test_dispersion_asymptotic_coefficient():
    """Far apart every damping ratio d -> -1 and every reduced distance
    m -> R / (2 sqrt(rv rv)), so R^6 E_disp tends to
    64 C6 e^(gamma6) sum_pairs pref (rv_i rv_j)^3 with the pair prefactors
    -beta_i beta_j (atom-atom), -n^2/4 (lone pair-lone pair) and -delta/2
    (atom-lone pair, both ways).  R^6 E is extrapolated to 1/R -> 0 from
    R = 2000 and 4000 A (its leading correction is linear in 1/R)."""
    P = PARAMS
    ra = np.array([P["rvdw_disp_o"], P["rvdw_disp_h"], P["rvdw_disp_h"]])
    ba = np.array([P["beta_o"], P["beta_h"], P["beta_h"]])
    rl = np.array([P["rvdw_disp_lp"]] * 2)
    s_at = float((ba * ra ** 3).sum())
    s_r = float((ra ** 3).sum())
    s_lp = float((rl ** 3).sum())
    pair_sum = -s_at ** 2 - P["n_lp"] ** 2 / 4.0 * s_lp ** 2 - P["disp_delta"] * s_r * s_lp
    ref = 64.0 * P["c6"] * np.exp(P["gamma6"]) * pair_sum

    def r6e(R):
        return _terms(_dimer_at(R / 2.91))["disp"] * R ** 6

    lim = 2.0 * r6e(4000.0) - r6e(2000.0)
    assert abs(lim / ref - 1.0) < 1e-4, (lim, ref)
