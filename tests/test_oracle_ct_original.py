"""Pins of the original many-body charge transfer (CT section: the acceptor
potentials V(a) and the donor-excluded V*(a) kept in e1, e2 and dE), the
oracle's `ct_pairs_original`, `atom_potential_pairs` and
`atom_potential_periodic`:

- a hand-laid donor with point charges and an acceptor with given
  potentials, every factor written out from the formulas (V* from the
  donor's charges by Coulomb's law);
- in a dimer the potential at an acceptor atom is the donor's alone, so
  V*(a) = 0 and each direction is the reduced form with ah replaced by
  ah + V(a1);
- the gas-phase acceptor potentials against the textbook multipole
  potential of the other molecules;
- in a periodic box the acceptor potentials do not depend on the Ewald
  splitting parameter (real space converged);
- forces of the whole evaluation equal minus the central finite-difference
  gradient of the energy (gas phase and periodic: the adjoint charges on
  the acceptor atoms and the lone pairs)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import core, terms
from synth import PARAMS
from test_oracle_pins import KE, PAIR, _phi_direct, _sites, periodic_pair  # noqa: F401

DT = torch.float64


def test_original_charge_transfer_hand_case():
    """The reduced hand layout (distances 2-5, cosines 0, 3/5, 4/5, 1) with
    given acceptor potentials V(a); the donor's sites carry point charges, so
    V*(a) = V(a) - k_e sum_s q_s / |a - x_s| is evaluated here by hand."""
    P = PARAMS
    qA = [-0.8, 0.3, 0.1, 0.25, 0.15]
    qB = [-0.7, 0.2, 0.2, 0.15, 0.15]
    A = dict(O=[0, 0, 0], H1=[-1, 0, 0], H2=[3, 0, 4], LP1=[0.5, 0, 0], LP2=[0, 0.5, 0], q=qA)
    B = dict(O=[3, 0, 0], H1=[3, 4, 0], H2=[2, 0, 0], LP1=[2.5, 0, 0], LP2=[3, 0, 0.5], q=qB)
    S = _sites([A, B])
    V = torch.tensor([[-20.0, -30.0], [-25.0, -15.0]], dtype=DT)
    Vat = torch.tensor([[12.0, -7.0, -4.0], [9.0, -6.0, -5.0]], dtype=DT)
    Vint = torch.tensor([[-50.0, 30.0, 35.0], [-45.0, 28.0, 33.0]], dtype=DT)
    E, min_de = terms.ct_pairs_original(S, V, Vat, Vint, *PAIR, P, 9.0)
    eta, t, m, n = P["ct_eta"], P["ct_t"], P["ct_m"], P["n_lp"]
    cs, cp = P["cs_lp"], P["cp_lp"]
    rvo, rvh = P["rvdw_ct_o"], P["rvdw_ct_h"]
    ae, ah = P["ct_ae"], P["ct_ah"]

    def sites(mol):
        O, H1, H2 = (np.asarray(mol[k], float) for k in ("O", "H1", "H2"))
        return [O, H1, H2, 0.5 * (O + H1), 0.5 * (O + H2)]

    def vstar(V_a, at, donor):
        return V_a - KE * sum(q / np.linalg.norm(np.asarray(at, float) - x)
                              for q, x in zip(donor["q"], sites(donor)))

    def transfer(V_lp, cos_a, r1, Vint_a1, Vs_a1, V_a1, acc):
        total = 0.0
        e1 = (math.exp(-eta * r1 / (2 * math.sqrt(rvo * rvo))) * (Vint_a1 + Vs_a1 - V_lp)
              * (cs * t + cp * m * cos_a))
        for r2, cos_b, Vint_a2, Vs_a2 in acc:
            e2 = (math.exp(-eta * r2 / (2 * math.sqrt(rvo * rvh))) * (Vint_a2 + Vs_a2 - V_lp)
                  * (cs * t + cp * m * cos_b))
            total += -n * (e1 - e2) ** 2 / (ae + V_lp - (ah + V_a1))
        return total

    # A's lone pairs -> B's bonds; V* at B's atoms without A's charges
    vs_b = [vstar(9.0, B["O"], A), vstar(-6.0, B["H1"], A), vstar(-5.0, B["H2"], A)]
    ref = transfer(-20.0, 1.0, 3.0, -45.0, vs_b[0], 9.0, [(5.0, 0.6, 28.0, vs_b[1]), (2.0, 1.0, 33.0, vs_b[2])])
    ref += transfer(-30.0, 0.0, 3.0, -45.0, vs_b[0], 9.0, [(5.0, 0.8, 28.0, vs_b[1]), (2.0, 0.0, 33.0, vs_b[2])])
    # B's lone pairs -> A's bonds; V* at A's atoms without B's charges
    vs_a = [vstar(12.0, A["O"], B), vstar(-7.0, A["H1"], B), vstar(-4.0, A["H2"], B)]
    ref += transfer(-25.0, 1.0, 3.0, -50.0, vs_a[0], 12.0, [(4.0, 1.0, 30.0, vs_a[1]), (4.0, 0.0, 35.0, vs_a[2])])
    ref += transfer(-15.0, 0.0, 3.0, -50.0, vs_a[0], 12.0, [(4.0, 0.0, 30.0, vs_a[1]), (4.0, 1.0, 35.0, vs_a[2])])
    assert abs(float(E) - ref) < 1e-12 * abs(ref), (float(E), ref)
    assert abs(min_de - min(ae - 30.0 - ah - 9.0, ae - 25.0 - ah - 12.0)) < 1e-12
    E_far, _ = terms.ct_pairs_original(S, V, Vat, Vint, *PAIR, P, 2.9)
    assert float(E_far) == 0.0


def test_dimer_acceptor_potential_is_the_donor_alone():
    """Gas-phase dimer: V(a) comes from the donor alone, so V*(a) = 0 and each
    direction is the reduced form with ah replaced by ah + V(a1), evaluated
    here item by item from the formula."""
    P = PARAMS
    s = synth.with_general_multipoles(synth.make_cluster(2, seed=41), seed=42)
    x = torch.tensor(s.pos, dtype=DT)
    S = core.build_sites(x, torch.tensor(s.mp_local, dtype=DT), P)
    i, j, sh = terms.mol_pairs(s.pos[:, 0], None, None)
    sh = torch.tensor(sh)
    V = terms.lp_potential_pairs(S, i, j, sh, P, None, None).numpy()
    Vat = terms.atom_potential_pairs(S, i, j, sh, P, None, None)
    Vint = terms.v_int(S, P)
    E, _ = terms.ct_pairs_original(S, torch.tensor(V), Vat, Vint, i, j, sh, P, None)
    eta, t, m, n = P["ct_eta"], P["ct_t"], P["ct_m"], P["n_lp"]
    cs, cp = P["cs_lp"], P["cp_lp"]
    rvo, rvh = P["rvdw_ct_o"], P["rvdw_ct_h"]
    X, LP, VI, VA = S["x"].numpy(), S["lp"].numpy(), Vint.numpy(), Vat.numpy()

    def cos(u, v):
        return float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))

    ref = 0.0
    for d, a in ((0, 1), (1, 0)):
        c = X[d, 0]
        for l in range(2):
            u = LP[d, l] - c
            e1 = (math.exp(-eta * np.linalg.norm(X[a, 0] - c) / (2 * rvo)) * (VI[a, 0] - V[d, l])
                  * (cs * t + cp * m * cos(u, X[a, 0] - c)))
            for h in (1, 2):
                e2 = (math.exp(-eta * np.linalg.norm(X[a, h] - c) / (2 * math.sqrt(rvo * rvh)))
                      * (VI[a, h] - V[d, l]) * (cs * t + cp * m * cos(u, X[a, h] - c)))
                ref += -n * (e1 - e2) ** 2 / (P["ct_ae"] + V[d, l] - (P["ct_ah"] + VA[a, 0]))
    assert abs(float(E) - ref) < 1e-11 * abs(ref), (float(E), ref)


def test_gas_acceptor_potential_is_the_multipole_potential():
    s = synth.with_general_multipoles(synth.make_cluster(4, seed=43), seed=44)
    S = core.build_sites(torch.tensor(s.pos, dtype=DT), torch.tensor(s.mp_local, dtype=DT), PARAMS)
    i, j, sh = terms.mol_pairs(s.pos[:, 0], None, None)
    Vat = terms.atom_potential_pairs(S, i, j, torch.tensor(sh), PARAMS, None, None).numpy()
    x, q, mu, th = S["x"].numpy(), S["q"].numpy(), S["mu"].numpy(), S["th"].numpy()
    for mol in range(4):
        others = [k for k in range(4) if k != mol]
        for a in range(3):
            ref = KE * _phi_direct(x[mol, a], x[others].reshape(-1, 3), q[others].reshape(-1),
                                   mu[others].reshape(-1, 3), th[others].reshape(-1, 3, 3))
            assert abs(Vat[mol, a] - ref) < 1e-12 * abs(ref), (mol, a, Vat[mol, a], ref)


@pytest.fixture(scope="module")
def periodic_pair_ct():
    s = synth.with_general_multipoles(synth.make_box(2, 20.0, seed=37, jitter=1.5), seed=38)
    outs = []
    for alpha in (0.78, 0.9):
        o = {"rc": 7.4, "grid": 80, "order": 12, "ewald": alpha, "ct_original": True}
        outs.append(oracle.evaluate(s, o, forces=False, tol_D=1e-11))
    return outs


def test_periodic_acceptor_potential_is_alpha_independent(periodic_pair_ct):
    a, b = periodic_pair_ct
    va, vb = a["v_atoms"], b["v_atoms"]
    assert np.abs(va - vb).max() < 5e-7 * np.abs(va).max(), np.abs(va - vb).max()


def _fd_check(s, o, idx, h=1e-5):
    opts = dict(o or {}, ct_original=True)
    ref = oracle.evaluate(s, opts, tol_D=1e-12)
    F = ref["forces"]
    for (m, a, c) in idx:
        sp = synth.System(pos=s.pos.copy(), mp_local=s.mp_local, box=s.box)
        sm = synth.System(pos=s.pos.copy(), mp_local=s.mp_local, box=s.box)
        sp.pos[m, a, c] += h
        sm.pos[m, a, c] -= h
        ep = oracle.evaluate(sp, opts, forces=False, tol_D=1e-12)["terms"]["total"]
        em = oracle.evaluate(sm, opts, forces=False, tol_D=1e-12)["terms"]["total"]
        fd = -(ep - em) / (2 * h)
        assert abs(F[m, a, c] - fd) < 2e-6 * max(1.0, abs(fd)), ((m, a, c), F[m, a, c], fd)


def test_forces_are_minus_the_gradient_gas():
    s = synth.with_general_multipoles(synth.make_cluster(4, seed=45), seed=46)
    _fd_check(s, None, [(0, 0, 0), (1, 1, 2), (2, 2, 1), (3, 0, 2)])


def test_forces_are_minus_the_gradient_periodic():
    """64 waters at liquid density (12.6 A box, rc 4.3 A): every molecule
    transfers charge to its neighbours."""
    s = synth.with_general_multipoles(synth.make_box(4, 12.6, seed=47), seed=48)
    _fd_check(s, {"rc": 4.3, "grid": 16, "order": 5, "ewald": 0.5}, [(0, 0, 0), (13, 1, 2), (40, 2, 1)])
