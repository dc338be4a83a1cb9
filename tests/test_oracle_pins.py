"""Oracle pins against hand evaluations and invariances, one per function
whose formula no other pin fixes:

- lone-pair and local-frame geometry of build_sites (R3, R4): distances,
  angles, the lone-pair plane, the frame axes of a molecule laid out by hand,
  and the rotated multipoles through the potential they produce;
- exchange-repulsion (Technical Appendix, bond-bond, bond-lone pair, lone
  pair-lone pair; readings R14, R15) on collinear layouts in which every
  cosine is +1 or -1, written out term by term from the appendix formulas;
- dispersion and exchange-dispersion (Technical Appendix; R16, R17) for one
  atom-atom, one atom-lone pair and one lone pair-lone pair pair;
- the reduced charge transfer (Eqs. 13-16; R13) on a hand-laid donor and
  acceptor with given potentials, and V_int on a hand-laid molecule;
- the lone-pair potential of the gas phase against the textbook multipole
  potential q/r + mu.r/r^3 + Theta:rr/r^5;
- the periodic lone-pair potential, permanent field, induced dipoles and
  polarization energy: with the real-space part converged, the Ewald
  splitting parameter must drop out (alpha independence).

Each expected value below is evaluated from the paper's formula for the
specific layout (with the cosines and distances of that layout filled in),
not by calling the oracle's own expression.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import core, terms
from synth import PARAMS

DT = torch.float64
KE = PARAMS["ke"]


def _sites(mols):
    """Hand-built sites dict for terms.*_pairs: mols is a list of dicts with
    O, H1, H2, LP1, LP2 (3-vectors) and q (5 charges; midpoints between O and
    each H).  Dipoles and quadrupoles are zero."""
    x, lp, q = [], [], []
    for m in mols:
        O, H1, H2 = (np.asarray(m[k], float) for k in ("O", "H1", "H2"))
        x.append([O, H1, H2, 0.5 * (O + H1), 0.5 * (O + H2)])
        lp.append([m["LP1"], m["LP2"]])
        q.append(m.get("q", [-0.8, 0.2, 0.2, 0.2, 0.2]))
    M = len(mols)
    return {"x": torch.tensor(np.array(x), dtype=DT), "lp": torch.tensor(np.array(lp, float), dtype=DT),
            "q": torch.tensor(np.array(q, float), dtype=DT), "mu": torch.zeros((M, 5, 3), dtype=DT),
            "th": torch.zeros((M, 5, 3, 3), dtype=DT)}


PAIR = (np.array([0]), np.array([1]), torch.zeros((1, 3), dtype=DT))
FAR = 1.0e3


# ---------------------------------------------------------------------------
# Geometry (R3, R4)
# ---------------------------------------------------------------------------

def _body_molecule():
    r, h = synth.WATER_GEOM["r_oh"], math.radians(synth.WATER_GEOM["hoh_deg"]) / 2
    O = np.zeros(3)
    H1 = np.array([r * math.sin(h), 0.0, r * math.cos(h)])
    H2 = np.array([-r * math.sin(h), 0.0, r * math.cos(h)])
    return np.stack([O, H1, H2])


def test_lone_pairs_and_frames_of_a_hand_laid_molecule():
    """O at the origin, H1 and H2 in the xz plane symmetric about +z.  Then
    the O frame is the identity (z = bisector, x toward H1, y = z x x), the
    lone pairs sit at (0, +-d sin t, -d cos t) with t half the tetrahedral
    angle (plane of the lone pairs = yz, perpendicular to the HOH plane xz),
    H1's z axis points from H1 to O and its x axis toward H2 within the
    plane."""
    pos = _body_molecule()
    S = core.build_sites(torch.tensor(pos[None], dtype=DT), torch.zeros((1, 5, 10), dtype=DT), PARAMS)
    d, t = PARAMS["d_lp"], math.radians(PARAMS["lp_half_deg"])
    lp = S["lp"][0].numpy()
    np.testing.assert_allclose(lp[0], [0.0, d * math.sin(t), -d * math.cos(t)], atol=1e-14)
    np.testing.assert_allclose(lp[1], [0.0, -d * math.sin(t), -d * math.cos(t)], atol=1e-14)
    # |O-LP| = d, angle LP-O-LP = twice 54.7356 degrees (tetrahedral)
    for k in range(2):
        assert abs(np.linalg.norm(lp[k]) - d) < 1e-14
    cosang = lp[0] @ lp[1] / d ** 2
    assert abs(math.degrees(math.acos(cosang)) - 2 * 54.7356103172) < 1e-8
    R = S["R"][0].numpy()                          # (5, 3, 3), columns x, y, z
    np.testing.assert_allclose(R[0], np.eye(3), atol=1e-14)
    z1 = -pos[1] / np.linalg.norm(pos[1])
    x1 = (pos[2] - pos[1]) - ((pos[2] - pos[1]) @ z1) * z1
    x1 /= np.linalg.norm(x1)
    np.testing.assert_allclose(R[1][:, 2], z1, atol=1e-14)
    np.testing.assert_allclose(R[1][:, 0], x1, atol=1e-14)
    np.testing.assert_allclose(R[1][:, 1], np.cross(z1, x1), atol=1e-14)
    # midpoint frames are those of their hydrogen; H2 mirrors H1
    np.testing.assert_allclose(R[3], R[1], atol=1e-15)
    np.testing.assert_allclose(R[4], R[2], atol=1e-15)
    mirror = np.diag([-1.0, 1.0, 1.0])
    np.testing.assert_allclose(R[2][:, 2], mirror @ R[1][:, 2], atol=1e-14)
    np.testing.assert_allclose(R[2][:, 0], mirror @ R[1][:, 0], atol=1e-14)
    np.testing.assert_allclose(S["x"][0, 3].numpy(), 0.5 * pos[1], atol=1e-15)


def test_lone_pair_plane_is_perpendicular_to_the_molecule_in_any_orientation():
    s = synth.make_cluster(6, seed=31)
    S = core.build_sites(torch.tensor(s.pos, dtype=DT), torch.tensor(s.mp_local, dtype=DT), PARAMS)
    for m in range(6):
        O, H1, H2 = s.pos[m]
        l1, l2 = S["lp"][m].numpy()
        n_hoh = np.cross(H1 - O, H2 - O)
        n_hoh /= np.linalg.norm(n_hoh)
        b = (H1 - O) / np.linalg.norm(H1 - O) + (H2 - O) / np.linalg.norm(H2 - O)
        b /= np.linalg.norm(b)
        # the lone pairs differ along the HOH normal and share a component
        # opposite to the bisector
        dl = l1 - l2
        assert abs(abs(dl @ n_hoh) - np.linalg.norm(dl)) < 1e-12
        t = math.radians(PARAMS["lp_half_deg"])
        for l in (l1, l2):
            assert abs((l - O) @ b + PARAMS["d_lp"] * math.cos(t)) < 1e-12
        # handedness: LP1 - LP2 points along z_O x x_O with x_O toward H1
        y = np.cross(b, (H1 - O) - ((H1 - O) @ b) * b)
        assert dl @ y > 0


def _phi_direct(P, x, q, mu, th):
    """Textbook potential of point multipoles at P (traceless quadrupole,
    phi = q/r + mu.r/r^3 + Theta:rr/r^5)."""
    out = 0.0
    for k in range(len(q)):
        r = P - x[k]
        rn = np.linalg.norm(r)
        out += q[k] / rn + mu[k] @ r / rn ** 3 + r @ th[k] @ r / rn ** 5
    return out


def test_rotated_multipoles_reproduce_the_local_frame_potential():
    """The potential of a site's global multipole at a point equals the
    potential of its local-frame multipole at the same point expressed in the
    site's frame coordinates (general dipole and quadrupole components)."""
    s = synth.with_general_multipoles(synth.make_cluster(3, seed=32), seed=33)
    S = core.build_sites(torch.tensor(s.pos, dtype=DT), torch.tensor(s.mp_local, dtype=DT), PARAMS)
    rng = np.random.default_rng(34)
    for m in range(3):
        for k in range(5):
            xk = S["x"][m, k].numpy()
            R = S["R"][m, k].numpy()                  # columns = frame axes
            loc = s.mp_local[m, k]
            th_l = np.array([[loc[4], loc[7], loc[8]], [loc[7], loc[5], loc[9]], [loc[8], loc[9], loc[6]]])
            for _ in range(3):
                P = xk + rng.normal(size=3) * 2.0
                g = _phi_direct(P, [xk], [S["q"][m, k].item()], [S["mu"][m, k].numpy()], [S["th"][m, k].numpy()])
                l = _phi_direct(R.T @ (P - xk), [np.zeros(3)], [loc[0]], [loc[1:4]], [th_l])
                assert abs(g - l) < 1e-12 * max(1.0, abs(l)), (m, k, g, l)


# ---------------------------------------------------------------------------
# Exchange-repulsion (Technical Appendix; R14, R15)
# ---------------------------------------------------------------------------

def _P(**upd):
    P = dict(PARAMS)
    P.update(upd)
    return P


def _M2(ga, qa, na, gb, qb, nb):
    """M^2 = g_a g_b (1 - Q_a / N_a^val)(1 - Q_b / N_b^val)."""
    return ga * gb * (1 - qa / na) * (1 - qb / nb)


def test_bond_bond_repulsion_collinear():
    """Bond a-b of molecule A (O_A at 0, H_A at 1 on the x axis) against bond
    c-d of molecule B (H_B at 3, O_B at 4): the p orbitals lie along the
    bonds, every cosine is +1 or -1.  The second O-H bond of each molecule is
    far away (outside the cutoff).  Per atom pair (x, y) the overlap is
    Cs_x Cs_y + Cs_y Cp_x f cos_x + Cs_x Cp_y f cos_y + 2 Cp_x Cp_y cos_x cos_y,
    each cosine at the atom carrying the p orbital, between the p direction
    (along its bond, away from the atom) and the direction to the other atom."""
    P = _P(cp_h=0.3, n_lp=0.0)
    qA = [-0.8, 0.25, 0.2, 0.2, 0.2]
    qB = [-0.7, 0.3, 0.2, 0.2, 0.2]
    A = dict(O=[0, 0, 0], H1=[1, 0, 0], H2=[0, 0, -FAR], LP1=[0, FAR, 0], LP2=[0, -FAR, 0], q=qA)
    B = dict(O=[4, 0, 0], H1=[3, 0, 0], H2=[4, 0, FAR], LP1=[4, FAR, 0], LP2=[4, -FAR, 0], q=qB)
    E = float(terms.rep_pairs(_sites([A, B]), *PAIR, P, 20.0))
    cs_o, cp_o, cs_h, cp_h, f = P["cs_o"], P["cp_o"], P["cs_h"], P["cp_h"], P["rep_f"]
    rv_o, rv_h = P["rvdw_rep_o"], P["rvdw_rep_h"]
    # (atom of A, atom of B): distance, cos at A's atom, cos at B's atom, Cs/Cp/g/q/Nval of both
    o_oo = cs_o * cs_o + cs_o * cp_o * f * (+1) + cs_o * cp_o * f * (+1) + 2 * cp_o * cp_o * (+1) * (+1)
    o_oh = cs_o * cs_h + cs_h * cp_o * f * (+1) + cs_o * cp_h * f * (-1) + 2 * cp_o * cp_h * (+1) * (-1)
    o_ho = cs_h * cs_o + cs_o * cp_h * f * (-1) + cs_h * cp_o * f * (+1) + 2 * cp_h * cp_o * (-1) * (+1)
    o_hh = cs_h * cs_h + cs_h * cp_h * f * (-1) + cs_h * cp_h * f * (-1) + 2 * cp_h * cp_h * (-1) * (-1)
    go, gh, no, nh = P["g_o"], P["g_h"], P["nval_o"], P["nval_h"]
    pairs = [  # overlap, r, rvdw product, M^2
        (o_oo, 4.0, rv_o * rv_o, _M2(go, qA[0], no, go, qB[0], no)),
        (o_oh, 3.0, rv_o * rv_h, _M2(go, qA[0], no, gh, qB[1], nh)),
        (o_ho, 3.0, rv_h * rv_o, _M2(gh, qA[1], nh, go, qB[0], no)),
        (o_hh, 2.0, rv_h * rv_h, _M2(gh, qA[1], nh, gh, qB[1], nh)),
    ]
    O1 = sum(o * math.sqrt(m2) * math.exp(-P["rep_alpha"] * r / (4 * math.sqrt(rr))) for o, r, rr, m2 in pairs)
    O2 = sum(o * math.sqrt(m2) * math.exp(-P["rep_alpha2"] * r / (4 * math.sqrt(rr))) for o, r, rr, m2 in pairs)
    rmid = 3.0                                     # midpoints at 0.5 and 3.5
    ref = P["occ_bond"] ** 2 * (P["rep_c1"] * O1 ** 2 / rmid + P["rep_c2"] * O2 ** 2 / rmid ** 2)
    assert abs(E - ref) < 1e-12 * abs(ref), (E, ref)


def test_bond_bond_repulsion_collinear_reversed():
    """Same line, B's bond turned around (O_B at 3, H_B at 4): the cosines at
    B's atoms change sign."""
    P = _P(cp_h=0.3, n_lp=0.0)
    q = [-0.8, 0.2, 0.2, 0.2, 0.2]
    A = dict(O=[0, 0, 0], H1=[1, 0, 0], H2=[0, 0, -FAR], LP1=[0, FAR, 0], LP2=[0, -FAR, 0], q=q)
    B = dict(O=[3, 0, 0], H1=[4, 0, 0], H2=[3, 0, FAR], LP1=[3, FAR, 0], LP2=[3, -FAR, 0], q=q)
    E = float(terms.rep_pairs(_sites([A, B]), *PAIR, P, 20.0))
    cs_o, cp_o, cs_h, cp_h, f = P["cs_o"], P["cp_o"], P["cs_h"], P["cp_h"], P["rep_f"]
    rv_o, rv_h = P["rvdw_rep_o"], P["rvdw_rep_h"]
    # p(O_A) = +x, p(H_A) = -x, p(O_B) = +x, p(H_B) = -x
    o_oo = cs_o * cs_o + cs_o * cp_o * f * (+1) + cs_o * cp_o * f * (-1) + 2 * cp_o * cp_o * (+1) * (-1)
    o_oh = cs_o * cs_h + cs_h * cp_o * f * (+1) + cs_o * cp_h * f * (+1) + 2 * cp_o * cp_h * (+1) * (+1)
    o_ho = cs_h * cs_o + cs_o * cp_h * f * (-1) + cs_h * cp_o * f * (-1) + 2 * cp_h * cp_o * (-1) * (-1)
    o_hh = cs_h * cs_h + cs_h * cp_h * f * (-1) + cs_h * cp_h * f * (+1) + 2 * cp_h * cp_h * (-1) * (+1)
    m_oo = _M2(P["g_o"], -0.8, P["nval_o"], P["g_o"], -0.8, P["nval_o"])
    m_oh = _M2(P["g_o"], -0.8, P["nval_o"], P["g_h"], 0.2, P["nval_h"])
    m_hh = _M2(P["g_h"], 0.2, P["nval_h"], P["g_h"], 0.2, P["nval_h"])
    pairs = [(o_oo, 3.0, rv_o * rv_o, m_oo), (o_oh, 4.0, rv_o * rv_h, m_oh),
             (o_ho, 2.0, rv_h * rv_o, m_oh), (o_hh, 3.0, rv_h * rv_h, m_hh)]
    O1 = sum(o * math.sqrt(m2) * math.exp(-P["rep_alpha"] * r / (4 * math.sqrt(rr))) for o, r, rr, m2 in pairs)
    O2 = sum(o * math.sqrt(m2) * math.exp(-P["rep_alpha2"] * r / (4 * math.sqrt(rr))) for o, r, rr, m2 in pairs)
    ref = P["occ_bond"] ** 2 * (P["rep_c1"] * O1 ** 2 / 3.0 + P["rep_c2"] * O2 ** 2 / 9.0)
    assert abs(E - ref) < 1e-12 * abs(ref), (E, ref)


def test_bond_lone_pair_repulsion_collinear():
    """Bond O_A-H_A (0 and 1 on the x axis) against the lone pair of B whose
    carrier O_B sits at 4 and which points back toward A (at 3.5).  Every
    other bond and lone pair is far away.  Per bond atom a the overlap is
    Cs_a Cs_j + Cs_j Cp_a f cos(AB, AC) + Cs_a Cp_j f cos(CA, CI)
    + f Cp_a Cp_j cos(AB, AC) cos(CA, CI), rho = r_ac / (4 sqrt(rv_a rv_lp))
    with r_ac the distance to the carrier, M^2 = g_a g_c (1 - Q_a/N_a)
    (1 - n/N_c), and the energy Occ n (C1 O1^2/r + C2 O2^2/r^2) with r the
    distance from the bond midpoint to the lone pair."""
    P = _P(cp_h=0.3)
    q = [-0.8, 0.2, 0.2, 0.2, 0.2]
    A = dict(O=[0, 0, 0], H1=[1, 0, 0], H2=[0, 0, -FAR], LP1=[0, FAR, 0], LP2=[0, -FAR, 0], q=q)
    B = dict(O=[4, 0, 0], H1=[4, FAR, 0], H2=[4, -FAR, 0], LP1=[3.5, 0, 0], LP2=[4, 0, FAR], q=q)
    E = float(terms.rep_pairs(_sites([A, B]), *PAIR, P, 20.0))
    cs_o, cp_o, cs_h, cp_h, f = P["cs_o"], P["cp_o"], P["cs_h"], P["cp_h"], P["rep_f"]
    cs_l, cp_l, n = P["cs_lp"], P["cp_lp"], P["n_lp"]
    # a = O_A: p = +x, A->C = +x (cos +1); C->A = -x, C->I = -x (cos +1)
    o_o = cs_o * cs_l + cs_l * cp_o * f * (+1) + cs_o * cp_l * f * (+1) + f * cp_o * cp_l * (+1) * (+1)
    # a = H_A: p = -x, H->C = +x (cos -1); C->H = -x, C->I = -x (cos +1)
    o_h = cs_h * cs_l + cs_l * cp_h * f * (-1) + cs_h * cp_l * f * (+1) + f * cp_h * cp_l * (-1) * (+1)
    cf_lp = 1 - n / P["nval_o"]
    m_o = P["g_o"] * P["g_o"] * (1 + 0.8 / P["nval_o"]) * cf_lp
    m_h = P["g_h"] * P["g_o"] * (1 - 0.2 / P["nval_h"]) * cf_lp
    rv_o, rv_h, rv_l = P["rvdw_rep_o"], P["rvdw_rep_h"], P["rvdw_rep_lp"]
    pairs = [(o_o, 4.0, rv_o * rv_l, m_o), (o_h, 3.0, rv_h * rv_l, m_h)]
    O1 = sum(o * math.sqrt(m2) * math.exp(-P["rep_alpha"] * r / (4 * math.sqrt(rr))) for o, r, rr, m2 in pairs)
    O2 = sum(o * math.sqrt(m2) * math.exp(-P["rep_alpha2"] * r / (4 * math.sqrt(rr))) for o, r, rr, m2 in pairs)
    r = 3.0                                        # bond midpoint 0.5, lone pair 3.5
    ref = P["occ_bond"] * n * (P["rep_c1"] * O1 ** 2 / r + P["rep_c2"] * O2 ** 2 / r ** 2)
    assert abs(E - ref) < 1e-12 * abs(ref), (E, ref)


def test_lone_pair_lone_pair_repulsion_collinear():
    """Lone pair I of A (carrier at 0, I at 0.5) against lone pair J of B
    (carrier at 4, J at 3.5); bonds switched off (Occ = 0), the other lone
    pairs far.  O_ij = Cs Cs + Cs Cp f cos(BJ, BI) + Cs Cp f cos(AI, AJ)
    + 2 Cp Cp cos(AI, AJ) cos(BJ, BI), rho from the carrier distance, the
    1/r factors from the lone-pair distance."""
    P = _P(occ_bond=0.0)
    q = [-0.8, 0.2, 0.2, 0.2, 0.2]
    A = dict(O=[0, 0, 0], H1=[0, FAR, 0], H2=[0, -FAR, 0], LP1=[0.5, 0, 0], LP2=[0, 0, FAR], q=q)
    B = dict(O=[4, 0, 0], H1=[4, FAR, 0], H2=[4, -FAR, 0], LP1=[4, 0, -FAR], LP2=[3.5, 0, 0], q=q)
    E = float(terms.rep_pairs(_sites([A, B]), *PAIR, P, 20.0))
    cs, cp, f, n = P["cs_lp"], P["cp_lp"], P["rep_f"], P["n_lp"]
    o = cs * cs + cs * cp * f * (+1) + cs * cp * f * (+1) + 2 * cp * cp * (+1) * (+1)
    M = math.sqrt(P["g_o"] ** 2 * (1 - n / P["nval_o"]) ** 2)
    rho = 4.0 / (4 * P["rvdw_rep_lp"])
    O1 = o * M * math.exp(-P["rep_alpha"] * rho)
    O2 = o * M * math.exp(-P["rep_alpha2"] * rho)
    ref = n * n * (P["rep_c1"] * O1 ** 2 / 3.0 + P["rep_c2"] * O2 ** 2 / 9.0)
    assert abs(E - ref) < 1e-12 * abs(ref), (E, ref)


# ---------------------------------------------------------------------------
# Dispersion and exchange-dispersion (Technical Appendix; R16, R17)
# ---------------------------------------------------------------------------

def _lone_pair_layout(ia, ib, r):
    """Molecule A's five points (O, H1, H2, LP1, LP2) far apart from each
    other; B's point ib at distance r from A's point ia, B's other points far
    from everything.  Only that one point pair is inside the cutoff."""
    a_pts = [[0, 0, 0], [FAR, 0, 0], [0, FAR, 0], [0, 0, FAR], [-FAR, 0, 0]]
    b_pts = [[5 * FAR + 100 * k, 5 * FAR, 5 * FAR] for k in range(5)]
    b_pts[ib] = list(np.asarray(a_pts[ia], float) + np.array([0.6, -0.8, 0.0]) * r)
    qA = [-0.78, 0.21, 0.17, 0.2, 0.2]
    qB = [-0.83, 0.19, 0.23, 0.2, 0.2]
    A = dict(O=a_pts[0], H1=a_pts[1], H2=a_pts[2], LP1=a_pts[3], LP2=a_pts[4], q=qA)
    B = dict(O=b_pts[0], H1=b_pts[1], H2=b_pts[2], LP1=b_pts[3], LP2=b_pts[4], q=qB)
    return _sites([A, B]), qA, qB


def _damped(P, r, rvi, rvj):
    m = r / (2 * math.sqrt(rvi * rvj))
    d = (rvi + rvj) * P["disp_alpha"] / r - 1.0
    return (P["c6"] * math.exp(-P["gamma6"] * d) / m ** 6 + P["c8"] * math.exp(-P["gamma8"] * d) / m ** 8
            + P["c10"] * math.exp(-P["gamma10"] * d) / m ** 10), m


@pytest.mark.parametrize("kind", ["at-at", "at-lp", "lp-at", "lp-lp"])
def test_dispersion_and_exchange_dispersion_single_pair(kind):
    P = PARAMS
    r = 2.9
    ia, ib = {"at-at": (0, 1), "at-lp": (2, 3), "lp-at": (4, 0), "lp-lp": (4, 4)}[kind]
    S, qA, qB = _lone_pair_layout(ia, ib, r)
    ed, ex = terms.disp_pairs(S, *PAIR, P, 20.0)
    rv = [P["rvdw_disp_o"], P["rvdw_disp_h"], P["rvdw_disp_h"], P["rvdw_disp_lp"], P["rvdw_disp_lp"]]
    beta = [P["beta_o"], P["beta_h"], P["beta_h"], P["beta_o"], P["beta_o"]]   # lone pairs: carrier O
    nval = [P["nval_o"], P["nval_h"], P["nval_h"], P["nval_o"], P["nval_o"]]
    carrier = [0, 1, 2, 0, 0]
    cfA = 1 - qA[carrier[ia]] / nval[ia]
    cfB = 1 - qB[carrier[ib]] / nval[ib]
    f, m = _damped(P, r, rv[ia], rv[ib])
    n = P["n_lp"]
    K = beta[ia] * beta[ib] * cfA * cfB
    if kind == "at-at":
        ref_d = -beta[ia] * beta[ib] * f
        ref_x = P["xd_c1"] * K * math.exp(-P["xd_a1"] * m)
    elif kind == "lp-lp":
        ref_d = -(n * n / 4) * f
        ref_x = (n * n / 4) * P["xd_c2"] * K * math.exp(-P["xd_a2"] * m)
    else:
        ref_d = -(P["disp_delta"] / 2) * f
        ref_x = (n / 2) * P["xd_c3"] * K * math.exp(-P["xd_a3"] * m)
    assert abs(float(ed) - ref_d) < 1e-12 * abs(ref_d), (kind, float(ed), ref_d)
    assert abs(float(ex) - ref_x) < 1e-12 * abs(ref_x), (kind, float(ex), ref_x)


# ---------------------------------------------------------------------------
# Reduced charge transfer (Eqs. 13-16; R13) and V_int
# ---------------------------------------------------------------------------

def test_reduced_charge_transfer_hand_case():
    """Donor A (carrier O at the origin, lone pairs along +x and +y) and
    acceptor B (O at (3,0,0), H1 at (3,4,0), H2 at (2,0,0)), and the mirror
    transfer from B's lone pairs (along -x and +z) to A's X-H bonds (A's H1 at
    (-1,0,0), H2 at (3,0,4)).  The potentials V on the lone pairs and V_int
    on the atoms are given numbers.  Distances 2, 3, 4, 5 and cosines 0, 3/5,
    4/5, 1, with cos(alpha) and cos(beta) different for the same lone pair."""
    P = PARAMS
    A = dict(O=[0, 0, 0], H1=[-1, 0, 0], H2=[3, 0, 4], LP1=[0.5, 0, 0], LP2=[0, 0.5, 0])
    B = dict(O=[3, 0, 0], H1=[3, 4, 0], H2=[2, 0, 0], LP1=[2.5, 0, 0], LP2=[3, 0, 0.5])
    S = _sites([A, B])
    V = torch.tensor([[-20.0, -30.0], [-25.0, -15.0]], dtype=DT)
    Vint = torch.tensor([[-50.0, 30.0, 35.0], [-45.0, 28.0, 33.0]], dtype=DT)
    E, min_de = terms.ct_pairs(S, V, Vint, *PAIR, P, 9.0)
    eta, t, m, n = P["ct_eta"], P["ct_t"], P["ct_m"], P["n_lp"]
    cs, cp = P["cs_lp"], P["cp_lp"]
    rvo, rvh = P["rvdw_ct_o"], P["rvdw_ct_h"]
    ae, ah = P["ct_ae"], P["ct_ah"]

    def transfer(V_lp, cos_a, r1, Vint_a1, acc):
        """One lone pair against the acceptor's X-H bonds: acc = [(r_c-a2, cos beta, Vint(a2))]."""
        total = 0.0
        e1 = math.exp(-eta * r1 / (2 * math.sqrt(rvo * rvo))) * (Vint_a1 - V_lp) * (cs * t + cp * m * cos_a)
        for r2, cos_b, Vint_a2 in acc:
            e2 = math.exp(-eta * r2 / (2 * math.sqrt(rvo * rvh))) * (Vint_a2 - V_lp) * (cs * t + cp * m * cos_b)
            total += -n * (e1 - e2) ** 2 / (ae + V_lp - ah)
        return total

    # A's lone pairs (+x, +y) -> B: O_B at distance 3, H1_B at 5, H2_B at 2
    ref = transfer(-20.0, 1.0, 3.0, -45.0, [(5.0, 0.6, 28.0), (2.0, 1.0, 33.0)])
    ref += transfer(-30.0, 0.0, 3.0, -45.0, [(5.0, 0.8, 28.0), (2.0, 0.0, 33.0)])
    # B's lone pairs (-x, +z) -> A: O_A at distance 3, H1_A at 4 (along -x), H2_A at 4 (along +z)
    ref += transfer(-25.0, 1.0, 3.0, -50.0, [(4.0, 1.0, 30.0), (4.0, 0.0, 35.0)])
    ref += transfer(-15.0, 0.0, 3.0, -50.0, [(4.0, 0.0, 30.0), (4.0, 1.0, 35.0)])
    assert abs(float(E) - ref) < 1e-12 * abs(ref), (float(E), ref)
    assert abs(min_de - (ae - 30.0 - ah)) < 1e-12
    # beyond the cutoff (carrier to acceptor heavy atom) nothing is transferred
    E_far, _ = terms.ct_pairs(S, V, Vint, *PAIR, P, 2.9)
    assert float(E_far) == 0.0


def test_v_int_hand_case():
    """Coulomb potential at O, H1, H2 from the charges of the other four
    sites of the same molecule (R13)."""
    q = [-0.8, 0.25, 0.15, 0.22, 0.18]
    S = _sites([dict(O=[0, 0, 0], H1=[1, 0, 0], H2=[0, 1, 0], LP1=[0, 0, 1], LP2=[0, 0, -1], q=q)])
    V = terms.v_int(S, PARAMS)[0].numpy()
    h = 1 / math.sqrt(2)
    ref_o = q[1] / 1 + q[2] / 1 + q[3] / 0.5 + q[4] / 0.5
    ref_h1 = q[0] / 1 + q[2] * h + q[3] / 0.5 + q[4] / math.sqrt(1.25)
    ref_h2 = q[0] / 1 + q[1] * h + q[3] / math.sqrt(1.25) + q[4] / 0.5
    np.testing.assert_allclose(V, KE * np.array([ref_o, ref_h1, ref_h2]), rtol=1e-14)


def test_gas_lone_pair_potential_is_the_multipole_potential():
    """V at every lone pair = sum over the sites of the other molecules of
    q/r + mu.r/r^3 + Theta:rr/r^5 (times k_e), general multipoles."""
    s = synth.with_general_multipoles(synth.make_cluster(4, seed=35), seed=36)
    S = core.build_sites(torch.tensor(s.pos, dtype=DT), torch.tensor(s.mp_local, dtype=DT), PARAMS)
    i, j, sh = terms.mol_pairs(s.pos[:, 0], None, None)
    V = terms.lp_potential_pairs(S, i, j, torch.tensor(sh), PARAMS, None, None).numpy()
    x, q, mu, th = S["x"].numpy(), S["q"].numpy(), S["mu"].numpy(), S["th"].numpy()
    for m in range(4):
        others = [k for k in range(4) if k != m]
        xs = x[others].reshape(-1, 3)
        for l in range(2):
            ref = KE * _phi_direct(S["lp"][m, l].numpy(), xs, q[others].reshape(-1), mu[others].reshape(-1, 3),
                                   th[others].reshape(-1, 3, 3))
            assert abs(V[m, l] - ref) < 1e-12 * abs(ref), (m, l, V[m, l], ref)


# ---------------------------------------------------------------------------
# Periodic potentials and polarization: the Ewald splitting drops out
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def periodic_pair():
    """8 waters (general multipoles) in a 20 A box, real-space cutoff 7.4 A
    (erfc(alpha rc) < 1e-13 for both alphas), PCG to 1e-11 D, evaluated at two
    Ewald splitting parameters.  The reciprocal sums use B-splines of order 12
    on an 80^3 grid so that their discretisation error (which falls slowly
    for quadrupoles at order 5) stays near 1e-8 of the values compared."""
    s = synth.with_general_multipoles(synth.make_box(2, 20.0, seed=37, jitter=1.5), seed=38)
    outs = []
    for alpha in (0.78, 0.9):
        o = {"rc": 7.4, "grid": 80, "order": 12, "ewald": alpha}
        outs.append(oracle.evaluate(s, o, forces=False, tol_D=1e-11))
    return outs


def test_periodic_lone_pair_potential_is_alpha_independent(periodic_pair):
    a, b = periodic_pair
    va, vb = a["v_lp"], b["v_lp"]
    assert np.abs(va - vb).max() < 5e-7 * np.abs(va).max(), np.abs(va - vb).max()


def test_periodic_field_dipoles_and_pol_energy_are_alpha_independent(periodic_pair):
    a, b = periodic_pair
    ea, eb = a["efield"], b["efield"]
    assert np.abs(ea - eb).max() < 5e-6 * np.abs(ea).max()
    assert np.abs(a["mu"] - b["mu"]).max() < 5e-6 * np.abs(a["mu"]).max()
    pa, pb = a["terms"]["pol"], b["terms"]["pol"]
    assert abs(pa - pb) < 5e-7 * abs(pa), (pa, pb)
    # the multipole energy of this sparse box is a small remainder of parts
    # of order 1e3 kcal/mol, so its bound is wider
    assert abs(a["terms"]["elec"] - b["terms"]["elec"]) < 1e-5 * abs(a["terms"]["elec"])
