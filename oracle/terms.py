"""Oracle energy terms of the SIBFA intermolecular potential (FP64).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg; never by the product path.

Every function returns an energy (kcal/mol) as a differentiable function of
the atom positions; forces are taken by automatic differentiation in
evaluate.py.  Terms follow Eq. 1 (E_inter as five contributions):
electrostatics with penetration (Eq. 2 and the section on multipolar
electrostatics), exchange-repulsion (Technical Appendix, bond-bond, lp-lp and
bond-lp), polarization (Technical Appendix, E_pol = 1/2 mu T mu - mu E),
reduced charge transfer (Eqs. 13-16) and dispersion with exchange-dispersion
(Technical Appendix).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import ewald as ew
from .core import (DT, dipole_dipole_energy, dipole_mp_energy, g_bare, g_erf, g_erfc,
                   g_exp, g_thole, mp_pair_energy, mp_potential, t64, tensors)

# ---------------------------------------------------------------------------
# Per-site parameter arrays for one water (site order O, H1, H2, M1, M2).
# ---------------------------------------------------------------------------


def site_tables(P):
    a_o, a_h = P["alpha_o"], P["alpha_h"]
    return {
        "z": t64([P["z_o"], P["z_h"], P["z_h"], 0.0, 0.0]),
        "is_atom": t64([1.0, 1.0, 1.0, 0.0, 0.0]),
        "b": t64([P["b_o"], P["b_h"], P["b_h"], 0.0, 0.0]),
        "alpha_damp": t64([a_o, a_h, a_h, P["alpha_m_damp"], P["alpha_m_damp"]]),
        "alpha_pol": t64([a_o, a_h, a_h]),
    }


def valence(S, P):
    """N_k = Z_k - q_k on atom sites, 0 on the bond midpoints."""
    tb = site_tables(P)
    return (tb["z"] - S["q"]) * tb["is_atom"]


# ---------------------------------------------------------------------------
# Molecule pairs (minimum image in a periodic box, all pairs in the gas phase)
# ---------------------------------------------------------------------------


def mol_pairs(O, box, cut):
    """Pairs i<j whose O-O distance is below `cut`, with the image shift that
    must be added to molecule j.  O: (M, 3) numpy.  box: edge lengths, or a
    3x3 cell matrix (columns = cell vectors; nearest image in fractional
    coordinates, exact for the nearly orthogonal cells used here)."""
    M = O.shape[0]
    if box is None:
        i, j = np.triu_indices(M, 1)
        return i, j, np.zeros((i.size, 3))
    box = np.asarray(box, dtype=np.float64)
    cell = box if box.ndim == 2 else None
    Is, Js, Ss = [], [], []
    for i0 in range(0, M, 256):
        i1 = min(M, i0 + 256)
        d = O[None, :, :] - O[i0:i1, None, :]
        if cell is None:
            sh = -box * np.round(d / box)
        else:
            sh = -np.round(d @ np.linalg.inv(cell).T) @ cell.T
        d = d + sh
        r2 = np.einsum("ijk,ijk->ij", d, d)
        ii, jj = np.nonzero(r2 < cut * cut)
        ii = ii + i0
        keep = jj > ii
        Is.append(ii[keep])
        Js.append(jj[keep])
        Ss.append(sh[ii[keep] - i0, jj[keep]])
    return np.concatenate(Is), np.concatenate(Js), np.concatenate(Ss)


def _take(S, idx, shift=None):
    out = {k: S[k][idx] for k in ("x", "lp", "q", "mu", "th")}
    if shift is not None:
        out["x"] = out["x"] + shift[:, None, :]
        out["lp"] = out["lp"] + shift[:, None, :]
    return out


def _mask(rn, rc):
    if rc is None:
        return torch.ones_like(rn)
    return (rn < rc).to(DT)


def _norm(v):
    return torch.linalg.vector_norm(v, dim=-1)


# ---------------------------------------------------------------------------
# Electrostatics and penetration (real space / gas phase)
# ---------------------------------------------------------------------------


def elec_pen_pairs(S, i, j, sh, P, rc, alpha):
    """Intermolecular multipole energy (erfc kernel if alpha, else 1/r) and the
    penetration correction over the 5x5 site pairs of each molecule pair.

    Penetration (reading of the charge-charge*, charge-dipole* and
    charge-quadrupole* corrections): an atom site carries a nucleus Z and a
    valence population N = Z - q whose cloud interacts through
    (1 - exp(-b r))/r.  Hence for charges q* = q + N exp(-b r), and the charge
    of a meets the dipole and quadrupole of b with an extra N_a exp(-b_a r)/r
    kernel.  Bond midpoints carry no valence (N = 0).
    """
    A, B = _take(S, i), _take(S, j, sh)
    r = A["x"][:, :, None, :] - B["x"][:, None, :, :]
    rn = _norm(r)
    m = _mask(rn, rc)
    g = g_erfc(rn, alpha, 4) if alpha is not None else g_bare(rn, 4)
    T = tensors(r, g, 4)
    U = mp_pair_energy(T, A["q"][:, :, None], A["mu"][:, :, None, :], A["th"][:, :, None, :, :],
                       B["q"][:, None, :], B["mu"][:, None, :, :], B["th"][:, None, :, :, :])
    e_elec = P["ke"] * (U * m).sum()

    tb = site_tables(P)
    NA = valence(A, P)[:, :, None]
    NB = valence(B, P)[:, None, :]
    ba = tb["b"][None, :, None]
    bb = tb["b"][None, None, :]
    ea, eb = torch.exp(-ba * rn), torch.exp(-bb * rn)
    qa, qb = A["q"][:, :, None], B["q"][:, None, :]
    qq = (qa * NB * eb + qb * NA * ea + NA * NB * ea * eb) / rn
    Ta = tensors(r, g_exp(rn, ba, 2), 2)
    Tb = tensors(-r, g_exp(rn, bb, 2), 2)
    zero = torch.zeros_like(rn)
    phi_b = mp_potential(Ta, zero, B["mu"][:, None, :, :], B["th"][:, None, :, :, :])
    phi_a = mp_potential(Tb, zero, A["mu"][:, :, None, :], A["th"][:, :, None, :, :])
    pen = qq + NA * phi_b + NB * phi_a
    e_pen = P["ke"] * (pen * m).sum()
    return e_elec, e_pen


def elec_periodic_corrections(S, P, alpha, G, box, K, order):
    """Reciprocal energy + Gaussian self energy - erf part of intramolecular
    site pairs (the potential is intermolecular, Eq. 1)."""
    M = S["q"].shape[0]
    x = S["x"].reshape(-1, 3)
    Q = ew.spread(x, S["q"].reshape(-1), S["mu"].reshape(-1, 3), S["th"].reshape(-1, 3, 3), box, K, order)
    e_rec = ew.grid_energy(Q, G)
    e_self = ew.self_energy(S["q"].reshape(-1), S["mu"].reshape(-1, 3), S["th"].reshape(-1, 3, 3), alpha, P["ke"])
    ia, ib = np.triu_indices(5, 1)
    r = S["x"][:, ia] - S["x"][:, ib]
    T = tensors(r, g_erf(_norm(r), alpha, 4), 4)
    U = mp_pair_energy(T, S["q"][:, ia], S["mu"][:, ia], S["th"][:, ia],
                       S["q"][:, ib], S["mu"][:, ib], S["th"][:, ib])
    e_excl = P["ke"] * U.sum()
    return e_rec - e_excl + e_self, Q


# ---------------------------------------------------------------------------
# Potential on the lone pairs from the permanent multipoles of all other
# molecules (needed by charge transfer, Eqs. 13-16).
# ---------------------------------------------------------------------------


def lp_potential_pairs(S, i, j, sh, P, rc, alpha):
    """Real-space / gas-phase contribution to V at the lone pairs, returned as
    an (M, 2) tensor (both molecules of every pair receive their share)."""
    M = S["q"].shape[0]
    A, B = _take(S, i), _take(S, j, sh)
    V = torch.zeros((M, 2), dtype=DT)

    def one(lp, src):
        r = lp[:, :, None, :] - src["x"][:, None, :, :]
        rn = _norm(r)
        g = g_erfc(rn, alpha, 2) if alpha is not None else g_bare(rn, 2)
        T = tensors(r, g, 2)
        phi = mp_potential(T, src["q"][:, None, :], src["mu"][:, None, :, :], src["th"][:, None, :, :, :])
        return (phi * _mask(rn, rc)).sum(-1) * P["ke"]

    V = V.index_add(0, torch.as_tensor(i), one(A["lp"], B))
    V = V.index_add(0, torch.as_tensor(j), one(B["lp"], A))
    return V


def lp_potential_periodic(S, P, alpha, Psi, box, K, order):
    """Reciprocal potential at the lone pairs minus the erf part of the own
    molecule's sites."""
    M = S["q"].shape[0]
    phi = ew.potential_derivs(S["lp"].reshape(-1, 3), Psi, box, K, order, 0)["phi"].reshape(M, 2)
    r = S["lp"][:, :, None, :] - S["x"][:, None, :, :]
    T = tensors(r, g_erf(_norm(r), alpha, 2), 2)
    own = mp_potential(T, S["q"][:, None, :], S["mu"][:, None, :, :], S["th"][:, None, :, :, :]).sum(-1)
    return phi - P["ke"] * own


def atom_potential_pairs(S, i, j, sh, P, rc, alpha):
    """Real-space / gas-phase potential at O, H1, H2 from the permanent
    multipoles of the other molecule of every pair, (M, 3): the acceptor
    potentials V_a of the original charge transfer (CT section; same kernel
    and per-site-pair cutoff as the lone-pair potential)."""
    M = S["q"].shape[0]
    A, B = _take(S, i), _take(S, j, sh)

    def one(at, src):
        r = at[:, :, None, :] - src["x"][:, None, :, :]
        rn = _norm(r)
        g = g_erfc(rn, alpha, 2) if alpha is not None else g_bare(rn, 2)
        T = tensors(r, g, 2)
        phi = mp_potential(T, src["q"][:, None, :], src["mu"][:, None, :, :], src["th"][:, None, :, :, :])
        return (phi * _mask(rn, rc)).sum(-1) * P["ke"]

    V = torch.zeros((M, 3), dtype=DT)
    V = V.index_add(0, torch.as_tensor(i), one(A["x"][:, :3], B))
    V = V.index_add(0, torch.as_tensor(j), one(B["x"][:, :3], A))
    return V


def atom_potential_periodic(S, P, alpha, Psi, box, K, order):
    """Reciprocal potential at O, H1, H2 minus the own molecule's part: the erf
    part of its other four sites and the Gaussian self potential of the atom's
    own charge, 2 alpha / sqrt(pi) q (its own dipole and traceless quadrupole
    have none at their centre)."""
    M = S["q"].shape[0]
    phi = ew.potential_derivs(S["x"][:, :3].reshape(-1, 3), Psi, box, K, order, 0)["phi"].reshape(M, 3)
    out = []
    for a in range(3):
        others = [t for t in range(5) if t != a]
        r = S["x"][:, a:a + 1, :] - S["x"][:, others, :]
        T = tensors(r, g_erf(_norm(r), alpha, 2), 2)
        own = mp_potential(T, S["q"][:, others], S["mu"][:, others], S["th"][:, others]).sum(-1)
        out.append(own + 2.0 * alpha / math.sqrt(math.pi) * S["q"][:, a])
    return phi - P["ke"] * torch.stack(out, -1)


# ---------------------------------------------------------------------------
# Charge transfer, reduced form (Eqs. 13-16)
# ---------------------------------------------------------------------------


def v_int(S, P):
    """Intramolecular potential on O, H1, H2: Coulomb potential from the
    charges of the other four sites of the same molecule (reading of the
    V_int approximation)."""
    x, q = S["x"], S["q"]
    out = []
    for a in range(3):
        v = 0.0
        for s in range(5):
            if s == a:
                continue
            v = v + q[:, s] / _norm(x[:, a] - x[:, s])
        out.append(P["ke"] * v)
    return torch.stack(out, -1)            # (M, 3)


def _cos(u, v):
    return (u * v).sum(-1) / (_norm(u) * _norm(v))


def ct_pairs(S, V, Vint, i, j, sh, P, rc):
    """sum over donor lone pairs l and acceptor X-H bonds k of other molecules
    (carrier-to-heavy-atom distance below rc) of -n (e1 - e2)^2 / dE with
    e1 = exp(-eta rho1) (Vint(a1) - V_l)(Cs t + Cp m cos alpha),
    e2 = exp(-eta rho2) (Vint(a2) - V_l)(Cs t + Cp m cos beta),
    dE = ae + V_l - ah."""
    n = P["n_lp"]
    cs, cp = P["cs_lp"], P["cp_lp"]
    t, mm = P["ct_t"], P["ct_m"]
    eta = P["ct_eta"]
    rvo, rvh = P["rvdw_ct_o"], P["rvdw_ct_h"]

    def direction(D, Ad, VD, VintA):
        c = D["x"][:, 0]                                   # carrier O (C,3)
        lp = D["lp"]                                       # (C,2,3)
        a1 = Ad["x"][:, 0]                                 # (C,3)
        a2 = Ad["x"][:, 1:3]                               # (C,2,3) H1, H2
        r1 = _norm(a1 - c)                                 # (C,)
        m = _mask(r1, rc)
        rho1 = r1 / (2.0 * math.sqrt(rvo * rvo))
        rho2 = _norm(a2 - c[:, None]) / (2.0 * math.sqrt(rvo * rvh))   # (C,2)
        u = lp - c[:, None]                                # (C,2,3)
        cos_a = _cos(u, (a1 - c)[:, None, :])              # (C,2)  [lp]
        cos_b = _cos(u[:, :, None, :], (a2 - c[:, None])[:, None, :, :])   # (C,2lp,2k)
        Vl = VD[:, :, None]                                # (C,2,1)
        e1 = (torch.exp(-eta * rho1)[:, None, None] * (VintA[:, 0][:, None, None] - Vl)
              * (cs * t + cp * mm * cos_a[:, :, None]))
        e2 = (torch.exp(-eta * rho2)[:, None, :] * (VintA[:, 1:3][:, None, :] - Vl)
              * (cs * t + cp * mm * cos_b))
        dE = P["ct_ae"] + Vl - P["ct_ah"]
        e = -n * (e1 - e2) ** 2 / dE
        return (e.sum((1, 2)) * m).sum(), dE

    A, B = _take(S, i), _take(S, j, sh)
    ia, ja = torch.as_tensor(i), torch.as_tensor(j)
    e_ab, d1 = direction(A, B, V[ia], Vint[ja])
    e_ba, d2 = direction(B, A, V[ja], Vint[ia])
    min_de = min(float(d1.detach().min()) if d1.numel() else 1.0,
                 float(d2.detach().min()) if d2.numel() else 1.0)
    return e_ab + e_ba, min_de


def ct_pairs_original(S, V, Vat, Vint, i, j, sh, P, rc):
    """The original many-body charge transfer (CT section, before its
    reduction): as ct_pairs, with the acceptor potentials kept,
    e1 = exp(-eta rho1) (Vint(a1) + V*(a1) - V_l)(Cs t + Cp m cos alpha),
    e2 = exp(-eta rho2) (Vint(a2) + V*(a2) - V_l)(Cs t + Cp m cos beta),
    dE = ae + V_l - (ah + V(a1)),
    where V(a) = Vat is the potential at acceptor atom a from every molecule
    but its own, and V*(a) = V(a) minus the potential at a of the donor's
    molecule (its five multipole sites, bare, at the pair's image)."""
    n = P["n_lp"]
    cs, cp = P["cs_lp"], P["cp_lp"]
    t, mm = P["ct_t"], P["ct_m"]
    eta = P["ct_eta"]
    rvo, rvh = P["rvdw_ct_o"], P["rvdw_ct_h"]

    def donor_potential(D, at):
        """Bare potential of the donor's sites at the acceptor atoms (C, 3)."""
        r = at[:, :, None, :] - D["x"][:, None, :, :]
        T = tensors(r, g_bare(_norm(r), 2), 2)
        return P["ke"] * mp_potential(T, D["q"][:, None, :], D["mu"][:, None, :, :],
                                      D["th"][:, None, :, :, :]).sum(-1)

    def direction(D, Ad, VD, VintA, VatA):
        c = D["x"][:, 0]
        lp = D["lp"]
        a1 = Ad["x"][:, 0]
        a2 = Ad["x"][:, 1:3]
        r1 = _norm(a1 - c)
        m = _mask(r1, rc)
        rho1 = r1 / (2.0 * math.sqrt(rvo * rvo))
        rho2 = _norm(a2 - c[:, None]) / (2.0 * math.sqrt(rvo * rvh))
        u = lp - c[:, None]
        cos_a = _cos(u, (a1 - c)[:, None, :])
        cos_b = _cos(u[:, :, None, :], (a2 - c[:, None])[:, None, :, :])
        Vl = VD[:, :, None]
        Vs = VatA - donor_potential(D, Ad["x"][:, :3])       # V*(a) for O, H1, H2 of the acceptor
        e1 = (torch.exp(-eta * rho1)[:, None, None] * (VintA[:, 0][:, None, None] + Vs[:, 0][:, None, None] - Vl)
              * (cs * t + cp * mm * cos_a[:, :, None]))
        e2 = (torch.exp(-eta * rho2)[:, None, :] * (VintA[:, 1:3][:, None, :] + Vs[:, None, 1:3] - Vl)
              * (cs * t + cp * mm * cos_b))
        dE = P["ct_ae"] + Vl - (P["ct_ah"] + VatA[:, 0][:, None, None])
        e = -n * (e1 - e2) ** 2 / dE
        return (e.sum((1, 2)) * m).sum(), dE

    A, B = _take(S, i), _take(S, j, sh)
    ia, ja = torch.as_tensor(i), torch.as_tensor(j)
    e_ab, d1 = direction(A, B, V[ia], Vint[ja], Vat[ja])
    e_ba, d2 = direction(B, A, V[ja], Vint[ia], Vat[ia])
    min_de = min(float(d1.detach().min()) if d1.numel() else 1.0,
                 float(d2.detach().min()) if d2.numel() else 1.0)
    return e_ab + e_ba, min_de


# ---------------------------------------------------------------------------
# Exchange-repulsion (Technical Appendix; S^2/R and S^2/R^2 overlap terms)
# ---------------------------------------------------------------------------


def _overlap(csx, cpx, px, csy, cpy, py, vxy, f, pp):
    """Atom-pair overlap O_xy = Cs_x Cs_y + Cs_y Cp_x f cos(p_x, x->y)
    + Cs_x Cp_y f cos(p_y, y->x) + pp Cp_x Cp_y cos(p_x, x->y) cos(p_y, y->x),
    where each p direction is measured at its own atom; pp = 2 for bond-bond
    and f for bond-lone pair."""
    cx = _cos(px, vxy)
    cy = _cos(py, -vxy)
    return csx * csy + csy * cpx * f * cx + csx * cpy * f * cy + pp * cpx * cpy * cx * cy


def rep_pairs(S, i, j, sh, P, rc):
    A, B = _take(S, i), _take(S, j, sh)
    f, a1, a2 = P["rep_f"], P["rep_alpha"], P["rep_alpha2"]
    C1, C2 = P["rep_c1"], P["rep_c2"]
    occ, n = P["occ_bond"], P["n_lp"]
    # per-atom data of a bond (heavy O = 0, H = 1)
    cs = [P["cs_o"], P["cs_h"]]
    cp = [P["cp_o"], P["cp_h"]]
    gg = [P["g_o"], P["g_h"]]
    nval = [P["nval_o"], P["nval_h"]]
    rv = [P["rvdw_rep_o"], P["rvdw_rep_h"]]
    rvl = P["rvdw_rep_lp"]

    def bond_atoms(Mo, k):
        """Atoms of bond O-H_k: positions, p directions, charge factors."""
        O, H = Mo["x"][:, 0], Mo["x"][:, k]
        cf = [1.0 - Mo["q"][:, 0] / nval[0], 1.0 - Mo["q"][:, k] / nval[1]]
        return [O, H], [H - O, O - H], cf

    def lp_pseudo(Mo, l):
        c = Mo["x"][:, 0]
        return c, Mo["lp"][:, l] - c, Mo["lp"][:, l]

    cf_lp = 1.0 - n / nval[0]
    E = 0.0
    # bond-bond
    for kb1 in (1, 2):
        for kb2 in (1, 2):
            xa, pa, cfa = bond_atoms(A, kb1)
            xb, pb, cfb = bond_atoms(B, kb2)
            O1 = O2 = 0.0
            for u in range(2):
                for v in range(2):
                    vxy = xb[v] - xa[u]
                    rho = _norm(vxy) / (4.0 * math.sqrt(rv[u] * rv[v]))
                    Mxy = torch.sqrt(gg[u] * gg[v] * cfa[u] * cfb[v])
                    o = _overlap(cs[u], cp[u], pa[u], cs[v], cp[v], pb[v], vxy, f, 2.0)
                    O1 = O1 + o * Mxy * torch.exp(-a1 * rho)
                    O2 = O2 + o * Mxy * torch.exp(-a2 * rho)
            rm = _norm(0.5 * (xa[0] + xa[1]) - 0.5 * (xb[0] + xb[1]))
            E = E + (occ * occ * (C1 * O1 ** 2 / rm + C2 * O2 ** 2 / rm ** 2) * _mask(rm, rc)).sum()
    # bond-lp, both directions
    for (X, Y) in ((A, B), (B, A)):
        for kb in (1, 2):
            for l in range(2):
                xa, pa, cfa = bond_atoms(X, kb)
                c, pl, lpos = lp_pseudo(Y, l)
                O1 = O2 = 0.0
                for u in range(2):
                    vxy = c - xa[u]
                    rho = _norm(vxy) / (4.0 * math.sqrt(rv[u] * rvl))
                    Mxy = torch.sqrt(gg[u] * P["g_o"] * cfa[u] * cf_lp)
                    o = _overlap(cs[u], cp[u], pa[u], P["cs_lp"], P["cp_lp"], pl, vxy, f, f)
                    O1 = O1 + o * Mxy * torch.exp(-a1 * rho)
                    O2 = O2 + o * Mxy * torch.exp(-a2 * rho)
                r = _norm(0.5 * (xa[0] + xa[1]) - lpos)
                E = E + (occ * n * (C1 * O1 ** 2 / r + C2 * O2 ** 2 / r ** 2) * _mask(r, rc)).sum()
    # lp-lp: angles use the other lone pair's position (cos(AI, AJ), cos(BJ, BI))
    for l1 in range(2):
        for l2 in range(2):
            ca, pi_, I = lp_pseudo(A, l1)
            cb, pj, J = lp_pseudo(B, l2)
            ci = _cos(pi_, J - ca)
            cj = _cos(pj, I - cb)
            o = (P["cs_lp"] ** 2 + P["cs_lp"] * P["cp_lp"] * f * cj + P["cs_lp"] * P["cp_lp"] * f * ci
                 + 2.0 * P["cp_lp"] ** 2 * ci * cj)
            rho = _norm(cb - ca) / (4.0 * rvl)
            Mij = math.sqrt(P["g_o"] * P["g_o"] * cf_lp * cf_lp)
            O1 = o * Mij * torch.exp(-a1 * rho)
            O2 = o * Mij * torch.exp(-a2 * rho)
            r = _norm(I - J)
            E = E + (n * n * (C1 * O1 ** 2 / r + C2 * O2 ** 2 / r ** 2) * _mask(r, rc)).sum()
    return E


# ---------------------------------------------------------------------------
# Dispersion and exchange-dispersion (Technical Appendix)
# ---------------------------------------------------------------------------


def disp_pairs(S, i, j, sh, P, rc):
    A, B = _take(S, i), _take(S, j, sh)
    n = P["n_lp"]
    rv = t64([P["rvdw_disp_o"], P["rvdw_disp_h"], P["rvdw_disp_h"], P["rvdw_disp_lp"], P["rvdw_disp_lp"]])
    beta = t64([P["beta_o"], P["beta_h"], P["beta_h"], P["beta_o"], P["beta_o"]])
    islp = torch.tensor([False, False, False, True, True])

    def pts(Mo):
        return torch.cat([Mo["x"][:, :3], Mo["lp"]], 1)           # (C,5,3)

    def cfac(Mo):
        qo = Mo["q"][:, 0]
        c = [1.0 - qo / P["nval_o"], 1.0 - Mo["q"][:, 1] / P["nval_h"], 1.0 - Mo["q"][:, 2] / P["nval_h"],
             1.0 - qo / P["nval_o"], 1.0 - qo / P["nval_o"]]
        return torch.stack(c, -1)                                   # (C,5)

    r = _norm(pts(A)[:, :, None] - pts(B)[:, None])
    rvi, rvj = rv[:, None], rv[None, :]
    mred = r / (2.0 * torch.sqrt(rvi * rvj))
    d = (rvi + rvj) * P["disp_alpha"] / r - 1.0
    f = (P["c6"] * torch.exp(-P["gamma6"] * d) / mred ** 6 + P["c8"] * torch.exp(-P["gamma8"] * d) / mred ** 8
         + P["c10"] * torch.exp(-P["gamma10"] * d) / mred ** 10)
    li, lj = islp[:, None], islp[None, :]
    at_at = (~li) & (~lj)
    lp_lp = li & lj
    pref = torch.where(at_at, -beta[:, None] * beta[None, :],
                       torch.where(lp_lp, torch.full((5, 5), -n * n / 4.0, dtype=DT),
                                   torch.full((5, 5), -P["disp_delta"] / 2.0, dtype=DT)))
    m = _mask(r, rc)
    e_disp = (pref * f * m).sum()
    K = beta[:, None] * beta[None, :] * cfac(A)[:, :, None] * cfac(B)[:, None, :]
    xd = torch.where(at_at, P["xd_c1"] * torch.exp(-P["xd_a1"] * mred),
                     torch.where(lp_lp, (n * n / 4.0) * P["xd_c2"] * torch.exp(-P["xd_a2"] * mred),
                                 (n / 2.0) * P["xd_c3"] * torch.exp(-P["xd_a3"] * mred)))
    e_xd = (K * xd * m).sum()
    return e_disp, e_xd


def disp_tail(n_mol, volume, rc, P):
    """Dispersion beyond the cutoff for a homogeneous fluid (pair distribution
    1 past rc): 2 pi N (N-1) / V sum over the point types u, v of one molecule
    (O, H1, H2, LP1, LP2) of the integral from rc to infinity of r^2 e_uv(r),
    with e_uv the damped C6/C8/C10 pair function of the Technical Appendix
    (prefactors as in disp_pairs).  Each C_n term integrates in closed form:
    with d = c/r - 1 (c = (rv_u + rv_v) alpha_disp) and m = r/k
    (k = 2 sqrt(rv_u rv_v)),
      int_rc^inf r^2 C_n e^{-g d} (k/r)^n dr
        = C_n e^{g} k^n (g c)^{3-n} Gamma(n-3) P(n-3, g c / rc),
    P the regularized lower incomplete gamma function (t = 1/r).  The
    exchange-dispersion, exponential in r, is negligible past the cutoff."""
    from scipy.special import gamma as Gf, gammainc
    n = P["n_lp"]
    rv = [P["rvdw_disp_o"], P["rvdw_disp_h"], P["rvdw_disp_h"], P["rvdw_disp_lp"], P["rvdw_disp_lp"]]
    beta = [P["beta_o"], P["beta_h"], P["beta_h"]]
    total = 0.0
    for u in range(5):
        for v in range(5):
            if u < 3 and v < 3:
                pref = -beta[u] * beta[v]
            elif u >= 3 and v >= 3:
                pref = -n * n / 4.0
            else:
                pref = -P["disp_delta"] / 2.0
            c = (rv[u] + rv[v]) * P["disp_alpha"]
            k = 2.0 * math.sqrt(rv[u] * rv[v])
            for order, C, g in ((6, P["c6"], P["gamma6"]), (8, P["c8"], P["gamma8"]), (10, P["c10"], P["gamma10"])):
                s = order - 3
                total += pref * C * math.exp(g) * k ** order * (g * c) ** (-s) * Gf(s) * gammainc(s, g * c / rc)
    return 2.0 * math.pi * n_mol * (n_mol - 1) / volume * total


# ---------------------------------------------------------------------------
# Polarization functionals (Technical Appendix: E_pol = 1/2 mu^T T mu - mu^T E)
# Induced dipoles live on O, H1, H2 (mu: (M, 3, 3)).
# ---------------------------------------------------------------------------


def _thole_A(P, a_pol_idx_tab, b_tab):
    return (a_pol_idx_tab * b_tab) ** (1.0 / 6.0)


def pol_linear_pairs(S, mu, i, j, sh, P, rc, alpha):
    """-mu^T E_perm, real-space / gas-phase part: every induced dipole of one
    molecule in the Thole-damped potential of the other molecule's multipoles."""
    tb = site_tables(P)
    A, B = _take(S, i), _take(S, j, sh)
    ia, ja = torch.as_tensor(i), torch.as_tensor(j)
    Ath = (tb["alpha_pol"][:, None] * tb["alpha_damp"][None, :]) ** (1.0 / 6.0)    # (3,5)

    def one(X, muX, Y):
        r = X["x"][:, :3, None, :] - Y["x"][:, None, :, :]                          # (C,3,5,3)
        rn = _norm(r)
        T = tensors(r, g_thole(rn, Ath, P["thole"], alpha, 3), 3)
        U = dipole_mp_energy(T, muX[:, :, None, :], Y["q"][:, None, :], Y["mu"][:, None, :, :],
                             Y["th"][:, None, :, :, :])
        return (U * _mask(rn, rc)).sum()

    return P["ke"] * (one(A, mu[ia], B) + one(B, mu[ja], A))


def pol_quadratic_pairs(S, mu, i, j, sh, P, rc, alpha):
    """Off-diagonal part of 1/2 mu^T T mu: Thole-damped dipole-dipole energy of
    induced dipoles on different molecules."""
    tb = site_tables(P)
    A, B = _take(S, i), _take(S, j, sh)
    ia, ja = torch.as_tensor(i), torch.as_tensor(j)
    Ath = (tb["alpha_pol"][:, None] * tb["alpha_pol"][None, :]) ** (1.0 / 6.0)     # (3,3)
    r = A["x"][:, :3, None, :] - B["x"][:, None, :3, :]
    rn = _norm(r)
    T = tensors(r, g_thole(rn, Ath, P["thole"], alpha, 2), 2)
    U = dipole_dipole_energy(T, mu[ia][:, :, None, :], mu[ja][:, None, :, :])
    return P["ke"] * (U * _mask(rn, rc)).sum()


def pol_diag(mu, P):
    a = site_tables(P)["alpha_pol"]
    return P["ke"] * ((mu * mu).sum(-1) / (2.0 * a)).sum()


def pol_periodic_quadratic(S, mu, P, alpha, G, box, K, order):
    """Reciprocal + self - intramolecular erf part of the induced-dipole
    self-interaction."""
    x = S["x"][:, :3].reshape(-1, 3)
    m = mu.reshape(-1, 3)
    Q = ew.spread(x, torch.zeros(m.shape[0], dtype=DT), m, None, box, K, order)
    e = ew.grid_energy(Q, G)
    e = e - P["ke"] * alpha / math.sqrt(math.pi) * (2 * alpha ** 2 / 3.0) * (m * m).sum()
    ia, ib = np.triu_indices(3, 1)
    r = S["x"][:, ia] - S["x"][:, ib]
    T = tensors(r, g_erf(_norm(r), alpha, 2), 2)
    e = e - P["ke"] * dipole_dipole_energy(T, mu[:, ia], mu[:, ib]).sum()
    return e


def pol_periodic_linear(S, mu, P, alpha, Psi_perm, box, K, order):
    """Reciprocal cross energy of induced dipoles with the permanent grid,
    self cross term, minus the erf part of intramolecular (dipole, site) pairs."""
    x = S["x"][:, :3].reshape(-1, 3)
    m = mu.reshape(-1, 3)
    Q = ew.spread(x, torch.zeros(m.shape[0], dtype=DT), m, None, box, K, order)
    e = (Q * Psi_perm).sum()
    e = e - P["ke"] * alpha / math.sqrt(math.pi) * (4 * alpha ** 2 / 3.0) * (m * S["mu"][:, :3].reshape(-1, 3)).sum()
    pa, ps = [], []
    for a in range(3):
        for s in range(5):
            if s != a:
                pa.append(a)
                ps.append(s)
    r = S["x"][:, pa] - S["x"][:, ps]
    T = tensors(r, g_erf(_norm(r), alpha, 3), 3)
    e = e - P["ke"] * dipole_mp_energy(T, mu[:, pa], S["q"][:, ps], S["mu"][:, ps], S["th"][:, ps]).sum()
    return e
