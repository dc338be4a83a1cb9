"""Oracle driver: one SIBFA energy + force evaluation in FP64.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg; never by the product path.

Order of the steps (the method's call order): sites and frames -> real-space
pair terms (electrostatics + penetration, exchange-repulsion, dispersion) ->
reciprocal / self / exclusion electrostatics -> potentials on the lone pairs
-> reduced charge transfer -> polarization solve (Jacobi-preconditioned
conjugate gradient on T mu = E) -> polarization energy.  Forces are the exact
gradient -dE/dx: autograd of each term, with the induced dipoles held at the
solution (E_pol is stationary in mu there) and the charge-transfer
dependence on the lone-pair potentials applied by the chain rule.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from synth import PARAMS

from . import ewald as ew
from . import terms as tm
from .core import DT, build_sites, t64

TERMS = ("elec", "pen", "rep", "disp", "xdisp", "pol", "ct")
SITE_MARGIN = 2.6       # A, molecule-list margin over rc (site extents < 1.3 A)


class _Setup:
    def __init__(self, system, opts, P):
        self.P = P
        self.mp = torch.as_tensor(system.mp_local, dtype=DT)
        self.periodic = system.box is not None
        # edge lengths of an orthorhombic box, or a 3x3 cell (columns = cell vectors)
        self.box = t64(system.box) if self.periodic else None
        if self.periodic:
            self.rc = float(opts["rc"])
            self.alpha = float(opts["ewald"])
            g = opts["grid"]
            self.K = (g, g, g) if isinstance(g, int) else tuple(g)
            self.order = int(opts.get("order", 5))
            self.G = ew.influence(self.box, self.K, self.order, self.alpha, P["ke"])
            cut = self.rc + SITE_MARGIN
        else:
            self.rc = None
            self.alpha = None
            cut = None
        O = np.asarray(system.pos[:, 0], dtype=np.float64)
        i, j, sh = tm.mol_pairs(O, system.box if self.periodic else None, cut)
        self.i, self.j, self.sh = i, j, t64(sh)

    def chunks(self, size):
        n = self.i.size
        for a in range(0, n, size):
            b = min(n, a + size)
            sh = self.sh[a:b]
            yield self.i[a:b], self.j[a:b], (sh if self.strain is None else sh @ self.strain.T)

    strain = None   # (I + eps) in virial mode: image shifts are lattice vectors and deform with the cell


def evaluate(system, opts=None, forces=True, tol_D=1e-10, max_iter=500, chunk=2048,
             P=None, mu_guess=None, pcg_log=None, per_term=False, keep_operators=False, virial=False):
    """Energies (kcal/mol) per term, forces (kcal/mol/A) on O, H1, H2, induced
    dipoles (e.A) on O, H1, H2, PCG iteration count and final residual (D).

    opts (periodic systems): rc, grid, order, ewald.  Gas phase: opts unused.

    virial=True: instead of forces, the virial W_ab = -dE/d eps_ab (kcal/mol)
    for the affine strain x -> (I + eps) x of every atom and of the periodic
    cell (the image shifts and the reciprocal lattice deform with it), by the
    same chain rule as the forces, with eps as the variable.  For a gas-phase
    system it equals sum_atoms F_a x_b."""
    P = PARAMS if P is None else P
    opts = opts or {}
    st = _Setup(system, opts, P)
    if virial:
        forces = True
        eps = torch.zeros((3, 3), dtype=DT, requires_grad=True)
        Fm = torch.eye(3, dtype=DT) + eps
        x = t64(system.pos) @ Fm.T
        wrt = eps
        st.strain = Fm
        if st.periodic:
            cell0 = st.box if ew.is_cell(st.box) else torch.diag(st.box)
            st.box = Fm @ cell0                       # cell matrix, columns = cell vectors
            st.G = ew.influence(st.box, st.K, st.order, st.alpha, P["ke"])
    else:
        x = torch.tensor(system.pos, dtype=DT, requires_grad=forces)
        wrt = x
    M = x.shape[0]
    F = torch.zeros_like(wrt) if forces else None
    FT = {k: torch.zeros_like(wrt) for k in TERMS} if (forces and per_term) else None
    E = {k: 0.0 for k in TERMS}

    def acc(e, name):
        E[name] += float(e.detach()) if torch.is_tensor(e) else float(e)

    def add_grad(e, name=None, retain=False):
        if forces and e.requires_grad:
            g, = torch.autograd.grad(e, [wrt], allow_unused=True, retain_graph=retain or virial)
            if g is not None:
                F.sub_(g)
                if FT is not None and name is not None:
                    FT[name].sub_(g)

    # ---- real-space pair terms --------------------------------------------
    for i, j, sh in st.chunks(chunk):
        S = build_sites(x, st.mp, P)
        e_el, e_pen = tm.elec_pen_pairs(S, i, j, sh, P, st.rc, st.alpha)
        e_rep = tm.rep_pairs(S, i, j, sh, P, st.rc)
        e_d, e_xd = tm.disp_pairs(S, i, j, sh, P, st.rc)
        acc(e_el, "elec"); acc(e_pen, "pen"); acc(e_rep, "rep"); acc(e_d, "disp"); acc(e_xd, "xdisp")
        if FT is None:
            add_grad(e_el + e_pen + e_rep + e_d + e_xd)
        else:
            for e, nm in ((e_el, "elec"), (e_pen, "pen"), (e_rep, "rep"), (e_d, "disp"), (e_xd, "xdisp")):
                add_grad(e, nm, retain=True)

    # ---- dispersion beyond the cutoff (homogeneous-fluid tail), if asked ------
    if st.periodic and opts.get("disp_tail"):
        cell = st.box if ew.is_cell(st.box) else torch.diag(st.box)
        e_tail = tm.disp_tail(M, 1.0, st.rc, P) / torch.linalg.det(cell)
        acc(e_tail, "disp")
        add_grad(e_tail, "disp")

    # ---- reciprocal, self and intramolecular corrections --------------------
    Psi_perm = None
    if st.periodic:
        S = build_sites(x, st.mp, P)
        e_corr, Q = tm.elec_periodic_corrections(S, P, st.alpha, st.G, st.box, st.K, st.order)
        acc(e_corr, "elec")
        add_grad(e_corr, "elec")
        Psi_perm = ew.convolve(Q, st.G).detach()

    # ---- potential on the lone pairs, charge transfer -----------------------
    def lp_potential(xx, S=None):
        S = build_sites(xx, st.mp, P) if S is None else S
        V = torch.zeros((M, 2), dtype=DT)
        for i, j, sh in st.chunks(chunk):
            V = V + tm.lp_potential_pairs(S, i, j, sh, P, st.rc, st.alpha)
        if st.periodic:
            S2 = build_sites(xx, st.mp, P)
            Qp = ew.spread(S2["x"].reshape(-1, 3), S2["q"].reshape(-1), S2["mu"].reshape(-1, 3),
                           S2["th"].reshape(-1, 3, 3), st.box, st.K, st.order)
            V = V + tm.lp_potential_periodic(S2, P, st.alpha, ew.convolve(Qp, st.G), st.box, st.K, st.order)
        return V

    # the original many-body charge transfer (opts["ct_original"]) also
    # needs the potential at the acceptor atoms O, H1, H2
    ct_orig = bool(opts.get("ct_original"))

    def atom_potential(xx):
        S = build_sites(xx, st.mp, P)
        V = torch.zeros((M, 3), dtype=DT)
        for i, j, sh in st.chunks(chunk):
            V = V + tm.atom_potential_pairs(S, i, j, sh, P, st.rc, st.alpha)
        if st.periodic:
            Qp = ew.spread(S["x"].reshape(-1, 3), S["q"].reshape(-1), S["mu"].reshape(-1, 3),
                           S["th"].reshape(-1, 3, 3), st.box, st.K, st.order)
            V = V + tm.atom_potential_periodic(S, P, st.alpha, ew.convolve(Qp, st.G), st.box, st.K, st.order)
        return V

    with torch.no_grad():
        V_lp = lp_potential(x.detach())
        V_at = atom_potential(x.detach()) if ct_orig else None
    Vleaf = V_lp.clone().requires_grad_(True)
    leaves = [Vleaf]
    if ct_orig:
        Valeaf = V_at.clone().requires_grad_(True)
        leaves.append(Valeaf)
    e_ct = 0.0
    min_de = math.inf
    lam = torch.zeros_like(V_lp)
    lam_a = torch.zeros_like(V_at) if ct_orig else None
    for i, j, sh in st.chunks(chunk):
        S = build_sites(x, st.mp, P)
        Vint = tm.v_int(S, P)
        if ct_orig:
            e, mde = tm.ct_pairs_original(S, Vleaf, Valeaf, Vint, i, j, sh, P, st.rc)
        else:
            e, mde = tm.ct_pairs(S, Vleaf, Vint, i, j, sh, P, st.rc)
        min_de = min(min_de, mde)
        e_ct += float(e.detach())
        if e.requires_grad:
            g = torch.autograd.grad(e, ([wrt] if forces else []) + leaves, allow_unused=True, retain_graph=virial)
            if forces:
                gx, g = g[0], g[1:]
                if gx is not None:
                    F.sub_(gx)
                    if FT is not None:
                        FT["ct"].sub_(gx)
            if g[0] is not None:
                lam += g[0]
            if ct_orig and g[1] is not None:
                lam_a += g[1]
    E["ct"] = e_ct
    if forces and float(lam.abs().sum()) > 0:
        # d/dx of sum lam . V_lp(x), one chunk of pairs at a time (the
        # gradient of the sum is the sum of the chunks' gradients)
        lamd = lam.detach()
        S = build_sites(x, st.mp, P)
        for i, j, sh in st.chunks(chunk):
            add_grad((lamd * tm.lp_potential_pairs(S, i, j, sh, P, st.rc, st.alpha)).sum(), "ct", retain=True)
        if st.periodic:
            Qp = ew.spread(S["x"].reshape(-1, 3), S["q"].reshape(-1), S["mu"].reshape(-1, 3),
                           S["th"].reshape(-1, 3, 3), st.box, st.K, st.order)
            add_grad((lamd * tm.lp_potential_periodic(S, P, st.alpha, ew.convolve(Qp, st.G), st.box, st.K,
                                                      st.order)).sum(), "ct", retain=True)
        del S
    if forces and ct_orig and float(lam_a.abs().sum()) > 0:
        # the same for sum lam_a . V(a)(x) over the acceptor atoms
        lamd = lam_a.detach()
        S = build_sites(x, st.mp, P)
        for i, j, sh in st.chunks(chunk):
            add_grad((lamd * tm.atom_potential_pairs(S, i, j, sh, P, st.rc, st.alpha)).sum(), "ct", retain=True)
        if st.periodic:
            Qp = ew.spread(S["x"].reshape(-1, 3), S["q"].reshape(-1), S["mu"].reshape(-1, 3),
                           S["th"].reshape(-1, 3, 3), st.box, st.K, st.order)
            add_grad((lamd * tm.atom_potential_periodic(S, P, st.alpha, ew.convolve(Qp, st.G), st.box, st.K,
                                                        st.order)).sum(), "ct", retain=True)
        del S

    # ---- polarization ---------------------------------------------------------
    a_pol = tm.site_tables(P)["alpha_pol"]

    # The polarization functional's linear (-mu.E_perm) and quadratic
    # (1/2 mu.T.mu) parts as a sequence of terms, one chunk of pairs each:
    # gradients are taken term by term, so only one chunk's graph is held.
    def linear_parts(xx, mu):
        S = build_sites(xx, st.mp, P)
        for i, j, sh in st.chunks(chunk):
            yield tm.pol_linear_pairs(S, mu, i, j, sh, P, st.rc, st.alpha)
        if st.periodic:
            yield tm.pol_periodic_linear(S, mu, P, st.alpha, Psi_perm_of(xx), st.box, st.K, st.order)

    def quadratic_parts(xx, mu):
        S = build_sites(xx, st.mp, P)
        yield tm.pol_diag(mu, P)
        for i, j, sh in st.chunks(chunk):
            yield tm.pol_quadratic_pairs(S, mu, i, j, sh, P, st.rc, st.alpha)
        if st.periodic:
            yield tm.pol_periodic_quadratic(S, mu, P, st.alpha, st.G, st.box, st.K, st.order)

    def grad_mu(parts, mu):
        g = torch.zeros_like(mu)
        for e in parts:
            if torch.is_tensor(e) and e.requires_grad:
                ge, = torch.autograd.grad(e, [mu], allow_unused=True, retain_graph=True)
                if ge is not None:
                    g = g + ge
        return g

    def Psi_perm_of(xx):
        if not xx.requires_grad:
            return Psi_perm
        S = build_sites(xx, st.mp, P)
        Qp = ew.spread(S["x"].reshape(-1, 3), S["q"].reshape(-1), S["mu"].reshape(-1, 3),
                       S["th"].reshape(-1, 3, 3), st.box, st.K, st.order)
        return ew.convolve(Qp, st.G)

    xd = x.detach()
    # E_perm = -d(-mu.E)/dmu ; T p = d(1/2 p.T.p)/dp   (both divided by ke below)
    mu0 = torch.zeros((M, 3, 3), dtype=DT, requires_grad=True)
    Efield = -grad_mu(linear_parts(xd, mu0), mu0) / P["ke"]

    def matvec(p):
        pp = p.detach().clone().requires_grad_(True)
        return grad_mu(quadratic_parts(xd, pp), pp) / P["ke"]

    debye = P["debye"]
    mu = (a_pol[None, :, None] * Efield) if mu_guess is None else torch.as_tensor(mu_guess, dtype=DT).clone()
    r = Efield - matvec(mu)
    z = a_pol[None, :, None] * r

    def resid_D(rv):
        return float(torch.sqrt(((a_pol[None, :, None] * rv) ** 2).sum(-1).mean())) * debye

    p = z.clone()
    rz = float((r * z).sum())
    it = 0
    res = resid_D(r)
    while res > tol_D and it < max_iter:
        Ap = matvec(p)
        step = rz / float((p * Ap).sum())
        mu = mu + step * p
        r = r - step * Ap
        z = a_pol[None, :, None] * r
        rz_new = float((r * z).sum())
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        res = resid_D(r)
        if pcg_log is not None:
            pcg_log.append(res)
    E["pol"] = -0.5 * P["ke"] * float((mu * Efield).sum())
    if forces:
        mud = mu.detach()
        for e in quadratic_parts(x, mud):
            add_grad(e, "pol", retain=True)
        for e in linear_parts(x, mud):
            add_grad(e, "pol", retain=True)

    E["total"] = sum(E[k] for k in TERMS)
    return {
        "terms": E,
        "forces": F.detach().numpy() if (forces and not virial) else None,
        "virial": F.detach().numpy() if virial else None,
        "forces_per_term": {k: v.numpy() for k, v in FT.items()} if FT is not None else None,
        "mu": mu.detach().numpy(),
        "efield": Efield.detach().numpy(),
        "v_lp": V_lp.detach().numpy(),
        "v_atoms": V_at.detach().numpy() if ct_orig else None,
        "iters": it,
        "resid_D": res,
        "min_ct_denominator": min_de,
        "pol_ops": ({"matvec": matvec, "alpha": a_pol,
                     "functional": lambda m: (sum(float(e) for e in quadratic_parts(xd, m)) +
                                              sum(float(e) for e in linear_parts(xd, m))) / P["ke"]}
                    if keep_operators else None),
    }


def energy_only(system, opts=None, **kw):
    """Total energy with a tightly converged polarization (for finite differences)."""
    out = evaluate(system, opts, forces=False, **kw)
    return out["terms"]["total"], out


def timed_evaluate(system, opts, **kw):
    t0 = time.perf_counter()
    out = evaluate(system, opts, **kw)
    return out, time.perf_counter() - t0
