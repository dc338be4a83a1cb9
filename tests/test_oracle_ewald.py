"""Oracle pins for the periodic electrostatics: total Ewald energy is
independent of alpha, the SPME reciprocal energy converges to the exact
k-space sum as the grid grows, and the Ewald result equals a direct
spherical lattice sum minus the tinfoil surface term."""
import math

import numpy as np
import torch

import oracle
import synth
from oracle import core, ewald, terms
from synth import PARAMS

DT = torch.float64


def _system():
    s = synth.make_box(2, 16.0, seed=21, jitter=1.5)     # 8 waters in a 16 A box
    return s


def _sites(s):
    return core.build_sites(torch.tensor(s.pos, dtype=DT), torch.tensor(s.mp_local, dtype=DT), PARAMS)


def _ewald_total(s, alpha, rc, recip):
    S = _sites(s)
    i, j, sh = terms.mol_pairs(s.pos[:, 0], s.box, rc + 2.6)
    e_real, _ = terms.elec_pen_pairs(S, i, j, torch.tensor(sh, dtype=DT), PARAMS, rc, alpha)
    x = S["x"].reshape(-1, 3)
    q, mu, th = S["q"].reshape(-1), S["mu"].reshape(-1, 3), S["th"].reshape(-1, 3, 3)
    if recip == "exact":
        mmax = int(math.ceil(6.2 * alpha / math.pi * s.box[0]))
        e_rec = ewald.exact_recip_energy(x, q, mu, th, torch.tensor(s.box), alpha, PARAMS["ke"], mmax)
    else:
        K = (recip, recip, recip)
        G = ewald.influence(torch.tensor(s.box), K, 5, alpha, PARAMS["ke"])
        e_rec = ewald.grid_energy(ewald.spread(x, q, mu, th, torch.tensor(s.box), K, 5), G)
    e_self = ewald.self_energy(q, mu, th, alpha, PARAMS["ke"])
    ia, ib = np.triu_indices(5, 1)
    r = S["x"][:, ia] - S["x"][:, ib]
    T = core.tensors(r, core.g_erf(torch.linalg.vector_norm(r, dim=-1), alpha, 4), 4)
    e_excl = PARAMS["ke"] * core.mp_pair_energy(T, S["q"][:, ia], S["mu"][:, ia], S["th"][:, ia],
                                                S["q"][:, ib], S["mu"][:, ib], S["th"][:, ib]).sum()
    return float(e_real), float(e_rec), float(e_self), float(e_excl), float(e_real + e_rec + e_self - e_excl)


def test_ewald_alpha_independence():
    s = _system()
    ra = _ewald_total(s, 1.0, 5.4, "exact")
    rb = _ewald_total(s, 1.1, 5.4, "exact")
    scale = sum(abs(v) for v in ra[:4])          # the parts are ~1000x the total
    assert abs(ra[-1] - rb[-1]) < 1e-10 * scale, (ra, rb)


def test_spme_converges_to_exact():
    s = _system()
    alpha = 0.45
    exact = _ewald_total(s, alpha, 5.4, "exact")[1]
    # charge, dipole and quadrupole errors change sign as K grows, so the
    # test asks for a large overall reduction rather than monotonic steps
    # (quadrupole cross terms converge like h^3: second derivatives of the splines)
    errs = [abs(_ewald_total(s, alpha, 5.4, K)[1] - exact) for K in (16, 32, 96)]
    assert errs[2] < 1e-2 * errs[0]
    assert errs[2] < 1e-5 * abs(exact)


def test_ewald_equals_spherical_lattice_sum():
    """E_ewald (tinfoil) = spherical lattice sum - 2 pi |D|^2 / (3 V)."""
    s = _system()
    ewald_total = _ewald_total(s, 0.9, 5.4, "exact")[-1]
    S = _sites(s)
    L = s.box[0]
    D = (S["q"][..., None] * S["x"]).sum((0, 1)) + S["mu"].sum((0, 1))
    surf = 2 * math.pi * float((D * D).sum()) / (3 * L ** 3) * PARAMS["ke"]
    xs, q, mu, th = S["x"].reshape(-1, 3), S["q"].reshape(-1), S["mu"].reshape(-1, 3), S["th"].reshape(-1, 3, 3)
    mol = torch.arange(s.n_mol).repeat_interleave(5)
    same = mol[:, None] == mol[None, :]
    ests = []
    for nmax in (6, 8):
        imgs = ewald.lattice_images(nmax) * L
        e = 0.0
        for k in range(imgs.shape[0]):
            r = xs[:, None, :] - xs[None, :, :] - imgs[k]
            keep = ~same if float(imgs[k].abs().sum()) == 0 else torch.ones_like(same)
            rn = torch.linalg.vector_norm(r, dim=-1)
            rn = torch.where(keep, rn, torch.ones_like(rn))
            T = core.tensors(r, core.g_bare(rn, 4), 4)
            U = core.mp_pair_energy(T, q[:, None], mu[:, None], th[:, None], q[None], mu[None], th[None])
            e += 0.5 * float((U * keep).sum())
        ests.append(e * PARAMS["ke"] - surf)
    # the shell sum converges toward the Ewald value
    assert abs(ests[1] - ewald_total) < abs(ests[0] - ewald_total) + 1e-9
    # the total is a near-cancellation of parts ~1000x larger: compare against them
    parts = _ewald_total(s, 0.9, 5.4, "exact")
    scale = abs(parts[1]) + abs(parts[2]) + abs(parts[3])
    assert abs(ests[1] - ewald_total) < 1e-7 * scale, (ests, ewald_total, scale)
