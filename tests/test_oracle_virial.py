"""Oracle pins for the virial W_ab = -dE/d eps_ab (affine strain x -> (I + eps) x
of every atom and of the periodic cell).

The oracle takes it by the chain rule with eps as the variable; these tests
hold it to things fixed independently of that code path: in the gas phase
it is sum_atoms F_a x_b with the (separately pinned) forces; in a periodic
box every component equals a central finite difference of the total energy
under the matching strain (diagonal strains rescale an orthorhombic box,
off-diagonal ones shear it into a triclinic cell); the triclinic SPME
reproduces the orthorhombic one for a diagonal cell and the exact Ewald
k-space sum for a sheared cell; and W is symmetric (rotational invariance).
The seeded 64-water box with rc = 5.75 A has no site pair within reach of
the cutoff for the strain step used, so the energy is smooth there."""
import copy
import math

import numpy as np
import torch

import synth
from oracle import evaluate, ewald

DT = torch.float64
H = 1e-5


def _box():
    s = synth.make_box(4, 12.42, seed=7)
    opts = {"rc": 5.75, "grid": 16, "order": 5, "ewald": 0.45}
    return s, opts


def _energy_strained(s, opts, a, b, h):
    s2 = copy.deepcopy(s)
    F = np.eye(3)
    F[a, b] += h
    s2.pos = s.pos @ F.T
    s2.box = F @ np.diag(s.box)
    return evaluate(s2, opts, forces=False, tol_D=1e-12)["terms"]["total"]


def test_gas_phase_virial_is_sum_of_force_times_position():
    s = synth.make_cluster(6, seed=3)
    o = evaluate(s, None, tol_D=1e-12)
    W = evaluate(s, None, tol_D=1e-12, virial=True)["virial"]
    ref = np.einsum("mka,mkb->ab", o["forces"], s.pos)
    assert np.abs(W - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(W - W.T).max() < 1e-10 * np.abs(W).max()


def test_periodic_virial_matches_strain_finite_differences():
    s, opts = _box()
    W = evaluate(s, opts, tol_D=1e-12, virial=True)["virial"]
    scale = np.abs(W).max()
    assert np.abs(W - W.T).max() < 1e-9 * scale
    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (1, 0), (1, 2), (0, 2)):
        fd = -(_energy_strained(s, opts, a, b, H) - _energy_strained(s, opts, a, b, -H)) / (2 * H)
        assert abs(fd - W[a, b]) < 1e-7 * scale, (a, b, fd, W[a, b])


def test_cell_input_equals_orthorhombic_box():
    s, opts = _box()
    s2 = copy.deepcopy(s)
    s2.box = np.diag(s.box)
    e0 = evaluate(s, opts, forces=False, tol_D=1e-12)["terms"]
    e1 = evaluate(s2, opts, forces=False, tol_D=1e-12)["terms"]
    for k in e0:
        assert abs(e0[k] - e1[k]) <= 1e-11 * max(1.0, abs(e0[k])), k


def test_triclinic_spme_matches_exact_ewald():
    g = torch.Generator().manual_seed(5)
    n = 9
    cell = torch.tensor([[9.0, 0.8, -0.5], [0.3, 10.0, 0.6], [-0.4, 0.2, 11.0]], dtype=DT)
    x = torch.rand(n, 3, generator=g, dtype=DT) @ cell.T
    q = torch.randn(n, generator=g, dtype=DT)
    q = q - q.mean()
    mu = 0.3 * torch.randn(n, 3, generator=g, dtype=DT)
    th = torch.randn(n, 3, 3, generator=g, dtype=DT)
    th = th + th.transpose(-1, -2)
    th = th - torch.eye(3, dtype=DT) * (th.diagonal(dim1=-1, dim2=-2).sum(-1) / 3.0)[:, None, None]
    alpha, ke = 0.35, 332.063713
    mmax = int(math.ceil(6.2 * alpha / math.pi * 11.5))
    e_exact = float(ewald.exact_recip_energy(x, q, mu, th, cell, alpha, ke, mmax))

    def err(K):
        e = ewald.grid_energy(ewald.spread(x, q, mu, th, cell, K, 5), ewald.influence(cell, K, 5, alpha, ke))
        return abs(float(e) - e_exact) / abs(e_exact)

    coarse, fine = err((24, 26, 28)), err((64, 70, 76))
    assert fine < 1e-6 and fine < coarse / 10
    # odd grid sizes (no Nyquist planes) converge to the same sum
    assert err((63, 69, 75)) < 1e-6


def test_noncubic_box_odd_grid_virial_matches_strain_finite_differences():
    """Orthorhombic 12.42 x 15.52 x 18.63 A box (120 waters) with SPME grids
    of 16 x 19 x 23 points (odd sizes: no Nyquist plane on two axes): every
    strain direction against central differences.  With seed 12 no masked
    pair crosses the cutoff under the strain step (differences at h and h/2
    agree to 2e-9 of max |W|); other seeds may have one."""
    s = synth.make_ortho_box((4, 5, 6), (12.42, 15.52, 18.63), seed=12)
    opts = {"rc": 4.25, "grid": (16, 19, 23), "order": 5, "ewald": 0.7}
    W = evaluate(s, opts, tol_D=1e-12, virial=True)["virial"]
    scale = np.abs(W).max()
    assert np.abs(W - W.T).max() < 1e-9 * scale
    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (2, 0), (1, 2)):
        fd = -(_energy_strained(s, opts, a, b, H) - _energy_strained(s, opts, a, b, -H)) / (2 * H)
        assert abs(fd - W[a, b]) < 1e-7 * scale, (a, b, fd, W[a, b])
