"""Oracle pins for the building blocks: radial-kernel recurrences, Cartesian
interaction tensors as true derivatives, multipole energies against point-charge
clusters, Thole factors, B-spline identities."""
import math

import numpy as np
import pytest
import torch

from oracle import core, ewald

DT = torch.float64


def _deriv_check(gfun, nmax, r0=None):
    r = torch.linspace(0.6, 6.0, 23, dtype=DT) if r0 is None else r0
    r = r.clone().requires_grad_(True)
    g = gfun(r)
    for n in range(nmax):
        d, = torch.autograd.grad(g[n].sum(), [r], retain_graph=True)
        np.testing.assert_allclose((d / r).detach().numpy(), g[n + 1].detach().numpy(),
                                   rtol=1e-10, atol=1e-13)


def test_bare_recurrence():
    _deriv_check(lambda r: core.g_bare(r, 5), 5)


def test_erfc_recurrence():
    _deriv_check(lambda r: core.g_erfc(r, 0.4, 5), 5)
    _deriv_check(lambda r: core.g_erfc(r, 0.9, 5), 5)


def test_exp_recurrence():
    _deriv_check(lambda r: core.g_exp(r, 3.0, 5), 5)


def test_thole_factors_are_derivatives():
    # lambda_{2n+1} g_n(1/r) must be a consistent derivative chain
    A, a = 0.9, 0.28
    _deriv_check(lambda r: [None] + core.g_thole(r, torch.tensor(A, dtype=DT), a, None, 4)[1:], 0)
    r = torch.linspace(0.4, 5.0, 17, dtype=DT).requires_grad_(True)
    g = core.g_thole(r, torch.tensor(A, dtype=DT), a, None, 4)
    for n in range(1, 4):
        d, = torch.autograd.grad(g[n].sum(), [r], retain_graph=True)
        np.testing.assert_allclose((d / r).detach().numpy(), g[n + 1].detach().numpy(), rtol=1e-10)
    # far away the damping vanishes
    gf = core.g_thole(torch.tensor([30.0], dtype=DT), torch.tensor(A, dtype=DT), a, None, 4)
    gb = core.g_bare(torch.tensor([30.0], dtype=DT), 4)
    for n in range(1, 5):
        assert abs(float(gf[n] / gb[n]) - 1.0) < 1e-12


def test_tensors_are_derivatives():
    x = torch.tensor([[0.7, -1.1, 0.4], [2.0, 0.3, -1.5]], dtype=DT, requires_grad=True)
    for gfun in (lambda r: core.g_bare(r, 4), lambda r: core.g_erfc(r, 0.5, 4),
                 lambda r: core.g_exp(r, 2.0, 4)):
        r = torch.linalg.vector_norm(x, dim=-1)
        T = core.tensors(x, gfun(r), 4)
        for n in range(4):
            flat = T[n].reshape(2, -1)
            for c in range(flat.shape[1]):
                d, = torch.autograd.grad(flat[:, c].sum(), [x], retain_graph=True)
                np.testing.assert_allclose(d.detach().numpy(),
                                           T[n + 1].reshape(2, -1, 3)[:, c].detach().numpy(),
                                           rtol=1e-10, atol=1e-13)


def _cluster_moments(qs, ss):
    q = qs.sum()
    mu = (qs[:, None] * ss).sum(0)
    th = 0.5 * sum(qk * (3 * np.outer(sk, sk) - sk @ sk * np.eye(3)) for qk, sk in zip(qs, ss))
    return q, mu, th


def _point_energy(qa, sa, ca, qb, sb, cb):
    e = 0.0
    for q1, s1 in zip(qa, sa):
        for q2, s2 in zip(qb, sb):
            e += q1 * q2 / np.linalg.norm(ca + s1 - cb - s2)
    return e


@pytest.mark.parametrize("kind", ["q", "mu", "th"])
@pytest.mark.parametrize("kind2", ["q", "mu", "th"])
def test_multipole_energy_matches_point_charges(kind, kind2):
    """A multipole of a given order is built from a small point-charge cluster
    with the right symmetry (odd moments vanish for an inversion-symmetric
    quadrupole cluster); far away its energy with another cluster equals the
    multipole expansion term."""
    order = {"q": 0, "mu": 1, "th": 2}
    rng = np.random.default_rng(10 * order[kind] + order[kind2])
    d = 0.01

    def make(kind):
        v = rng.normal(size=3)
        w = rng.normal(size=3)
        if kind == "q":
            return np.array([0.7]), np.zeros((1, 3))
        if kind == "mu":
            return np.array([1.0, -1.0]), np.array([d * v, -d * v])
        # quadrupole: +q at +-v, -q at +-w (inversion symmetric, zero charge)
        return np.array([1.0, 1.0, -1.0, -1.0]), np.array([d * v, -d * v, d * w, -d * w])

    qa, sa = make(kind)
    qb, sb = make(kind2)
    ca = np.zeros(3)
    cb = np.array([4.0, -2.5, 3.0])
    exact = _point_energy(qa, sa, ca, qb, sb, cb)
    ma = _cluster_moments(qa, sa)
    mb = _cluster_moments(qb, sb)
    x = torch.tensor(ca - cb, dtype=DT)
    r = torch.linalg.vector_norm(x)
    T = core.tensors(x, core.g_bare(r, 4), 4)
    t = lambda a: torch.tensor(a, dtype=DT)
    U = float(core.mp_pair_energy(T, t(ma[0]), t(ma[1]), t(ma[2]), t(mb[0]), t(mb[1]), t(mb[2])))
    size = [abs(ma[0]), np.linalg.norm(ma[1]), np.linalg.norm(ma[2])][order[kind]]
    size *= [abs(mb[0]), np.linalg.norm(mb[1]), np.linalg.norm(mb[2])][order[kind2]]
    scale = size / float(r) ** (order[kind] + order[kind2] + 1)
    assert abs(U - exact) <= 1e-3 * scale, (U, exact, scale)
    assert abs(U) > 0.05 * scale


def test_bspline_partition_of_unity():
    w = torch.rand(50, dtype=DT)
    j = torch.arange(5, dtype=DT)
    v = w[:, None] + j
    np.testing.assert_allclose(ewald.bspline(5, v).sum(-1).numpy(), 1.0, atol=1e-14)
    for k in (1, 2, 3):
        np.testing.assert_allclose(ewald.bspline_deriv(5, v, k).sum(-1).numpy(), 0.0, atol=1e-12)
    # M_5 at the integers: (1, 11, 11, 1)/24
    np.testing.assert_allclose(ewald.bspline(5, torch.arange(1.0, 5.0, dtype=DT)).numpy() * 24,
                               [1, 11, 11, 1], atol=1e-13)
