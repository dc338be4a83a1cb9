"""Oracle Ewald machinery for point multipoles up to quadrupoles (FP64).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg; never by the product path.

The periodic electrostatics follows the paper's use of smooth particle mesh
Ewald for multipoles and polarization (Computational Details; section
"Overview" on the N log N SPME): real space with erfc kernels, reciprocal space
on a B-spline grid (Essmann et al. 1995, extended to multipoles by applying
the multipole differential operator to the spline weights), the Gaussian self
energy, and removal of the erf part of intramolecular pairs.  An exact Ewald
k-space sum is provided to pin the SPME.
"""
from __future__ import annotations

import itertools
import math

import torch

from .core import DT, SQRT_PI, t64


# ---------------------------------------------------------------------------
# Cardinal B-splines M_n (support [0, n]) and their derivatives.
# ---------------------------------------------------------------------------

def bspline(n, v):
    """M_n(v) by the recursion M_n(v) = [v M_{n-1}(v) + (n-v) M_{n-1}(v-1)]/(n-1),
    with M_2(v) = 1 - |v - 1| on [0, 2]."""
    if n == 2:
        return torch.where((v >= 0) & (v <= 2), 1.0 - torch.abs(v - 1.0), torch.zeros_like(v))
    return (v * bspline(n - 1, v) + (n - v) * bspline(n - 1, v - 1.0)) / (n - 1)


def bspline_deriv(n, v, k):
    """k-th derivative: sum_j (-1)^j C(k, j) M_{n-k}(v - j)."""
    if k == 0:
        return bspline(n, v)
    out = torch.zeros_like(v)
    for j in range(k + 1):
        out = out + ((-1) ** j) * math.comb(k, j) * bspline(n - k, v - j)
    return out


def spline_weights(x, box, K, order, nderiv):
    """For points x (N, 3): grid indices (N, 3, order) and weights
    W[d][k] (N, 3, order) = d^k/dx^k of M_n(u - grid) with u = K x / L.
    The grid points that touch u are floor(u) - j, j = 0..order-1, with spline
    argument frac(u) + j."""
    Kt = t64(K)
    u = x * (Kt / box)
    fl = torch.floor(u.detach())
    w = u - fl
    j = torch.arange(order, dtype=DT)
    v = w[..., None] + j                     # (N, 3, order)
    idx = (fl[..., None].long() - torch.arange(order)) % torch.as_tensor(K)[None, :, None]
    scale = (Kt / box)[None, :, None]
    W = [bspline_deriv(order, v, k) * scale ** k for k in range(nderiv + 1)]
    return idx, W


def _dir_product(W, N, order, a):
    """Tensor-product weights (N, o, o, o) with derivative multi-index a=(kx,ky,kz)."""
    wx, wy, wz = W[a[0]][:, 0], W[a[1]][:, 1], W[a[2]][:, 2]
    return wx[:, :, None, None] * wy[:, None, :, None] * wz[:, None, None, :]


def _flat_index(idx, K):
    ix, iy, iz = idx[:, 0], idx[:, 1], idx[:, 2]
    return (ix[:, :, None, None] * (K[1] * K[2]) + iy[:, None, :, None] * K[2]
            + iz[:, None, None, :])


# multi-indices for first / second / third Cartesian derivatives
D1 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]


def _mi(*axes):
    a = [0, 0, 0]
    for ax in axes:
        a[ax] += 1
    return tuple(a)


# ---------------------------------------------------------------------------
# General (triclinic) cells.  `box` is either the three edge lengths of an
# orthorhombic box or a 3x3 cell matrix h whose columns are the cell vectors
# (x = h s, s the fractional coordinates).  The grid coordinate of x is
# u = A x with A = diag(K) h^-1, so a Cartesian gradient is A^T times the
# gradient in u: multipoles are mapped to grid coordinates before the spread
# (mu_u = A mu, Theta_u = A Theta A^T) and potential derivatives back after
# the gather.  The virial (strain derivative) is taken through h.
# ---------------------------------------------------------------------------

def is_cell(box):
    return torch.is_tensor(box) and box.dim() == 2


def grid_map(cell, K):
    """A = diag(K) h^-1."""
    return t64(K)[:, None] * torch.linalg.inv(cell)


def _cell_weights(x, cell, K, order, nderiv):
    """Spline indices and weights in grid coordinates (derivatives with respect to u)."""
    A = grid_map(cell, K)
    u = x @ A.T
    fl = torch.floor(u.detach())
    w = u - fl
    j = torch.arange(order, dtype=DT)
    v = w[..., None] + j
    idx = (fl[..., None].long() - torch.arange(order)) % torch.as_tensor(K)[None, :, None]
    W = [bspline_deriv(order, v, k) for k in range(nderiv + 1)]
    return idx, W, A


def _spread_cell(x, q, mu, th, cell, K, order):
    N = x.shape[0]
    idx, W, A = _cell_weights(x, cell, K, order, 2)
    coef = q[:, None, None, None] * _dir_product(W, N, order, (0, 0, 0))
    if mu is not None:
        mu_u = mu @ A.T
        for a in range(3):
            coef = coef + mu_u[:, a, None, None, None] * _dir_product(W, N, order, D1[a])
    if th is not None:
        th_u = A @ th @ A.T
        for a in range(3):
            for b in range(3):
                coef = coef + (th_u[:, a, b] / 3.0)[:, None, None, None] * _dir_product(W, N, order, _mi(a, b))
    flat = _flat_index(idx, K).reshape(-1)
    Q = torch.zeros(K[0] * K[1] * K[2], dtype=DT).index_add(0, flat, coef.reshape(-1))
    return Q.reshape(K[0], K[1], K[2])


def _potential_derivs_cell(x, Psi, cell, K, order, nderiv):
    N = x.shape[0]
    idx, W, A = _cell_weights(x, cell, K, order, nderiv)
    flat = _flat_index(idx, K)
    vals = Psi.reshape(-1)[flat.reshape(-1)].reshape(N, order, order, order)

    def contract(a):
        return (_dir_product(W, N, order, a) * vals).sum((1, 2, 3))

    out = {"phi": contract((0, 0, 0))}
    if nderiv >= 1:
        d1 = torch.stack([contract(D1[a]) for a in range(3)], -1)
        out["d1"] = d1 @ A
    if nderiv >= 2:
        d2 = torch.stack([torch.stack([contract(_mi(a, b)) for b in range(3)], -1) for a in range(3)], -2)
        out["d2"] = A.T @ d2 @ A
    if nderiv >= 3:
        d3 = torch.stack([torch.stack([torch.stack([contract(_mi(a, b, c)) for c in range(3)], -1)
                                       for b in range(3)], -2) for a in range(3)], -3)
        out["d3"] = torch.einsum("ndef,da,eb,fc->nabc", d3, A, A, A)
    return out


def _influence_cell(cell, K, order, alpha, ke):
    """G on the grid for a general cell: reciprocal vectors m = h^-T k."""
    V = torch.abs(torch.linalg.det(cell))
    ks = []
    for d in range(3):
        k = torch.arange(K[d], dtype=DT)
        ks.append(torch.where(k > K[d] // 2, k - K[d], k))
    kx, ky, kz = torch.meshgrid(*ks, indexing="ij")
    kk = torch.stack([kx, ky, kz], -1).reshape(-1, 3)
    m = kk @ torch.linalg.inv(cell)            # rows: m^T = k^T h^-1
    m2 = (m * m).sum(-1).reshape(K[0], K[1], K[2])
    B = (bspline_moduli(K[0], order)[:, None, None] * bspline_moduli(K[1], order)[None, :, None]
         * bspline_moduli(K[2], order)[None, None, :])
    safe = torch.where(m2 > 0, m2, torch.ones_like(m2))
    G = torch.where(m2 > 0, torch.exp(-math.pi ** 2 * m2 / alpha ** 2) * B / (math.pi * V * safe),
                    torch.zeros_like(m2))
    return G * (K[0] * K[1] * K[2]) * ke


def spread(x, q, mu, th, box, K, order):
    """Grid Q(k) = sum_i [q_i + mu_i . grad_i + (1/3) Theta_i : grad_i grad_i] W_i(k)."""
    N = x.shape[0]
    if is_cell(box):
        return _spread_cell(x, q, mu, th, box, K, order)
    idx, W = spline_weights(x, box, K, order, 2)
    coef = q[:, None, None, None] * _dir_product(W, N, order, (0, 0, 0))
    if mu is not None:
        for a in range(3):
            coef = coef + mu[:, a, None, None, None] * _dir_product(W, N, order, D1[a])
    if th is not None:
        for a in range(3):
            for b in range(3):
                coef = coef + (th[:, a, b] / 3.0)[:, None, None, None] * _dir_product(W, N, order, _mi(a, b))
    flat = _flat_index(idx, K).reshape(-1)
    Q = torch.zeros(K[0] * K[1] * K[2], dtype=DT).index_add(0, flat, coef.reshape(-1))
    return Q.reshape(K[0], K[1], K[2])


def bspline_moduli(K, order):
    """|b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2."""
    kk = torch.arange(order - 1, dtype=DT)
    Mk = bspline(order, kk + 1.0)
    m = torch.arange(K, dtype=DT)
    ph = 2 * math.pi * m[:, None] * kk[None, :] / K
    re = (Mk * torch.cos(ph)).sum(-1)
    im = (Mk * torch.sin(ph)).sum(-1)
    den = re * re + im * im
    # For odd orders the sum vanishes at m = K/2; there the denominator is
    # replaced by the mean of its two neighbours (the weight at that frequency
    # is far below rounding for the grids used).
    small = den < 1e-7
    if bool(small.any()):
        nb = 0.5 * (torch.roll(den, 1) + torch.roll(den, -1))
        den = torch.where(small, nb, den)
    return 1.0 / den


def influence(box, K, order, alpha, ke):
    """G(m) such that E_rec = 1/2 sum_k Q(k) Psi(k), Psi = IFFT(G FFT(Q)):
    G(m) = K1 K2 K3 ke exp(-pi^2 |m~|^2/alpha^2) B(m) / (pi V |m~|^2), G(0) = 0,
    with m~ = (m1/L1, m2/L2, m3/L3) and folded integer frequencies m."""
    if is_cell(box):
        return _influence_cell(box, K, order, alpha, ke)
    box = t64(box)
    V = float(box[0] * box[1] * box[2])
    freqs = []
    for d in range(3):
        m = torch.arange(K[d], dtype=DT)
        m = torch.where(m > K[d] // 2, m - K[d], m)
        freqs.append(m / box[d])
    mx, my, mz = torch.meshgrid(*freqs, indexing="ij")
    m2 = mx * mx + my * my + mz * mz
    B = (bspline_moduli(K[0], order)[:, None, None] * bspline_moduli(K[1], order)[None, :, None]
         * bspline_moduli(K[2], order)[None, None, :])
    G = torch.where(m2 > 0,
                    torch.exp(-math.pi ** 2 * m2 / alpha ** 2) * B / (math.pi * V * torch.where(m2 > 0, m2, torch.ones_like(m2))),
                    torch.zeros_like(m2))
    return G * (K[0] * K[1] * K[2]) * ke


def convolve(Q, G):
    return torch.fft.ifftn(G * torch.fft.fftn(Q)).real


def grid_energy(Q, G):
    return 0.5 * (Q * convolve(Q, G)).sum()


def potential_derivs(x, Psi, box, K, order, nderiv):
    """phi and its Cartesian derivatives up to nderiv at points x from the
    convolved grid Psi.  Returns dict: 'phi' (N,), 'd1' (N,3), 'd2' (N,3,3),
    'd3' (N,3,3,3)."""
    if is_cell(box):
        return _potential_derivs_cell(x, Psi, box, K, order, nderiv)
    N = x.shape[0]
    idx, W = spline_weights(x, box, K, order, nderiv)
    flat = _flat_index(idx, K)
    vals = Psi.reshape(-1)[flat.reshape(-1)].reshape(N, order, order, order)

    def contract(a):
        return (_dir_product(W, N, order, a) * vals).sum((1, 2, 3))

    out = {"phi": contract((0, 0, 0))}
    if nderiv >= 1:
        out["d1"] = torch.stack([contract(D1[a]) for a in range(3)], -1)
    if nderiv >= 2:
        out["d2"] = torch.stack([torch.stack([contract(_mi(a, b)) for b in range(3)], -1)
                                 for a in range(3)], -2)
    if nderiv >= 3:
        out["d3"] = torch.stack([torch.stack([torch.stack([contract(_mi(a, b, c)) for c in range(3)], -1)
                                              for b in range(3)], -2) for a in range(3)], -3)
    return out


# ---------------------------------------------------------------------------
# Exact Ewald reciprocal sum (validation of the SPME), self energy.
# ---------------------------------------------------------------------------

def exact_recip_energy(x, q, mu, th, box, alpha, ke, mmax):
    """(ke / 2 pi V) sum_{m != 0} exp(-pi^2 m~^2/alpha^2)/m~^2 |S(m)|^2 with
    S(m) = sum_j [q_j + 2 pi i m~.mu_j - (4 pi^2/3) m~.Theta_j.m~] exp(2 pi i m~.r_j).
    For a 3x3 cell h (columns = cell vectors), m~ = h^-T m and V = |det h|."""
    rng = torch.arange(-mmax, mmax + 1, dtype=DT)
    mm = torch.stack(torch.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    mm = mm[(mm != 0).any(-1)]
    if is_cell(box):
        V = float(torch.abs(torch.linalg.det(box)))
        mt = mm @ torch.linalg.inv(box)
    else:
        box = t64(box)
        V = float(box[0] * box[1] * box[2])
        mt = mm / box
    m2 = (mt * mt).sum(-1)
    E = x.new_zeros(())
    for chunk in torch.split(torch.arange(mt.shape[0]), 4096):
        m = mt[chunk]
        ph = 2 * math.pi * x @ m.T                                   # (N, C)
        a_re = q[:, None] - (4 * math.pi ** 2 / 3.0) * torch.einsum("ca,nab,cb->nc", m, th, m)
        a_im = 2 * math.pi * (mu @ m.T)
        c, s = torch.cos(ph), torch.sin(ph)
        s_re = (a_re * c - a_im * s).sum(0)
        s_im = (a_re * s + a_im * c).sum(0)
        w = torch.exp(-math.pi ** 2 * m2[chunk] / alpha ** 2) / m2[chunk]
        E = E + (w * (s_re * s_re + s_im * s_im)).sum()
    return E * ke / (2 * math.pi * V)


def self_energy(q, mu, th, alpha, ke):
    """Gaussian self energy of point multipoles (q, mu, traceless Theta with the
    1/3 convention): -ke alpha/sqrt(pi) sum [q^2 + (2 alpha^2/3) mu.mu
    + (8 alpha^4/45) Theta:Theta]."""
    s = (q * q + (2 * alpha ** 2 / 3.0) * (mu * mu).sum(-1)
         + (8 * alpha ** 4 / 45.0) * (th * th).sum((-1, -2)))
    return -ke * alpha / SQRT_PI * s.sum()


def lattice_images(nmax):
    """Integer image vectors n with |n| <= nmax (spherical ordering)."""
    r = range(-nmax, nmax + 1)
    pts = [p for p in itertools.product(r, r, r) if p[0] ** 2 + p[1] ** 2 + p[2] ** 2 <= nmax * nmax]
    return t64(pts)
