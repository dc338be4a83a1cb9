"""Oracle building blocks: local frames, extra centres, radial kernels and
Cartesian interaction tensors (FP64, PyTorch CPU).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg; never by the product path.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64
SQRT_PI = math.sqrt(math.pi)


def t64(a):
    return torch.as_tensor(a, dtype=DT)


# ---------------------------------------------------------------------------
# Local frames and sites (section "Multipolar Electrostatics": multipoles are
# stored in a local frame of their molecule and rotated to the global frame
# at each step; exchange-repulsion section: explicit lone-pair extra centres).
# ---------------------------------------------------------------------------

def frame(zvec, xvec):
    """Right-handed orthonormal frame with z along zvec and x in the (z, xvec)
    plane.  Returns (..., 3, 3) whose columns are the x, y, z axes."""
    z = zvec / torch.linalg.vector_norm(zvec, dim=-1, keepdim=True)
    xp = xvec - (xvec * z).sum(-1, keepdim=True) * z
    x = xp / torch.linalg.vector_norm(xp, dim=-1, keepdim=True)
    y = torch.linalg.cross(z, x, dim=-1)
    return torch.stack([x, y, z], dim=-1)


def sym_from6(v):
    """[xx, yy, zz, xy, xz, yz] -> symmetric 3x3."""
    xx, yy, zz, xy, xz, yz = (v[..., k] for k in range(6))
    r0 = torch.stack([xx, xy, xz], -1)
    r1 = torch.stack([xy, yy, yz], -1)
    r2 = torch.stack([xz, yz, zz], -1)
    return torch.stack([r0, r1, r2], -2)


def build_sites(pos, mp_local, P):
    """Global sites of every water.

    pos: (M, 3, 3) atoms O, H1, H2.  mp_local: (M, 5, 10).
    Frames: O uses z = bisector of the two unit O->H vectors and x toward H1;
    H_k and the midpoint M_k use z along H_k->O and x toward the other H.
    Lone pairs sit at d_lp from O along -cos(t) z_O +/- sin(t) y_O.
    """
    O, H1, H2 = pos[:, 0], pos[:, 1], pos[:, 2]
    u1 = (H1 - O) / torch.linalg.vector_norm(H1 - O, dim=-1, keepdim=True)
    u2 = (H2 - O) / torch.linalg.vector_norm(H2 - O, dim=-1, keepdim=True)
    RO = frame(u1 + u2, H1 - O)
    R1 = frame(O - H1, H2 - H1)
    R2 = frame(O - H2, H1 - H2)
    R = torch.stack([RO, R1, R2, R1, R2], dim=1)            # (M,5,3,3)
    xs = torch.stack([O, H1, H2, 0.5 * (O + H1), 0.5 * (O + H2)], dim=1)
    th = math.radians(P["lp_half_deg"])
    d = P["d_lp"]
    zO, yO = RO[..., 2], RO[..., 1]
    lp = torch.stack([O + d * (-math.cos(th) * zO + math.sin(th) * yO),
                      O + d * (-math.cos(th) * zO - math.sin(th) * yO)], dim=1)
    mp = t64(mp_local)
    q = mp[..., 0]
    mu = torch.einsum("msij,msj->msi", R, mp[..., 1:4])
    th_l = sym_from6(mp[..., 4:10])
    Th = R @ th_l @ R.transpose(-1, -2)
    return {"x": xs, "lp": lp, "q": q, "mu": mu, "th": Th, "R": R}


# ---------------------------------------------------------------------------
# Radial kernels.  For a kernel g0(r), g_{n+1}(r) = (1/r) d g_n / dr, so the
# Cartesian derivatives of g0(|x|) are polynomials in x with these weights.
# ---------------------------------------------------------------------------

def g_bare(r, nmax):
    """1/r: g_n = (-1)^n (2n-1)!! / r^(2n+1)."""
    out, df = [], 1.0
    for n in range(nmax + 1):
        out.append(((-1) ** n) * df / r ** (2 * n + 1))
        df *= 2 * n + 1
    return out


def g_erfc(r, alpha, nmax):
    """erfc(alpha r)/r (Ewald real space): Smith's B_n recursion,
    B_n = [(2n-1) B_{n-1} + (2 alpha^2)^n exp(-alpha^2 r^2)/(alpha sqrt(pi))]/r^2,
    and g_n = (-1)^n B_n."""
    r2 = r * r
    ex = torch.exp(-alpha * alpha * r2) / (alpha * SQRT_PI)
    b = torch.erfc(alpha * r) / r
    out = [b]
    for n in range(1, nmax + 1):
        b = ((2 * n - 1) * b + (2 * alpha * alpha) ** n * ex) / r2
        out.append(((-1) ** n) * b)
    return out


def g_erf(r, alpha, nmax):
    """erf(alpha r)/r = 1/r - erfc(alpha r)/r."""
    return [a - b for a, b in zip(g_bare(r, nmax), g_erfc(r, alpha, nmax))]


def _rev_bessel(n, x):
    """Reverse Bessel polynomial theta_n(x): theta_0 = 1, theta_1 = x + 1,
    theta_n = (2n-1) theta_{n-1} + x^2 theta_{n-2}."""
    if n == 0:
        return torch.ones_like(x)
    a, b = torch.ones_like(x), x + 1.0
    for k in range(2, n + 1):
        a, b = b, (2 * k - 1) * b + x * x * a
    return b


def g_exp(r, b, nmax):
    """exp(-b r)/r: g_n = (-1)^n exp(-b r) theta_n(b r) / r^(2n+1)."""
    e = torch.exp(-b * r)
    x = b * r
    return [((-1) ** n) * e * _rev_bessel(n, x) / r ** (2 * n + 1) for n in range(nmax + 1)]


def thole_lambdas(r, A, a):
    """Exponential Thole damping factors lambda_3, lambda_5, lambda_7, lambda_9
    for u = r/A, t = a u^3 (a = Thole parameter, A = (alpha_i alpha_j)^(1/6))."""
    t = a * (r / A) ** 3
    e = torch.exp(-t)
    l3 = 1.0 - e
    l5 = 1.0 - (1.0 + t) * e
    l7 = 1.0 - (1.0 + t + 0.6 * t * t) * e
    l9 = 1.0 - (1.0 + t + (18.0 / 35.0) * t * t + (9.0 / 35.0) * t ** 3) * e
    return [l3, l5, l7, l9]


def g_thole(r, A, a, alpha=None, nmax=4):
    """Thole-damped kernel weights g_1..g_nmax (g_0 is never needed because the
    damping acts on induced dipoles only).  Gas phase: lambda_{2n+1} g_n(1/r).
    Periodic: erfc kernel plus (lambda - 1) g_n(1/r) in real space."""
    lam = thole_lambdas(r, A, a)
    gb = g_bare(r, nmax)
    if alpha is None:
        out = [torch.zeros_like(r)] + [lam[n - 1] * gb[n] for n in range(1, nmax + 1)]
    else:
        ge = g_erfc(r, alpha, nmax)
        out = [torch.zeros_like(r)] + [ge[n] + (lam[n - 1] - 1.0) * gb[n] for n in range(1, nmax + 1)]
    return out


# ---------------------------------------------------------------------------
# Cartesian interaction tensors T_n = d^n g0(|x|) / dx^n for a radial kernel.
# ---------------------------------------------------------------------------

_I3 = torch.eye(3, dtype=DT)


def tensors(x, g, nmax):
    """x: (..., 3); g: list of (...) tensors.  Returns [T0, T1, ..., T_nmax]."""
    d = _I3
    T = [g[0]]
    if nmax >= 1:
        T.append(x * g[1][..., None])
    if nmax >= 2:
        xx = x[..., :, None] * x[..., None, :]
        T.append(xx * g[2][..., None, None] + d * g[1][..., None, None])
    if nmax >= 3:
        xxx = xx[..., :, :, None] * x[..., None, None, :]
        dx = (d[:, :, None] * x[..., None, None, :]
              + d[:, None, :] * x[..., None, :, None]
              + d[None, :, :] * x[..., :, None, None])
        T.append(xxx * g[3][..., None, None, None] + dx * g[2][..., None, None, None])
    if nmax >= 4:
        xxxx = xxx[..., None] * x[..., None, None, None, :]
        dxx = (d[:, :, None, None] * xx[..., None, None, :, :]
               + d[:, None, :, None] * xx[..., None, :, None, :]
               + d[:, None, None, :] * xx[..., None, :, :, None]
               + d[None, :, :, None] * xx[..., :, None, None, :]
               + d[None, :, None, :] * xx[..., :, None, :, None]
               + d[None, None, :, :] * xx[..., :, :, None, None])
        dd = (d[:, :, None, None] * d[None, None, :, :]
              + d[:, None, :, None] * d[None, :, None, :]
              + d[:, None, None, :] * d[None, :, :, None])
        T.append(xxxx * g[4][..., None, None, None, None]
                 + dxx * g[3][..., None, None, None, None]
                 + dd * g[2][..., None, None, None, None])
    return T


def mp_potential(T, qb, mub, thb):
    """Potential of multipole b at displacement x = r - r_b:
    phi = q T0 - mu . T1 + (1/3) Theta : T2."""
    return (qb * T[0] - (mub * T[1]).sum(-1)
            + (thb * T[2]).sum((-1, -2)) / 3.0)


def mp_pair_energy(T, qa, mua, tha, qb, mub, thb):
    """Interaction energy of multipole a (at r_a) with multipole b (at r_b),
    x = r_a - r_b: U = q_a phi_b + mu_a . D phi_b + (1/3) Theta_a : DD phi_b."""
    phi = qb * T[0] - (mub * T[1]).sum(-1) + (thb * T[2]).sum((-1, -2)) / 3.0
    dphi = (qb[..., None] * T[1] - (T[2] * mub[..., None, :]).sum(-1)
            + (T[3] * thb[..., None, :, :]).sum((-1, -2)) / 3.0)
    ddphi = (qb[..., None, None] * T[2] - (T[3] * mub[..., None, None, :]).sum(-1)
             + (T[4] * thb[..., None, None, :, :]).sum((-1, -2)) / 3.0)
    return qa * phi + (mua * dphi).sum(-1) + (tha * ddphi).sum((-1, -2)) / 3.0


def dipole_mp_energy(T, mua, qb, mub, thb):
    """Energy of a point dipole mu_a at r_a in the potential of multipole b:
    mu_a . D phi_b (x = r_a - r_b); needs T1..T3."""
    dphi = (qb[..., None] * T[1] - (T[2] * mub[..., None, :]).sum(-1)
            + (T[3] * thb[..., None, :, :]).sum((-1, -2)) / 3.0)
    return (mua * dphi).sum(-1)


def dipole_dipole_energy(T, mua, mub):
    """-mu_a . T2 . mu_b (x = r_a - r_b)."""
    return -(mua * (T[2] * mub[..., None, :]).sum(-1)).sum(-1)
