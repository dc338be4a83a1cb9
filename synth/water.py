"""Seeded water systems and the synthetic SIBFA parameter table.

Everything here is input data.  Geometries follow the workload recipes:
rigid waters (O-H 0.9572 A, HOH 104.52 deg) with uniform random orientations
on a jittered cubic lattice (minimum O-O 2.5 A), or compact gas-phase
clusters.  Each molecule draws its own local-frame multipoles: q_O uniform in
[-0.85, -0.75], the four other sites (H1, H2 and the two O-H bond midpoints)
carry -q_O/4 so the molecule is neutral; in each site's local frame the
dipole lies along z (O: uniform in [0, 0.3] e.A; H: [0, 0.1]; midpoints:
[-0.1, 0.1]) and the quadrupole is diagonal and traceless (diagonal entries
uniform in [-0.5, 0.5] e.A^2 on O, [-0.1, 0.1] on H, [-0.2, 0.2] on the
midpoints, then the mean removed).  This mimics the axial layout of
ISA-derived water multipoles.

Site order inside a molecule: 0 = O, 1 = H1, 2 = H2, 3 = M1 (midpoint O-H1),
4 = M2 (midpoint O-H2).  Lone pairs: 0, 1.  Local multipole layout per site:
[q, mu_x, mu_y, mu_z, Th_xx, Th_yy, Th_zz, Th_xy, Th_xz, Th_yz].

The parameter values the paper prints are used where it prints them (O
exchange-repulsion radius 1.4755 A, O dispersion radius 1.2594 A, lone-pair
dispersion radius 0.9042 A, Thole 0.28, ideal geometry); every other value is
synthetic, chosen so that (1) the near-linear water dimer at r_OO = 2.91 A has
component energies close to the paper's Table 1 first column (repulsion
6.9, dispersion -2.14, charge transfer -1.06 kcal/mol), (2) the dimer energy
has no well inside 2.3 A in any of 25 sampled relative orientations (the
repulsion outgrows dispersion and charge transfer there), and (3) the
charge-transfer denominator ae + V - ah cannot reach zero at any potential a
lone pair meets in the liquid, so that velocity-Verlet runs of the water
boxes stay stable for thousands of steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_SITES = 5
N_LP = 2
N_MP = 10

WATER_GEOM = {
    "r_oh": 0.9572,          # A
    "hoh_deg": 104.52,       # degrees
    "d_lp": 0.5,             # A, O -> lone pair distance
    "lp_half_deg": 54.7356103172,  # half of the tetrahedral angle
    "mass_o": 15.999,
    "mass_h": 1.008,
}

# Synthetic SIBFA parameter table (kcal/mol, A, e).  Printed values noted.
PARAMS = {
    "ke": 332.063713,         # kcal A / (mol e^2)
    "debye": 4.80321,         # D per e.A
    # geometry of the extra centres
    "d_lp": WATER_GEOM["d_lp"],
    "lp_half_deg": WATER_GEOM["lp_half_deg"],
    # polarization (isotropic, Thole)
    "alpha_o": 1.0,
    "alpha_h": 0.5,
    "alpha_m_damp": 0.75,     # midpoint polarizability used only inside Thole damping
    "thole": 0.28,            # printed
    # penetration: nuclear charge and valence damping exponent per atom type
    "z_o": 6.0,
    "z_h": 1.0,
    "b_o": 3.0,
    "b_h": 3.4,
    # exchange-repulsion
    "cs_o": 0.5,
    "cp_o": math.sqrt(3.0) / 2.0,
    "cs_h": 1.0,
    "cp_h": 0.0,
    "cs_lp": 0.5,
    "cp_lp": math.sqrt(3.0) / 2.0,
    "g_o": 1.0,
    "g_h": 0.6,
    "nval_o": 6.0,
    "nval_h": 1.0,
    "rvdw_rep_o": 1.4755,     # printed
    "rvdw_rep_h": 1.10,
    "rvdw_rep_lp": 1.30,
    "rep_alpha": 14.0,
    "rep_alpha2": 16.3333,
    "rep_c1": 93884.0,
    "rep_c2": 46942.0,
    "rep_f": 0.8,
    "occ_bond": 2.0,
    "n_lp": 2.0,
    # dispersion
    "rvdw_disp_o": 1.2594,    # printed
    "rvdw_disp_h": 0.95,
    "rvdw_disp_lp": 0.9042,   # printed
    "disp_alpha": 1.2,
    "beta_o": 1.0,
    "beta_h": 0.45,
    "c6": 0.5459,
    "c8": 0.4453,
    "c10": 0.3591,
    "gamma6": 2.0,
    "gamma8": 2.3,
    "gamma10": 2.6,
    "disp_delta": 0.30,
    # exchange-dispersion
    "xd_c1": 20.0,
    "xd_a1": 4.5,
    "xd_c2": 8.0,
    "xd_a2": 4.5,
    "xd_c3": 10.0,
    "xd_a3": 4.5,
    # reduced charge transfer
    "ct_eta": 2.2,
    "ct_t": 0.3944,
    "ct_m": 0.3133,
    "ct_ae": 2000.0,          # lone-pair ionization potential (kcal/mol)
    "ct_ah": 60.0,            # heavy-atom electron affinity (kcal/mol)
    "rvdw_ct_o": 1.50,
    "rvdw_ct_h": 1.10,
}


@dataclass
class System:
    """A set of rigid-geometry waters.

    pos:      (M, 3, 3) float64, atoms O, H1, H2 of each molecule (A)
    mp_local: (M, 5, 10) float64, local-frame multipoles per site
    box:      (3,) float64 orthorhombic box lengths, or None in the gas phase
    """
    pos: np.ndarray
    mp_local: np.ndarray
    box: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_mol(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_atoms(self) -> int:
        return 3 * self.n_mol

    def masses(self) -> np.ndarray:
        m = np.empty((self.n_mol, 3))
        m[:, 0] = WATER_GEOM["mass_o"]
        m[:, 1:] = WATER_GEOM["mass_h"]
        return m


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a Shoemake quaternion."""
    u1, u2, u3 = rng.random(3)
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    qw = a * math.sin(2 * math.pi * u2)
    qx = a * math.cos(2 * math.pi * u2)
    qy = b * math.sin(2 * math.pi * u3)
    qz = b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def _water_body() -> np.ndarray:
    """O, H1, H2 in a body frame: O at origin, bisector along +z, plane xz."""
    r = WATER_GEOM["r_oh"]
    h = math.radians(WATER_GEOM["hoh_deg"]) / 2.0
    return np.array([
        [0.0, 0.0, 0.0],
        [r * math.sin(h), 0.0, r * math.cos(h)],
        [-r * math.sin(h), 0.0, r * math.cos(h)],
    ])


def _random_multipoles(rng: np.random.Generator, n_mol: int) -> np.ndarray:
    """Per-molecule draws with an ISA-like layout in each site's local frame:
    dipoles along the local z axis (the O bisector, the bond for H and the
    midpoints) and diagonal traceless quadrupoles.  Bounds: |mu| <= 0.3 e.A
    and quadrupole entries <= 0.5 e.A^2 on O; the H and midpoint moments are
    drawn from smaller ranges inside the same bounds."""
    mp = np.zeros((n_mol, N_SITES, N_MP))
    q_o = rng.uniform(-0.85, -0.75, size=n_mol)
    mp[:, 0, 0] = q_o
    mp[:, 1:, 0] = (-q_o / 4.0)[:, None]
    mu_rng = np.array([[0.0, 0.3], [0.0, 0.1], [0.0, 0.1], [-0.1, 0.1], [-0.1, 0.1]])
    th_rng = np.array([0.5, 0.1, 0.1, 0.2, 0.2])
    for s in range(N_SITES):
        mp[:, s, 3] = rng.uniform(mu_rng[s, 0], mu_rng[s, 1], size=n_mol)
        d = rng.uniform(-th_rng[s], th_rng[s], size=(n_mol, 3))
        d -= d.mean(axis=1, keepdims=True)
        mp[:, s, 4:7] = d
    return mp


def general_multipoles(rng: np.random.Generator, n_mol: int) -> np.ndarray:
    """Per-molecule draws with no symmetry in the local frames, for parity
    tests of the full rotation (all dipole components, off-diagonal
    quadrupoles): charges as in the workloads (q_O uniform in [-0.85, -0.75],
    -q_O/4 on the other four sites); on every site a dipole of uniformly random
    direction with |mu| uniform in [0, 0.3] e.A, and a quadrupole whose six
    independent entries are uniform in [-0.5, 0.5] e.A^2 before the trace is
    removed from the diagonal."""
    mp = np.zeros((n_mol, N_SITES, N_MP))
    q_o = rng.uniform(-0.85, -0.75, size=n_mol)
    mp[:, 0, 0] = q_o
    mp[:, 1:, 0] = (-q_o / 4.0)[:, None]
    d = rng.normal(size=(n_mol, N_SITES, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    mp[:, :, 1:4] = d * rng.uniform(0.0, 0.3, size=(n_mol, N_SITES, 1))
    th = rng.uniform(-0.5, 0.5, size=(n_mol, N_SITES, 6))
    th[..., 0:3] -= th[..., 0:3].mean(axis=-1, keepdims=True)
    mp[:, :, 4:10] = th
    return mp


def with_general_multipoles(system: "System", seed: int) -> "System":
    """The same geometry with general_multipoles drawn from `seed`."""
    rng = np.random.default_rng(seed)
    meta = dict(system.meta)
    meta["multipoles"] = ("general", seed)
    return System(pos=system.pos.copy(), mp_local=general_multipoles(rng, system.n_mol),
                  box=None if system.box is None else system.box.copy(), meta=meta)


MIN_ATOM_DIST = 1.7   # A, minimum intermolecular atom-atom distance of a starting structure


def _place_molecules(rng, propose, n, box, min_oo, min_atom=MIN_ATOM_DIST, tries=400):
    """Sequential placement of rigid waters: each molecule draws a position
    (propose(k)) and a uniform random orientation until its O is at least
    min_oo from every placed O and each of its atoms at least min_atom from
    every atom of another molecule (minimum image in a box).  A spatial hash
    limits the test to nearby molecules."""
    body = _water_body()
    pos = np.empty((n, 3, 3))
    reach = min_atom + 2.0 * WATER_GEOM["r_oh"]          # O-O range that can violate min_atom
    cut = max(min_oo, reach)
    if box is not None:
        nc = np.maximum(1, np.floor(box / cut).astype(int))
        cs = box / nc
    else:
        nc = None
        cs = np.array([cut] * 3)
    cells = {}

    def key(p):
        c = np.floor(p / cs).astype(int)
        if nc is not None:
            c %= nc
        return tuple(c)

    def nearby(p):
        c0 = np.floor(p / cs).astype(int)
        out = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    c = c0 + (dx, dy, dz)
                    if nc is not None:
                        c %= nc
                    out.extend(cells.get(tuple(c), ()))
        return sorted(set(out))

    for k in range(n):
        best = None
        for _ in range(tries):
            p = propose(k)
            atoms = p + body @ random_rotation(rng).T
            ok = True
            for j in nearby(p):
                d = pos[j][None, :, :] - atoms[:, None, :]
                if box is not None:
                    d -= box * np.round(d / box)
                r2 = np.einsum("abk,abk->ab", d, d)
                if r2[0, 0] < min_oo * min_oo or r2.min() < min_atom * min_atom:
                    ok = False
                    break
            if ok:
                best = atoms
                break
            if best is None:
                best = atoms
        pos[k] = best
        cells.setdefault(key(pos[k, 0]), []).append(k)
    return pos


def make_box(n_side: int, box_len: float, seed: int, n_remove: int = 0,
             jitter: float = 0.4, min_oo: float = 2.5) -> System:
    """Waters on a jittered n_side^3 cubic lattice in a cubic periodic box."""
    rng = np.random.default_rng(seed)
    a = box_len / n_side
    idx = np.stack(np.meshgrid(np.arange(n_side), np.arange(n_side), np.arange(n_side),
                               indexing="ij"), -1).reshape(-1, 3)
    if n_remove:
        keep = np.sort(rng.permutation(idx.shape[0])[: idx.shape[0] - n_remove])
        idx = idx[keep]
    centers = (idx + 0.5) * a
    box = np.array([box_len] * 3, dtype=np.float64)

    def propose(k):
        return centers[k] + (rng.uniform(-jitter, jitter, size=3) if jitter > 0 else 0.0)

    pos = _place_molecules(rng, propose, centers.shape[0], box, min_oo)
    mp = _random_multipoles(rng, pos.shape[0])
    return System(pos=pos, mp_local=mp, box=box,
                  meta={"kind": "box", "n_side": n_side, "seed": seed})


def make_ortho_box(n_sides, box_lens, seed: int, jitter: float = 0.4, min_oo: float = 2.5) -> System:
    """Waters on a jittered nx x ny x nz lattice in an orthorhombic periodic
    box of edges box_lens (a non-cubic cell for the per-axis paths)."""
    rng = np.random.default_rng(seed)
    n = np.asarray(n_sides, dtype=np.int64)
    box = np.asarray(box_lens, dtype=np.float64)
    a = box / n
    idx = np.stack(np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij"),
                   -1).reshape(-1, 3)
    centers = (idx + 0.5) * a

    def propose(k):
        return centers[k] + (rng.uniform(-jitter, jitter, size=3) if jitter > 0 else 0.0)

    pos = _place_molecules(rng, propose, centers.shape[0], box, min_oo)
    mp = _random_multipoles(rng, pos.shape[0])
    return System(pos=pos, mp_local=mp, box=box,
                  meta={"kind": "ortho_box", "n_sides": tuple(int(v) for v in n), "seed": seed})


def make_cluster_sizes(sizes, seed: int):
    """A gas-phase batch with the given cluster sizes (in order); each cluster
    is make_cluster with its own seed drawn from `seed`.  Returns the same
    triple as make_cluster_batch."""
    rng = np.random.default_rng(seed)
    seeds = rng.integers(0, 2**31 - 1, size=len(sizes))
    parts = [make_cluster(int(n), seed=int(s)) for n, s in zip(sizes, seeds)]
    start = np.zeros(len(sizes) + 1, dtype=np.int32)
    start[1:] = np.cumsum(sizes)
    allsys = System(pos=np.concatenate([c.pos for c in parts]), mp_local=np.concatenate([c.mp_local for c in parts]),
                    box=None, meta={"kind": "cluster_batch", "n_clusters": len(sizes), "seed": seed})
    return allsys, start, parts


def make_cluster(n_mol: int, seed: int, min_oo: float = 2.5) -> System:
    """Gas-phase cluster: O uniform in a sphere of radius 3 n^(1/3) A."""
    rng = np.random.default_rng(seed)
    radius = 3.0 * n_mol ** (1.0 / 3.0)

    def propose(k):
        while True:
            p = rng.uniform(-radius, radius, size=3)
            if p @ p <= radius * radius:
                return p

    pos = _place_molecules(rng, propose, n_mol, None, min_oo)
    mp = _random_multipoles(rng, n_mol)
    return System(pos=pos, mp_local=mp, box=None,
                  meta={"kind": "cluster", "n_mol": n_mol, "seed": seed})


def make_dimer(r_oo: float = 2.91, seed: int = 0) -> System:
    """Near-linear water dimer: H1 of the donor points at the acceptor O."""
    body = _water_body()
    # donor: rotate so O->H1 lies along +x
    h = math.radians(WATER_GEOM["hoh_deg"]) / 2.0
    c, s = math.cos(math.pi / 2 - h), math.sin(math.pi / 2 - h)
    rot_y = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    donor = body @ rot_y.T
    u = donor[1] / np.linalg.norm(donor[1])
    rot = _rot_between(u, np.array([1.0, 0.0, 0.0]))
    donor = donor @ rot.T
    # acceptor: bisector pointing away along +x, tilted ~ 57 deg out of line
    t = math.radians(57.0)
    rot_t = np.array([[math.cos(t), 0, math.sin(t)], [0, 1, 0], [-math.sin(t), 0, math.cos(t)]])
    acc_body = body @ _rot_between(np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])).T
    acc = acc_body @ rot_t.T + np.array([r_oo, 0.0, 0.0])
    pos = np.stack([donor, acc])
    rng = np.random.default_rng(seed)
    mp = _random_multipoles(rng, 2)
    return System(pos=pos, mp_local=mp, box=None, meta={"kind": "dimer", "r_oo": r_oo})


def _rot_between(a, b):
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    v = np.cross(a, b)
    c = float(a @ b)
    if np.linalg.norm(v) < 1e-12:
        return np.eye(3) if c > 0 else -np.eye(3)
    vx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + vx + vx @ vx * (1.0 / (1.0 + c))


def maxwell_velocities(system: System, temperature: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities in A/fs with the centre-of-mass momentum removed."""
    rng = np.random.default_rng(seed)
    kb = 0.0019872041            # kcal/(mol K)
    conv = 4.184e-4              # (kcal/mol/amu) -> A^2/fs^2
    m = system.masses()
    sig = np.sqrt(kb * temperature / m * conv)
    v = rng.normal(size=system.pos.shape) * sig[..., None]
    p = (v * m[..., None]).reshape(-1, 3).sum(0)
    v -= p / m.sum()
    return v


# Workload presets.  Sizes and settings follow the water-box and cluster
# recipes; the run options (cutoff, grid, Ewald alpha, tolerance) are returned
# beside the system.
CONFIGS = {
    "water216": dict(n_side=6, box=18.62, seed=1, n_remove=0, rc=7.0, grid=24,
                     ewald=0.4, pcg_tol=1e-8),
    "water4096": dict(n_side=16, box=49.66, seed=2, n_remove=0, rc=9.0, grid=64,
                      ewald=0.4, pcg_tol=1e-6),
    "water32000": dict(n_side=32, box=98.6, seed=3, n_remove=768, rc=9.0, grid=108,
                       ewald=0.4, pcg_tol=1e-6),
    # the paper's own MD setting (Computational Details): 216 waters in an
    # 18.643 A box, SPME grid 120^3, Ewald and repulsion cutoff 7 A, PCG
    # 1e-5 D (run with the Beeman integrator at 1 fs)
    "water216_paper": dict(n_side=6, box=18.643, seed=1, n_remove=0, rc=7.0, grid=120,
                           ewald=0.4, pcg_tol=1e-5),
}


def make_config(name: str):
    """Return (System, run-options dict) for a named workload preset."""
    c = CONFIGS[name]
    sysm = make_box(c["n_side"], c["box"], c["seed"], n_remove=c["n_remove"])
    opts = {"rc": c["rc"], "grid": c["grid"], "order": 5, "ewald": c["ewald"],
            "pcg_tol": c["pcg_tol"]}
    return sysm, opts


def make_cluster_batch(n_clusters: int, seed: int, n_min: int = 2, n_max: int = 32):
    """A batch of independent gas-phase clusters, sizes uniform in
    [n_min, n_max]; each cluster is make_cluster with its own seed drawn from
    the batch seed.  Returns (System of all molecules, cluster_start array of
    n_clusters + 1 ints, list of the per-cluster Systems)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_min, n_max + 1, size=n_clusters)
    seeds = rng.integers(0, 2**31 - 1, size=n_clusters)
    parts = [make_cluster(int(n), seed=int(s)) for n, s in zip(sizes, seeds)]
    start = np.zeros(n_clusters + 1, dtype=np.int32)
    start[1:] = np.cumsum(sizes)
    allsys = System(pos=np.concatenate([c.pos for c in parts]), mp_local=np.concatenate([c.mp_local for c in parts]),
                    box=None, meta={"kind": "cluster_batch", "n_clusters": n_clusters, "seed": seed})
    return allsys, start, parts
