#!/usr/bin/env python
"""SIBFA energy + force benchmark on one GB300 (or N independent replicas).

Default workload: the 32,000-water box (96,000 atoms, 98.6 A, rc 9 A, SPME
108^3 order 5, alpha 0.4 A^-1), mixed precision (FP32 pair and grid
arithmetic, FP64 accumulation and solver scalars), PCG tolerance 1e-6 D
with warm start (by default the initial guess extrapolates the dipoles of
the last five steps, a quartic; --warm-start 1 takes the previous step's),
velocity-Verlet NVE at 0.5 fs from 300 K after an untimed relaxation and
velocity-rescaled equilibration; the plain FP64 GPU path is timed on the
same workload.  --workload water4096 (4096 waters, 49.66 A, SPME 64^3),
clusters4096 and served select the other workloads.  A step is one
velocity-Verlet step: one full energy + force evaluation (sites, neighbour
list, real-space pair terms, SPME, charge transfer, polarization solve,
forces) plus the two half kicks.  Metric: atom-steps/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun with N ranks every rank runs its own replica (weak scaling;
the method has no cross-replica exchange), rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s SIBFA E+F (SPME+pol) vs FP64 GPU path; served p50/p99 latency"
UNIT = "atom-steps/s"
WORKLOAD = ("water4096: 4096 rigid-geometry waters (12,288 atoms), cubic box 49.66 A, rc 9 A, SPME 64^3 order 5, "
            "alpha 0.4/A, PCG 1e-6 D warm start, velocity-Verlet NVE 0.5 fs from 300 K")
SAMPLE = ("oracle sample: 512 waters (1,536 atoms) at the same density, rc 9 A, SPME 32^3 (1.29 points/A, as 64^3 "
          "on 49.66 A) order 5, alpha 0.4, PCG 1e-6 D; one full energy + force evaluation per step")
# Algorithmic FP32 work per unit (fused multiply-add = 2, a transcendental or
# reciprocal square root = 1), energy and full gradient of one unordered unit:
# multipole site pair with Ewald kernel, energy, gradient, torque, field and
# penetration 300 (the middle of the 250-350 estimate); charge-transfer
# donor-acceptor pair 100.  Repulsion and dispersion are counted from their
# formulas (Technical Appendix): one atom pair of an overlap (two cosines,
# the s/p overlap, two exponentials, and their gradients at the four points)
# is 63 + 125 flops; a bond-bond item has four atom pairs plus the midpoint
# distance, the S^2/R and S^2/R^2 energy and the gradient assembly (850);
# bond-lone pair and lone pair-bond items two atom pairs (455); lone
# pair-lone pair one overlap with two cosines (220); a dispersion point pair
# the C6/C8/C10 damped terms and exchange-dispersion with their radial
# derivative (70).
FLOPS_PERM_SITE_PAIR = 300
FLOPS_REP = {"rep_bb": 850, "rep_bl": 455, "rep_lb": 455, "rep_ll": 220}
FLOPS_DISP_ITEM = 70
FLOPS_CT_ITEM = 100


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip timing the FP64 GPU path")
    ap.add_argument("--warm-start", type=int, default=5, choices=[1, 2, 3, 4, 5, 6],
                    help="PCG initial guess along the trajectory: 1 previous dipoles, 2-6 extrapolation through "
                         "the last 2-6 steps' dipoles")
    ap.add_argument("--workload", default="water32000",
                    choices=["water216", "water4096", "water32000", "water216_paper", "clusters4096", "served"])
    ap.add_argument("--equil-steps", type=int, default=600,
                    help="untimed velocity-rescaled MD steps (300 K) after the relaxation, before the NVE steps")
    ap.add_argument("--rates", default="20,50,100", help="served: arrival rates (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=6.0, help="served: arrival window per rate (s)")
    ap.add_argument("--ct-original", action="store_true",
                    help="the original many-body charge transfer instead of the reduced one")
    ap.add_argument("--npt-steps", type=int, default=1000,
                    help="water4096, water216_paper: untimed constant-pressure steps after the timed ones (0: none)")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="reference arm: host threads for the oracle (0: PyTorch's default, all cores)")
    ap.add_argument("--served-fp64", action="store_true",
                    help="served: also run the same mix through the FP64 path at the highest rate")
    return ap.parse_args()


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def unordered_pairs(O, box, cut):
    """Unordered molecule pairs (i < j) whose minimum-image O-O distance is
    below `cut`, with the image shift to add to molecule j's points."""
    from scipy.spatial import cKDTree
    L = np.asarray(box, dtype=np.float64)
    Ow = np.mod(O, L)
    pr = cKDTree(Ow, boxsize=L).query_pairs(cut, output_type="ndarray")
    if pr.size == 0:
        return np.zeros((0,), np.int64), np.zeros((0,), np.int64), np.zeros((0, 3))
    i, j = pr[:, 0], pr[:, 1]
    d = O[j] - O[i]
    sh = -L * np.round(d / L)
    return i, j, sh


def count_units(pos, box, rc, pts):
    """Algorithmic units of one evaluation's real-space kernels, with each
    kernel's cutoff semantics (per point pair, on the distance of the term's
    radial factor):
      site_pairs  ordered (target site, source site) pairs within rc: the
                  permanent kernel evaluates every pair from both sides
                  (target-site formulation: energy, gradient, torque and
                  field of the target);
      lp_pairs    ordered (lone pair, source site) pairs within rc;
      rep_items   unordered repulsion orbital pairs within rc, and by class:
                  rep_bb bond-bond (bond midpoints), rep_bl and rep_lb
                  bond-lone pair and lone pair-bond (midpoint to lone pair),
                  rep_ll lone pair-lone pair;
      disp_items  unordered (point, point) dispersion pairs within rc over
                  O, H1, H2, LP1, LP2;
      ct_items    unordered donor-acceptor pairs: 8 per molecule pair whose
                  O-O distance is below rc.
    pts: (M, 7, 3) absolute O, H1, H2, M1, M2, LP1, LP2."""
    O = pos[:, 0]
    i, j, sh = unordered_pairs(O, box, rc + 2.6)
    n = dict(site_pairs=0, lp_pairs=0, rep_items=0, rep_bb=0, rep_bl=0, rep_lb=0, rep_ll=0, disp_items=0,
             ct_items=0)
    rc2 = rc * rc
    for a in range(0, i.size, 65536):
        ii, jj, ss = i[a:a + 65536], j[a:a + 65536], sh[a:a + 65536]
        Pi, Pj = pts[ii], pts[jj] + ss[:, None, :]

        def within(A, B):
            d = A[:, :, None, :] - B[:, None, :, :]
            return np.einsum("nabk,nabk->nab", d, d) < rc2

        ss_ = within(Pi[:, :5], Pj[:, :5])
        n["site_pairs"] += 2 * int(ss_.sum())
        n["lp_pairs"] += int(within(Pi[:, 5:7], Pj[:, :5]).sum() + within(Pj[:, 5:7], Pi[:, :5]).sum())
        mi = 0.5 * (Pi[:, 0:1] + Pi[:, 1:3])            # bond midpoints (n, 2, 3)
        mj = 0.5 * (Pj[:, 0:1] + Pj[:, 1:3])
        li, lj = Pi[:, 5:7], Pj[:, 5:7]
        cls = {"rep_bb": int(within(mi, mj).sum()), "rep_bl": int(within(mi, lj).sum()),
               "rep_lb": int(within(li, mj).sum()), "rep_ll": int(within(li, lj).sum())}
        for k, v in cls.items():
            n[k] += v
        n["rep_items"] += sum(cls.values())
        qi = np.concatenate([Pi[:, :3], li], 1)
        qj = np.concatenate([Pj[:, :3], lj], 1)
        n["disp_items"] += int(within(qi, qj).sum())
        dO = Pj[:, 0] - Pi[:, 0]
        n["ct_items"] += 8 * int((np.einsum("nk,nk->n", dO, dO) < rc2).sum())
    return n


def count_units_clusters(start, M):
    """The same units for a batch of gas-phase clusters (all pairs inside each
    cluster, no cutoff)."""
    n = np.diff(np.asarray(start, dtype=np.int64))
    pairs = int((n * (n - 1) // 2).sum())           # unordered molecule pairs
    return dict(site_pairs=2 * 25 * pairs, lp_pairs=2 * 10 * pairs, rep_items=16 * pairs, rep_bb=4 * pairs,
                rep_bl=4 * pairs, rep_lb=4 * pairs, rep_ll=4 * pairs, disp_items=25 * pairs, ct_items=8 * pairs)


def kernel_flops(n):
    """Algorithmic FP32 flops per launch set, from the per-unit figures above."""
    return {"real_perm": n["site_pairs"] * FLOPS_PERM_SITE_PAIR,
            "short": sum(n[k] * f for k, f in FLOPS_REP.items()) + n["disp_items"] * FLOPS_DISP_ITEM,
            "ct": n["ct_items"] * FLOPS_CT_ITEM}


def spme_pass_bytes(K, n_sites):
    """Algorithmic bytes of one SPME pass over a grid of G = K0 K1 K2 points:
    spread write 4G, forward FFT read + write ~12G, convolution read + write
    16G, influence function read 4G (FP64 on the half spectrum), inverse FFT
    ~12G, gather read 4G (56 G in all), plus 64 B read and 80 B written per
    site (multipole in, potential derivatives out)."""
    G = int(np.prod(K))
    return 56 * G + 144 * n_sites


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def measured_traffic(kernel_key, workload):
    """DRAM bytes (read + write) per step of a kernel from the committed ncu
    summary, or None when its source changed after the counters were taken or
    none were taken for this workload."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)[workload][kernel_key]
    except (OSError, ValueError, KeyError):
        return None
    h = hashlib.sha256()
    for p in rec.get("sources", []):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec.get("dram_bytes_per_step")


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def measure_fp32_peak(pkg, local):
    """FP32 FMA rate of this GPU: a kernel of independent FMA chains on every
    SM (8 blocks of 256 threads per SM, ~20 ms per launch), best of five,
    with the SM clock sampled meanwhile.  The number of SMs is the device's."""
    import torch
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    best = 0.0
    with Clocks(local) as clk:
        for _ in range(5):
            fl, ms = pkg.sibfa_alu_peak(False, 16384, 8 * nsm)
            best = max(best, fl / (ms * 1e-3) / 1e12)
    c = clk.summary()
    return {"tflops": best, "sms": nsm, "sm_mhz": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"],
            "basis": ("measured: FP32 FMA-chain kernel on all %d SMs, best of 5 launches (%.1f TFLOP/s at a median "
                      "%s MHz SM clock)" % (nsm, best, c["sm_mhz"]))}


def points_from_pos(pos, P):
    """Absolute site and lone-pair positions (for counting units only)."""
    O, H1, H2 = pos[:, 0], pos[:, 1], pos[:, 2]
    u1 = (H1 - O) / np.linalg.norm(H1 - O, axis=-1, keepdims=True)
    u2 = (H2 - O) / np.linalg.norm(H2 - O, axis=-1, keepdims=True)
    z = u1 + u2
    z /= np.linalg.norm(z, axis=-1, keepdims=True)
    x = (H1 - O) - ((H1 - O) * z).sum(-1, keepdims=True) * z
    x /= np.linalg.norm(x, axis=-1, keepdims=True)
    y = np.cross(z, x)
    th = math.radians(P["lp_half_deg"])
    d = P["d_lp"]
    lp1 = O + d * (-math.cos(th) * z + math.sin(th) * y)
    lp2 = O + d * (-math.cos(th) * z - math.sin(th) * y)
    return np.stack([O, H1, H2, 0.5 * (O + H1), 0.5 * (O + H2), lp1, lp2], 1)


def dist_setup():
    """Process group of a torchrun launch (NCCL on GPUs; gloo without CUDA,
    for the host-side tests of the multi-rank logic)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, rank, ws
    return None, 0, 1


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    """The slowest rank's time (the job's time)."""
    if dist is None:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(ws, atoms_per_rank, step_ms):
    """Whole-job atom-steps/s: every rank advances its own replica of
    atoms_per_rank atoms by one step in step_ms (the slowest rank's time)."""
    return ws * atoms_per_rank / (step_ms / 1000.0)


def sample_system():
    import synth
    s = synth.make_box(8, 24.83, seed=2)
    return s, {"rc": 9.0, "grid": 32, "order": 5, "ewald": 0.4}


def cpu_baseline(steps=1, workload=None):
    """The oracle on the host cores: the whole 216-water box (one evaluation
    at its PCG tolerance), else the 512-water sample of the large boxes."""
    import torch
    import oracle
    if workload == "water216":
        import synth
        s, o = synth.make_config("water216")
        tol, sample = o["pcg_tol"], "the whole 216-water box; one full energy + force evaluation per step"
    else:
        (s, o), tol, sample = sample_system(), 1e-6, SAMPLE
    t = time.perf_counter()
    for _ in range(steps):
        oracle.evaluate(s, o, tol_D=tol)
    dt = time.perf_counter() - t
    return {"value": s.n_atoms * steps / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": sample, "seconds": dt}


def run_reference(args, dist, rank, ws):
    if rank != 0:
        return
    import torch
    import oracle
    if args.cpu_threads > 0:
        torch.set_num_threads(args.cpu_threads)
    s, o = sample_system()
    for _ in range(args.warmup):
        oracle.evaluate(s, o, tol_D=1e-6)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.evaluate(s, o, tol_D=1e-6)
    dt = time.perf_counter() - t
    v = s.n_atoms * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS.get(args.workload, WORKLOAD), "sample": SAMPLE},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": SAMPLE},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The paper's MD setting (Computational Details; intramolecular potential of
# its flexible water): Beeman at 1 fs, MM3-style anharmonic bond and angle
# with a Urey-Bradley H-H term about 0.9572 A, 108.5 deg and 1.5326 A, and
# the dispersion beyond the 7 A cutoff as a homogeneous-fluid tail (the
# paper's 20 A dispersion cutoff exceeds half of the 18.643 A box).
PAPER_MD = dict(md_integrator="beeman", md_anharmonic=True, md_k_ub=38.25, md_r_ub=1.5326, md_theta0_deg=108.5,
                disp_tail=True)

WORKLOADS = {
    "water4096": WORKLOAD,
    "water32000": ("water32000: 32,000 rigid-geometry waters (96,000 atoms; 32^3 lattice, 768 seeded removals), cubic "
                   "box 98.6 A, rc 9 A, SPME 108^3 order 5, alpha 0.4/A, PCG 1e-6 D warm start, velocity-Verlet NVE "
                   "0.5 fs from 300 K"),
    "water216": ("water216: 216 rigid-geometry waters (648 atoms), cubic box 18.62 A, rc 7 A, SPME 24^3 order 5, "
                 "alpha 0.4/A, PCG 1e-8 D warm start, velocity-Verlet NVE 0.5 fs from 300 K"),
    "water216_paper": ("water216_paper: the paper's MD setting, 216 waters (648 atoms) in an 18.643 A box, SPME "
                       "120^3 order 5, Ewald and repulsion cutoff 7 A with the dispersion beyond it as a "
                       "homogeneous-fluid tail, PCG 1e-5 D warm start, Beeman NVE at 1 fs with MM3-style anharmonic "
                       "bond/angle and Urey-Bradley support terms"),
    "clusters4096": ("clusters4096: 4096 independent gas-phase water clusters, sizes uniform in 2-32 (70,240 waters, "
                     "210,720 atoms), all pairs within each cluster, no cutoff or Ewald, one context and one launch "
                     "per kernel, PCG 1e-6 D per cluster with warm start, velocity-Verlet NVE 0.5 fs from 300 K"),
}


GUESS = {1: "previous step's dipoles", 2: "linear extrapolation of the last 2 steps' dipoles",
         3: "quadratic extrapolation of the last 3 steps' dipoles",
         4: "cubic extrapolation of the last 4 steps' dipoles",
         5: "quartic extrapolation of the last 5 steps' dipoles",
         6: "quintic extrapolation of the last 6 steps' dipoles"}


def setup(name, pkg, synth, precision, stream, warm=1, ct_original=False):
    """Context, device arrays and unit counts of a workload."""
    import torch
    if name in ("water216", "water4096", "water32000", "water216_paper"):
        s, o = synth.make_config(name)
        extra = dict(PAPER_MD) if name == "water216_paper" else {}
        if ct_original:
            extra["ct_original"] = True
        ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                               ewald_alpha=o["ewald"], pcg_tol_D=o["pcg_tol"], precision=precision,
                               warm_start=warm, stream=stream, **extra)
        make_api = lambda: pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=True, box=s.box, rc=o["rc"],  # noqa: E731
                                            grid=o["grid"], ewald_alpha=o["ewald"], pcg_tol_D=o["pcg_tol"],
                                            precision=precision, warm_start=warm, stream=stream, **extra)
        seed = {"water216": 1, "water4096": 2, "water32000": 3, "water216_paper": 1}[name]
    else:
        s, start, _ = synth.make_cluster_batch(4096, seed=4)
        o = {"rc": None, "cluster_start": start}
        ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=False, pcg_tol_D=1e-6, precision=precision,
                               warm_start=warm, stream=stream, cluster_start=start, ct_original=ct_original)
        make_api = lambda: pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=False, pcg_tol_D=1e-6,  # noqa: E731
                                            precision=precision, warm_start=warm, stream=stream,
                                            cluster_start=start, ct_original=ct_original)
        seed = 4
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    vel = torch.tensor(synth.maxwell_velocities(s, 300.0, seed=seed).reshape(-1), dtype=torch.float64, device="cuda")
    masses = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
    return s, o, ctx, make_api, pos, vel, masses


KB_KCAL = 0.0019872041          # kcal/(mol K)
AMU_A2_FS2 = 4.184e-4           # kcal/mol per amu A^2/fs^2


def kinetic(vel, masses3):
    """Kinetic energy (kcal/mol) of device velocities (A/fs)."""
    return 0.5 * float((masses3 * vel * vel).sum()) / AMU_A2_FS2


def intra_energy(pos, **support):
    return float(intra_energy_t(pos, **support))


def intra_energy_t(pos, k_bond=529.6, r0=0.9572, k_angle=34.05, theta0_deg=104.52, md_anharmonic=False,
                   md_k_ub=0.0, md_r_ub=1.5326, **_):
    """The MD driver's intramolecular support potential (kcal/mol) at device
    positions, as the run options define it: k_bond dr^2 per O-H bond and
    k_angle dth^2 per H-O-H angle, with the MM3-style anharmonic factors and
    the Urey-Bradley H-H term when asked."""
    import torch
    x = pos.reshape(-1, 3, 3)
    b1, b2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    r1, r2 = b1.norm(dim=-1), b2.norm(dim=-1)
    dth = torch.acos(((b1 * b2).sum(-1) / (r1 * r2)).clamp(-1.0, 1.0)) - math.radians(theta0_deg)

    def bond(dr):
        return k_bond * dr ** 2 * ((1 - 2.55 * dr + (7.0 / 12.0) * 2.55 ** 2 * dr ** 2) if md_anharmonic else 1.0)

    D = dth * (180.0 / math.pi)
    ang = k_angle * dth ** 2 * ((1 - 0.014 * D + 5.6e-5 * D ** 2 - 7e-7 * D ** 3 + 9e-10 * D ** 4)
                                if md_anharmonic else 1.0)
    e = bond(r1 - r0) + bond(r2 - r0) + ang
    if md_k_ub > 0:
        e = e + md_k_ub * ((x[:, 1] - x[:, 2]).norm(dim=-1) - md_r_ub) ** 2
    return e.sum()


BAR_PER_KCAL_MOL_A3 = 69476.95    # 1 kcal/mol/A^3 in bar


def intra_virial(pos, **support):
    """W_ab = -dE/d eps_ab of the support potential under x -> (I + eps) x."""
    import torch
    eps = torch.zeros((3, 3), dtype=torch.float64, device=pos.device, requires_grad=True)
    x = pos.detach().reshape(-1, 3) @ (torch.eye(3, dtype=torch.float64, device=pos.device) + eps).T
    g, = torch.autograd.grad(intra_energy_t(x, **support), [eps])
    return -g.cpu().numpy()


def berendsen_npt(pkg, ctx, pos, vel, masses, box, n_steps, every=10, dt_fs=1.0, p_bar=1.0, tau_ps=1.0,
                  kappa_per_bar=4.5e-5, support=None, min_half_box=0.0):
    """Constant pressure by Berendsen's weak coupling: MD steps in chunks of
    `every`; after each chunk the pressure P = (2 K + tr W) / (3 V) from the
    kinetic energy, the library's virial (with the dispersion tail) and the
    support potential's virial, then all atoms and the box scaled by
    mu = [1 - kappa (every dt / tau) (p_bar - P)]^(1/3) (clamped to 1 +/- 1%);
    the scaled box reaches the context through a dipole solve at the scaled
    positions before the next chunk.  The run stops early, flagged, when the
    scaled box would leave less than min_half_box in its half (the cutoff plus
    twice the site extent must fit).  Returns the box, the volumes and the
    pressures after each chunk."""
    import torch
    support = support or {}
    m3 = masses.repeat_interleave(3)
    box = np.asarray(box, dtype=np.float64).copy()
    F = torch.zeros_like(pos)
    vols, press = [], []
    stopped = None
    for chunk in range(n_steps // every):
        pkg.sibfa_md_steps(ctx, pos, vel, masses, dt_fs, every)
        W = np.zeros((3, 3))
        pkg.sibfa_energy_forces(ctx, pos, F, box=box, virial=W)
        W = W + intra_virial(pos, **support)
        V = float(np.prod(box))
        P = (2.0 * kinetic(vel, m3) + np.trace(W)) / (3.0 * V) * BAR_PER_KCAL_MOL_A3
        mu = (1.0 - kappa_per_bar * (every * dt_fs * 1e-3 / tau_ps) * (p_bar - P)) ** (1.0 / 3.0)
        mu = min(1.01, max(0.99, mu))
        if 0.5 * float(np.min(box)) * mu < min_half_box:
            stopped = (chunk + 1) * every
            press.append(P)
            break
        box *= mu
        pos.mul_(mu)
        pkg.sibfa_solve_dipoles(ctx, pos, None, 0.0, box=box)
        vols.append(float(np.prod(box)))
        press.append(P)
    return {"box": box, "volumes": vols, "pressure_bar": np.array(press), "stopped_at_step": stopped}


def equilibrate(pkg, ctx, pos, vel, masses, n_min=20, n_thermo=200, temp=300.0, every=5, dt_fs=0.5):
    """Untimed preparation of an MD workload from its random starting
    structure: capped steepest descent, then velocity-Verlet steps with the
    velocities rescaled to `temp` every `every` steps, which removes the heat
    that the relaxation of the lattice releases."""
    m3 = masses.repeat_interleave(3)
    ndof = vel.numel() - 3
    pkg.sibfa_minimize(ctx, pos, n_min, 0.01)
    for _ in range(n_thermo // every):
        pkg.sibfa_md_steps(ctx, pos, vel, masses, dt_fs, every)
        T = 2.0 * kinetic(vel, m3) / (ndof * KB_KCAL)
        vel.mul_(math.sqrt(temp / T))
    return 2.0 * kinetic(vel, m3) / (ndof * KB_KCAL)


PHASES = ("sites", "neighbors", "real_perm", "short", "spme_perm", "ct", "pcg", "real_tmu", "real_polforce",
          "spme_polforce", "finalize")


def read_phases(pkg, ctx, steps):
    out = {}
    for name in PHASES:
        ms, n = pkg.sibfa_profile_get(ctx, name)
        out[name] = {"ms_per_step": ms / steps, "launches": n}
    return out


def timed_steps(pkg, ctx, pos, vel, masses, steps, stream, flush, dt_fs=0.5, keep=False, energy=False, support=None):
    """steps velocity-Verlet steps, each timed with CUDA events on the
    caller's stream after an L2 flush; returns (ms total, iterations,
    snapshots, total energies).  With energy=True the total energy (kinetic +
    intermolecular + intramolecular support) after each step is recorded,
    outside the timed span."""
    import torch
    m3 = masses.repeat_interleave(3)
    total, iters, snaps, etot = 0.0, [], [], []
    for _ in range(steps):
        flush.zero_()                       # evict L2 (512 MB > 129 MB) before every timed step
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e = pkg.sibfa_md_steps(ctx, pos, vel, masses, dt_fs, 1)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
        iters.append(pkg.sibfa_last_stats(ctx)[0])
        if keep:
            snaps.append(pos.clone())
        if energy:
            etot.append(kinetic(vel, m3) + e["total"] + intra_energy(pos, **(support or {})))
    return total, iters, snaps, etot


def smooth235(n):
    """Smallest 2,3,5-smooth integer >= n."""
    k = int(math.ceil(n))
    while True:
        m = k
        for f in (2, 3, 5):
            while m % f == 0:
                m //= f
        if m == 1:
            return k
        k += 1


def served_pool(synth, rng):
    """Seeded job inputs for the served stream: gas-phase clusters (2-32
    waters) and periodic boxes (216-8192 waters at 29.915 A^3 per water,
    grid the smallest 2,3,5-smooth size >= 1.3 points/A, rc 9 A or, in boxes
    too small for it, half the box minus the neighbour-list margin)."""
    clusters = [synth.make_cluster(int(n), seed=5000 + k) for k, n in enumerate(rng.integers(2, 33, size=64))]
    boxes = []
    for k, n in enumerate((216, 512, 1000, 2048, 4096, 8192)):
        side = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
        L = (n * 29.915) ** (1.0 / 3.0)
        s = synth.make_box(side, L, seed=6000 + k, n_remove=side ** 3 - n)
        rc = min(9.0, 0.5 * L - 2.7)
        boxes.append((s, dict(rc=rc, grid=smooth235(1.3 * L), ewald=0.4)))
    return clusters, boxes


def run_served(args, pkg, synth, precision=None, rates=None):
    """Poisson arrivals at each rate for a fixed window; 70% clusters, 30%
    boxes, 1-50 MD steps per job; latency = completion - arrival.  A rate the
    server cannot keep up with is drained for at most 20 s after the window;
    jobs still running then are reported as unfinished and their work is not
    counted."""
    import torch
    rng = np.random.default_rng(5)
    clusters, boxes = served_pool(synth, rng)
    vel_c = [synth.maxwell_velocities(c, 300.0, seed=k) for k, c in enumerate(clusters)]
    vel_b = [synth.maxwell_velocities(b[0], 300.0, seed=k) for k, b in enumerate(boxes)]
    out = []
    precision = pkg.PREC_MIXED if precision is None else precision
    for rate in rates or [float(r) for r in args.rates.split(",")]:
        srv = pkg.Server(synth.PARAMS, slots=3, device_mem_bytes=64 << 30, max_pending=100000, batch_waters=16384,
                         precision=precision, pcg_tol_D=1e-6)
        # warm the server: one job of every box shape and one cluster, untimed
        warm = [srv.submit(b[0].pos, b[0].mp_local, periodic=True, box=b[0].box, rc=b[1]["rc"], grid=b[1]["grid"],
                           ewald_alpha=b[1]["ewald"], n_steps=1) for b in boxes]
        warm.append(srv.submit(clusters[0].pos, clusters[0].mp_local, n_steps=1))
        pending = set(warm)
        while pending:
            pending = {t for t in pending if srv.poll(t) is None}
            time.sleep(0.001)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * args.serve_seconds * 2) + 10))
        arrivals = arrivals[arrivals < args.serve_seconds]
        kinds = rng.random(arrivals.size) < 0.7
        steps = rng.integers(1, 51, size=arrivals.size)
        which = rng.integers(0, 1 << 30, size=arrivals.size)
        t0 = time.perf_counter()
        live, lat, atom_steps, busy, nxt = {}, [], 0, 0, 0
        last_done = t0
        deadline = args.serve_seconds + 20.0     # a stream that cannot drain is reported, not waited for
        while (nxt < arrivals.size or live) and time.perf_counter() - t0 < deadline:
            now = time.perf_counter() - t0
            while nxt < arrivals.size and arrivals[nxt] <= now:
                if kinds[nxt]:
                    c = clusters[which[nxt] % len(clusters)]
                    v = vel_c[which[nxt] % len(clusters)]
                    t = srv.submit(c.pos, c.mp_local, vel=v, n_steps=int(steps[nxt]))
                    n_at = 3 * c.n_mol
                else:
                    b, o = boxes[which[nxt] % len(boxes)]
                    v = vel_b[which[nxt] % len(boxes)]
                    t = srv.submit(b.pos, b.mp_local, vel=v, periodic=True, box=b.box, rc=o["rc"], grid=o["grid"],
                                   ewald_alpha=o["ewald"], n_steps=int(steps[nxt]))
                    n_at = 3 * b.n_mol
                if t is None:
                    busy += 1
                else:
                    live[t] = (arrivals[nxt], n_at * int(steps[nxt]))
                nxt += 1
            for t in list(live):
                r = srv.poll(t)
                if r is not None:
                    arr, work = live.pop(t)
                    done = time.perf_counter()
                    lat.append((done - t0 - arr) * 1e3)
                    if r["status"] == 0:
                        atom_steps += work
                    last_done = done
            time.sleep(0.0005)
        wall = last_done - t0
        srv.close()
        lat = np.array(lat)
        out.append({"rate_per_s": rate, "precision": "fp64" if precision == pkg.PREC_FP64 else "mixed",
                    "jobs": int(lat.size), "busy_refused": busy, "unfinished": len(live),
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "atom_steps_per_s": atom_steps / wall, "wall_s": wall})
        print(json.dumps({"served_rate": out[-1]}), file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    return out


def main():
    args = parse()
    dist, rank, ws = dist_setup()
    if args.impl == "reference":
        run_reference(args, dist, rank, ws)
        return
    if args.workload == "served":
        import synth
        import paper_2201_00804_gb300 as pkg
        from paper_2201_00804_gb300 import build
        build.build()
        res = run_served(args, pkg, synth)
        # the same mix through the plain FP64 path, at the highest rate (saturated)
        res64 = run_served(args, pkg, synth, precision=pkg.PREC_FP64,
                           rates=[max(float(r) for r in args.rates.split(","))]) if args.served_fp64 else None
        best = max(res, key=lambda r: r["atom_steps_per_s"])
        line = {"metric": METRIC, "value": best["atom_steps_per_s"], "unit": UNIT, "n_gpus": 1,
                "steps": int(sum(r["jobs"] for r in res)), "warmup": 1, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "served: Poisson arrivals, 70% gas-phase clusters (2-32 waters), 30% "
                                       "periodic boxes (216-8192 waters, 1.3 grid points/A), 1-50 velocity-Verlet "
                                       "steps per job, mixed precision, PCG 1e-6 D",
                           "window_s_per_rate": args.serve_seconds},
                "served": res, "served_fp64_path": res64}
        print(json.dumps(line), flush=True)
        return
    import torch

    import synth
    import paper_2201_00804_gb300 as pkg
    from paper_2201_00804_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    s, o, ctx, make_api, pos, vel, masses = setup(args.workload, pkg, synth, pkg.PREC_MIXED, stream, args.warm_start,
                                                  args.ct_original)
    M = s.n_mol
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    # The random starting structures are far from equilibrium: relax them and
    # equilibrate at 300 K first (untimed), then warm up in NVE.
    dt = 1.0 if args.workload == "water216_paper" else 0.5
    support = PAPER_MD if args.workload == "water216_paper" else None
    if support:
        support = dict(support, theta0_deg=support["md_theta0_deg"])
    t_equil = equilibrate(pkg, ctx, pos, vel, masses, n_min=20, n_thermo=args.equil_steps, dt_fs=dt)
    pos0, vel0 = pos.clone(), vel.clone()
    for _ in range(max(3, args.warmup)):
        pkg.sibfa_md_steps(ctx, pos, vel, masses, dt, 1)
    torch.cuda.synchronize()
    l0 = pkg.sibfa_kernel_launches(ctx)
    barrier(dist)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        total_ms, iters, snapshots, etot = timed_steps(pkg, ctx, pos, vel, masses, args.steps, stream, flush,
                                                       dt_fs=dt, keep=True, energy=True, support=support)
    torch.cuda.synchronize()
    barrier(dist)
    launches = pkg.sibfa_kernel_launches(ctx) - l0
    tb, tjoin, tdone, tms = pkg.sibfa_tuned_schedule(ctx)
    # Phase spans of the overlapped schedule, after the timed region (the
    # per-phase events cost about 1% of a step, so the timed steps run
    # without them): CUDA events around each phase on its own stream.
    n_live = min(10, args.steps)
    pkg.sibfa_set_profiling(ctx, True)
    pkg.sibfa_profile_clear(ctx)
    timed_steps(pkg, ctx, pos, vel, masses, n_live, stream, flush, dt_fs=dt, support=support)
    phases = read_phases(pkg, ctx, n_live)
    # Serial pass (after the timed region, same trajectory): every phase alone
    # on the GPU, so a phase's span is its kernels' own duration.  In the
    # timed steps the short-range and charge-transfer kernels share the SMs
    # with the solve from lower-priority streams and their spans include the
    # waits.
    n_serial = 3
    pkg.sibfa_set_profiling(ctx, 2)
    pkg.sibfa_profile_clear(ctx)
    _, iters_serial, _, _ = timed_steps(pkg, ctx, pos, vel, masses, n_serial, stream, flush, dt_fs=dt)
    phases_serial = read_phases(pkg, ctx, n_serial)
    pkg.sibfa_set_profiling(ctx, False)
    peak = measure_fp32_peak(pkg, local)
    step_ms = max_over_ranks(dist, total_ms) / args.steps
    value = weak_value(ws, 3 * M, step_ms)

    # Rooflines.  Pair kernels: algorithmic FP32 flops per step (unit counts
    # x per-unit figures) over the kernel's CUDA-event time on the stream it
    # runs on in the serial pass, against the FP32 FMA rate measured on this
    # device; the same over its span in the timed steps is reported as
    # achieved_live.  SPME: the permanent pass's algorithmic bytes over its
    # serial event time, against the measured HBM copy bandwidth.
    P = synth.PARAMS
    pos_h = pos.cpu().numpy().reshape(M, 3, 3)
    if args.workload in ("water216", "water4096", "water32000", "water216_paper"):
        units = count_units(pos_h, s.box, o["rc"], points_from_pos(pos_h, P))
    else:
        units = count_units_clusters(o["cluster_start"], M)
    kfl = kernel_flops(units)
    kernels = {"real_perm": ("k_real_perm<float, %d, 0, 0, 5, 0>" % int(args.workload != "clusters4096"),
                             "site targets: multipole + penetration energy, gradient, torque sensitivities, "
                             "Thole field; 1 launch per step"),
               "short": ("k_short<float, %d, 0, 0|1>" % int(args.workload != "clusters4096"),
                         "repulsion (part 0) and dispersion + exchange-dispersion (part 1); 2 launches per step, "
                         "timed together"),
               "ct": ("k_ct<float, %d, 0>" % int(args.workload != "clusters4096"),
                      "reduced charge transfer; 1 launch per step")}
    lines = {}
    for key, (kname, what) in kernels.items():
        ms, ms_live = phases_serial[key]["ms_per_step"], phases[key]["ms_per_step"]
        if ms <= 0:
            continue
        ach = kfl[key] / (ms * 1e-3) / 1e12
        ach_live = kfl[key] / (ms_live * 1e-3) / 1e12 if ms_live > 0 else None
        lines[key] = {"bound": "alu", "kernel": kname, "what": what, "achieved": ach, "peak": peak["tflops"],
                      "unit": "TFLOP/s", "frac": ach / peak["tflops"], "flops_per_step": kfl[key],
                      "ms_per_step": ms, "timing": "serial pass, kernel alone on the GPU",
                      "achieved_live": ach_live, "frac_live": ach_live / peak["tflops"] if ach_live else None,
                      "ms_per_step_live": ms_live, "traffic": measured_traffic(key, args.workload)}
    if args.workload != "clusters4096":
        K = o["grid"] if not np.isscalar(o["grid"]) else (o["grid"],) * 3
        nbytes = spme_pass_bytes(K, 5 * M)
        ms = phases_serial["spme_perm"]["ms_per_step"]
        hbm = measured_hbm_peak()
        lines["spme_perm"] = {"bound": "hbm", "kernel": "spme permanent pass (spread, cuFFT r2c, convolution, "
                              "cuFFT c2r, gather to 3rd derivatives, intramolecular corrections)",
                              "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "bytes_per_pass": nbytes, "ms_per_step": ms,
                              "timing": "serial pass", "ms_per_step_live": phases["spme_perm"]["ms_per_step"],
                              "traffic": None, "peak_basis": "hbm_gbs of MEASURED_PEAKS.json (copy bandwidth)"}
        it = float(np.mean(iters_serial))
        pcg_ms = phases_serial["pcg"]["ms_per_step"]
        lines["pcg_iteration"] = {"bound": "hbm", "kernel": "one PCG iteration (real-space T.p from the pair list, "
                                  "SPME of the direction, cooperative vector step)",
                                  "achieved": nbytes / (pcg_ms / (it + 1) * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": nbytes / (pcg_ms / (it + 1) * 1e-3) / 1e9 / hbm,
                                  "ms_per_iteration": pcg_ms / (it + 1), "iterations_per_step": it,
                                  "bytes_per_iteration_spme": nbytes, "timing": "serial pass (device loop, the solve alone on the GPU)",
                                  "traffic": None}
    dom = max(("real_perm", "short"), key=lambda k: lines[k]["ms_per_step"] if k in lines else -1)
    roofline = dict(lines[dom])
    roofline["peak_basis"] = peak["basis"]
    roofline["units"] = units
    # End to end through the C ABI with host buffers: a second context
    # evaluates, from pinned host memory, the positions of the trajectory that
    # the first context advances on the device (untimed); each timed call
    # copies the positions in and the forces and energies out.
    api = make_api()
    F_host = torch.zeros(M * 9, dtype=torch.float64).pin_memory()
    hosts = [snap.cpu().pin_memory() for snap in snapshots]
    # untimed: the new context's schedule tuning (its first full evaluations)
    for k in range(32):
        pkg.sibfa_energy_forces(api, hosts[k % len(hosts)], F_host)
        if pkg.sibfa_tuned_shape(api)[1]:
            break
    pkg.sibfa_energy_forces(api, hosts[0], F_host)
    e2e_s = 0.0
    for pos_host in hosts:
        t = time.perf_counter()
        pkg.sibfa_energy_forces(api, pos_host, F_host)
        e2e_s += time.perf_counter() - t
    e2e_s = max_over_ranks(dist, e2e_s)
    e2e = {"value": ws * 3 * M * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(hosts[0].numel() * 8), "host_memory": "pinned",
           "d2h_bytes_per_step": int(F_host.numel() * 8 + 8 * 8 + 4)}
    pkg.sibfa_destroy(api)
    # The paper's setting runs at constant pressure: an untimed Berendsen
    # stretch (1 bar, tau 1 ps, water's compressibility, pressure every 10
    # steps) after the timed steps, reported as the density it reaches (the
    # 4096-water box and the paper's 216-water setting).
    npt = None
    if args.workload in ("water4096", "water216_paper") and args.npt_steps > 0 and not args.ct_original:
        # the box may not shrink below what the cutoff and the largest site
        # extent the library accepts (1.3 A) need
        out = berendsen_npt(pkg, ctx, pos, vel, masses, s.box, n_steps=args.npt_steps, every=10, dt_fs=dt,
                            support=support, min_half_box=o["rc"] + 2.6)
        vols, pr = np.array(out["volumes"] or [float(np.prod(s.box))]), out["pressure_bar"]
        grams = M * 18.01528 / 0.602214076          # g per mol of waters / (A^3 -> cm^3 * N_A)
        half = len(vols) // 2
        npt = {"steps": args.npt_steps, "barostat": "Berendsen, 1 bar, tau 1 ps, kappa 4.5e-5/bar, every 10 steps",
               "density_start_g_cm3": grams / float(np.prod(s.box)), "density_end_g_cm3": grams / vols[-1],
               "density_mean_second_half_g_cm3": float(np.mean(grams / vols[half:])),
               "pressure_mean_second_half_bar": float(np.mean(pr[half:])),
               "pressure_first_last_bar": [float(pr[0]), float(pr[-1])],
               "box_end_A": [float(b) for b in out["box"]],
               "stopped_at_step": out["stopped_at_step"]}
        if out["stopped_at_step"] is not None:
            npt["note"] = ("stopped where the box would shrink below 2 (rc + 2.6 A), the room the cutoff and the "
                           "largest site extent need: at 1 bar the synthetic table's liquid is denser than this "
                           "box and cutoff allow")
    pkg.sibfa_destroy(ctx)

    # The plain FP64 GPU path on the same workload and starting state (the
    # comparison the metric names): a few steps, same timing method.
    fp64 = None
    if not args.no_fp64_path:
        _, _, c64, _, p64, v64, m64 = setup(args.workload, pkg, synth, pkg.PREC_FP64, stream, args.warm_start,
                                            args.ct_original)
        p64.copy_(pos0)
        v64.copy_(vel0)
        # untimed: warm-up steps, and steps until the context's schedule tuning
        # (its first full evaluations) has fixed a candidate
        for k in range(40):
            pkg.sibfa_md_steps(c64, p64, v64, m64, dt, 1)
            if k >= 1 and pkg.sibfa_tuned_shape(c64)[1]:
                break
        torch.cuda.synchronize()
        n64 = 10
        ms64, it64, _, _ = timed_steps(pkg, c64, p64, v64, m64, n64, stream, flush, dt_fs=dt)
        ms64 = max_over_ranks(dist, ms64) / n64
        pkg.sibfa_destroy(c64)
        fp64 = {"value": ws * 3 * M / (ms64 / 1000.0), "unit": UNIT, "ms_per_step": ms64, "steps": n64,
                "pcg_iters_mean": float(np.mean(it64)), "speedup_of_mixed": ms64 / step_ms}

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline and args.workload in ("water216", "water4096", "water32000"):
        cpu = cpu_baseline(workload=args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "FP32 pair/grid arithmetic, FP64 accumulation",
                   "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{ws}",
                   "pcg_initial_guess": GUESS[args.warm_start],
                   "charge_transfer": ("original many-body form (acceptor potentials kept)" if args.ct_original
                                       else "reduced form (Eqs. 13-16)")},
        "clocks": clk.summary(), "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
        "rooflines": lines, "fp32_peak": peak,
        "cpu_baseline": cpu, "fp64_gpu_path": fp64, "pcg_iters_mean": float(np.mean(iters)), "phases_ms": phases,
        "phases_ms_serial": phases_serial,
        "nve": {"equilibration": f"20 capped steepest-descent steps, {args.equil_steps} velocity-rescaled steps at "
                                 f"300 K (T after: {t_equil:.1f} K), {max(3, args.warmup)} NVE warm-up steps",
                "total_energy_first": etot[0], "total_energy_last": etot[-1],
                "drift_kcal_per_mol_atom_per_ps": (etot[-1] - etot[0]) / (3 * M) / (dt * 1e-3 * max(1, len(etot) - 1)),
                "temperature_end_K": 2.0 * kinetic(vel, masses.repeat_interleave(3)) / ((vel.numel() - 3) * KB_KCAL)},
        "tuned": {"short_blocks_per_sm": tb, "short_joined_before_solve": tjoin, "fixed": tdone,
                  "candidates_ms": {f"{c}{'+join' if j else ''}": round(t, 4)
                                    for (c, j), t in zip(((3, 0), (0, 0), (2, 0), (0, 1), (3, 1)), tms)}},
        "npt": npt,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
