"""Unit counting behind the bench's roofline line: bench.count_units (a
molecule-list walk with the O-O minimum image, as the kernel does) equals a
brute-force count over every ordered molecule pair and every point pair
with the minimum image taken on the point-point displacement itself, on the
216-water box at rc 7 A; and the per-launch flops are the per-unit figures
times those counts."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def brute_force(pts, box, rc):
    M = pts.shape[0]
    L = np.asarray(box)
    atom = np.array([1, 1, 1, 0, 0], bool)
    n = dict(site_pairs=0, pen_atom_atom=0, pen_atom_mid=0, pen_mid_atom=0, thole_pairs=0, lp_pairs=0)
    sites, lps = pts[:, :5], pts[:, 5:7]
    for i in range(M):
        others = np.arange(M) != i
        d = sites[others][None, :, :, :] - sites[i][:, None, None, :]      # (5, M-1, 5, 3)
        d -= L * np.round(d / L)
        inr = np.sqrt((d * d).sum(-1)) < rc
        n["site_pairs"] += int(inr.sum())
        n["pen_atom_atom"] += int(inr[atom][:, :, atom].sum())
        n["pen_atom_mid"] += int(inr[atom][:, :, ~atom].sum())
        n["pen_mid_atom"] += int(inr[~atom][:, :, atom].sum())
        n["thole_pairs"] += int(inr[:3].sum())
        dl = sites[others][None, :, :, :] - lps[i][:, None, None, :]
        dl -= L * np.round(dl / L)
        n["lp_pairs"] += int((np.sqrt((dl * dl).sum(-1)) < rc).sum())
    return n


def test_count_units_equals_brute_force():
    s, o = synth.make_config("water216")
    pts = bench.points_from_pos(s.pos, synth.PARAMS)
    got = bench.count_units(s.pos, s.box, o["rc"], pts)
    ref = brute_force(pts, s.box, o["rc"])
    assert got == ref
    assert ref["site_pairs"] > 0 and ref["pen_mid_atom"] == ref["pen_atom_mid"]
    flops = bench.unit_flops(got)
    assert flops == (got["site_pairs"] * bench.FLOPS_PERM_SITE_PAIR + got["pen_atom_atom"] * bench.FLOPS_PEN_ATOM_ATOM
                     + got["pen_atom_mid"] * bench.FLOPS_PEN_ATOM_MID + got["pen_mid_atom"] * bench.FLOPS_PEN_MID_ATOM
                     + got["thole_pairs"] * bench.FLOPS_THOLE_PAIR)


def test_cluster_counts_are_all_ordered_pairs():
    start = np.array([0, 2, 5, 9])
    n = bench.count_units_clusters(start, 9)
    pairs = 2 * 1 + 3 * 2 + 4 * 3
    assert n["site_pairs"] == 25 * pairs and n["thole_pairs"] == 15 * pairs and n["lp_pairs"] == 10 * pairs
