"""Unit counting behind the bench's roofline lines: bench.count_units (a
k-d-tree molecule-pair walk with the O-O minimum image, as the kernels'
neighbour list) equals a brute-force count over every ordered molecule pair
and every point pair with the minimum image taken on the point-point
displacement itself, on the 216-water box at rc 7 A; the cluster counts are
all pairs of each cluster; the per-kernel flops are the per-unit figures
times those counts."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def brute_force(pts, box, rc):
    """pts: (M, 7, 3) O, H1, H2, M1, M2, LP1, LP2."""
    M = pts.shape[0]
    L = np.asarray(box)
    n = dict(site_pairs=0, lp_pairs=0, rep_items=0, rep_bb=0, rep_bl=0, rep_lb=0, rep_ll=0, disp_items=0,
             ct_items=0)

    def cnt(A, B):
        d = A[:, None, :] - B[None, :, :]
        d -= L * np.round(d / L)
        return int((np.sqrt((d * d).sum(-1)) < rc).sum())

    mids = 0.5 * (pts[:, 0:1] + pts[:, 1:3])
    for i in range(M):
        for j in range(M):
            if i == j:
                continue
            n["site_pairs"] += cnt(pts[i, :5], pts[j, :5])
            n["lp_pairs"] += cnt(pts[i, 5:7], pts[j, :5])
            if j > i:
                n["rep_bb"] += cnt(mids[i], mids[j])
                n["rep_bl"] += cnt(mids[i], pts[j, 5:7])
                n["rep_lb"] += cnt(pts[i, 5:7], mids[j])
                n["rep_ll"] += cnt(pts[i, 5:7], pts[j, 5:7])
                q = [0, 1, 2, 5, 6]
                n["disp_items"] += cnt(pts[i, q], pts[j, q])
                n["ct_items"] += 8 * cnt(pts[i, 0:1], pts[j, 0:1])
    n["rep_items"] = n["rep_bb"] + n["rep_bl"] + n["rep_lb"] + n["rep_ll"]
    return n


def test_count_units_equals_brute_force():
    s, o = synth.make_config("water216")
    pts = bench.points_from_pos(s.pos, synth.PARAMS)
    got = bench.count_units(s.pos, s.box, o["rc"], pts)
    ref = brute_force(pts, s.box, o["rc"])
    assert got == ref
    assert ref["site_pairs"] > 0 and ref["rep_items"] > 0 and ref["ct_items"] > 0
    fl = bench.kernel_flops(got)
    assert fl["real_perm"] == got["site_pairs"] * bench.FLOPS_PERM_SITE_PAIR
    assert fl["short"] == (850 * got["rep_bb"] + 455 * (got["rep_bl"] + got["rep_lb"]) + 220 * got["rep_ll"]
                           + 70 * got["disp_items"])
    assert fl["ct"] == got["ct_items"] * bench.FLOPS_CT_ITEM


def test_cluster_counts_are_all_pairs():
    start = np.array([0, 2, 5, 9])
    n = bench.count_units_clusters(start, 9)
    pairs = 1 + 3 + 6                       # unordered molecule pairs of clusters of 2, 3, 4
    assert n == dict(site_pairs=2 * 25 * pairs, lp_pairs=2 * 10 * pairs, rep_items=16 * pairs, rep_bb=4 * pairs,
                     rep_bl=4 * pairs, rep_lb=4 * pairs, rep_ll=4 * pairs, disp_items=25 * pairs, ct_items=8 * pairs)


def test_spme_pass_bytes():
    assert bench.spme_pass_bytes((64, 64, 64), 20480) == 56 * 64 ** 3 + 144 * 20480
