"""Full-size parity: the 4096-water box (rc 9 A, SPME 64^3) and the
32,000-water box (rc 9 A, SPME 108^3) in the launch configuration the
benchmark times (mixed precision, PCG 1e-6 D) against the oracle's stored
results (tests/golden/<box>_oracle.npz, written by
tests/golden/make_golden.py): every energy term and the forces and induced
dipoles of a seeded sample of 256 molecules; and the FP64 path at a tight
solver tolerance."""
import os

import numpy as np
import pytest

import synth
from gpu_util import MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D, TERMS, run_gpu

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", params=["water4096", "water32000"])
def gold(request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()
    g = np.load(os.path.join(GOLDEN, f"{request.param}_oracle.npz"))
    names = [str(x) for x in g["term_names"]]
    return {"name": request.param, "terms": dict(zip(names, g["terms"])), "sample": g["sample"],
            "forces": g["forces"], "mu": g["mu"]}


def _check(gpu, gold, e_rel, f_rel, mu_d):
    rt, gt = gold["terms"], gpu["terms"]
    scale = sum(abs(rt[k]) for k in TERMS)
    for k in TERMS:
        assert abs(gt[k] - rt[k]) < e_rel * scale, (k, gt[k], rt[k])
    assert abs(gt["total"] - rt["total"]) < e_rel * abs(rt["total"]), (gt["total"], rt["total"])
    Fs = gpu["forces"][gold["sample"]]
    ferr = np.sqrt(np.mean((Fs - gold["forces"]) ** 2) / np.mean(gold["forces"] ** 2))
    assert ferr < f_rel, ferr
    dmu = (gpu["mu"][gold["sample"]] - gold["mu"]).reshape(-1, 3) * 4.80321
    mu_err = np.sqrt((dmu ** 2).sum(-1).mean())
    assert mu_err < mu_d, mu_err


def test_mixed_bench_configuration(gold):
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config(gold["name"])
    gpu = run_gpu(s, o, pkg.PREC_MIXED, o["pcg_tol"])
    _check(gpu, gold, MIXED_E_REL, MIXED_F_RMS_REL, MIXED_MU_RMS_D)


def test_fp64_path(gold):
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config(gold["name"])
    gpu = run_gpu(s, o, pkg.PREC_FP64, 1e-10)
    _check(gpu, gold, 1e-9, 1e-8, 1e-8)
