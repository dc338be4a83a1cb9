"""The allocation-free cluster electrostatics entry point.

Callers such as memory-pool-owned engines, MD plugins whose force callbacks
may not call cudaMalloc, or code recorded into CUDA graphs cannot let the
library allocate.  sibfa_cluster_elec_noalloc keeps its scratch in a fixed
device array; this test calls it through the C ABI twice in a row and checks
both results against the elec and pen energies of the regular entry point
(sibfa_energy_forces, FP64 path) on the same cluster.  The file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import synth
from gpu_util import FP64_E_REL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()
    return torch


def test_noalloc_matches_energy_forces_twice(torch_cuda):
    torch = torch_cuda
    import paper_2201_00804_gb300 as pkg
    from paper_2201_00804_gb300.sibfa import sibfa_cluster_elec_noalloc

    s = synth.make_cluster(24, seed=77)
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, periodic=False, precision=pkg.PREC_FP64, pcg_tol_D=1e-10)
    try:
        ref = pkg.sibfa_energy_forces(ctx, np.ascontiguousarray(s.pos.reshape(-1)))
    finally:
        pkg.sibfa_destroy(ctx)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    mp = torch.tensor(s.mp_local.reshape(-1), dtype=torch.float64, device="cuda")
    scale = abs(ref["elec"]) + abs(ref["pen"])
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        sibfa_cluster_elec_noalloc(synth.PARAMS, pos, mp, out, stream=stream)
        stream.synchronize()
        elec, pen = out.cpu().tolist()
        assert abs(elec - ref["elec"]) < FP64_E_REL * scale, (call, elec, ref["elec"])
        assert abs(pen - ref["pen"]) < FP64_E_REL * scale, (call, pen, ref["pen"])


def test_noalloc_rejects_oversized_cluster(torch_cuda):
    torch = torch_cuda
    from paper_2201_00804_gb300.sibfa import SibfaError, sibfa_cluster_elec_noalloc

    n = 513
    pos = torch.zeros(n * 9, dtype=torch.float64, device="cuda")
    mp = torch.zeros(n * 50, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(SibfaError, match="exceeds the maximum"):
        sibfa_cluster_elec_noalloc(synth.PARAMS, pos, mp, out)
