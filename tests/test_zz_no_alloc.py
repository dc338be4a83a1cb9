"""The allocation-free cluster electrostatics entry point.

Some callers cannot let the library allocate device memory: engines whose
memory pool or arena owns every device byte, and MD plugins whose force
callbacks may not call cudaMalloc (an allocation can synchronize the device
and stall the host engine's other streams).  sibfa_cluster_elec_noalloc keeps
its scratch in a fixed device array.  These tests call it through the C ABI:
twice in a row against the elec and pen energies of the regular entry point
(sibfa_energy_forces, FP64 path) on the same cluster; at the largest accepted
size (512 waters, the scratch array filled to its end) against the oracle's
pair sums; around a call, the device memory in use stays the same; host
buffers and buffers of the wrong length are refused before any launch.  The
file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from gpu_util import FP64_E_REL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()
    return torch


def _call(pos, mp, stream=None):
    from paper_2201_00804_gb300.sibfa import sibfa_cluster_elec_noalloc
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    sibfa_cluster_elec_noalloc(synth.PARAMS, pos, mp, out, stream=stream)
    return out


def test_noalloc_matches_energy_forces_twice(torch_cuda):
    import paper_2201_00804_gb300 as pkg

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
        stream = torch.cuda.current_stream()
        out = _call(pos, mp, stream=stream)
        stream.synchronize()
        elec, pen = out.cpu().tolist()
        assert abs(elec - ref["elec"]) < FP64_E_REL * scale, (call, elec, ref["elec"])
        assert abs(pen - ref["pen"]) < FP64_E_REL * scale, (call, pen, ref["pen"])


def test_noalloc_largest_cluster_matches_oracle_and_allocates_nothing(torch_cuda):
    """512 waters fill the scratch array to its end.  The regular context does
    not take a single 512-molecule cluster (its neighbour slots hold 384), so
    the reference is the oracle's multipole and penetration pair sums."""
    from oracle import core, terms

    s = synth.make_cluster(512, seed=78)
    S = core.build_sites(torch.tensor(s.pos, dtype=torch.float64), torch.tensor(s.mp_local, dtype=torch.float64),
                         synth.PARAMS)
    i, j, sh = terms.mol_pairs(s.pos[:, 0], None, None)
    e_ref, p_ref = 0.0, 0.0
    for a in range(0, i.size, 4096):
        e, p = terms.elec_pen_pairs(S, i[a:a + 4096], j[a:a + 4096], torch.tensor(sh[a:a + 4096]), synth.PARAMS,
                                    None, None)
        e_ref += float(e)
        p_ref += float(p)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    mp = torch.tensor(s.mp_local.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    from paper_2201_00804_gb300.sibfa import sibfa_cluster_elec_noalloc
    sibfa_cluster_elec_noalloc(synth.PARAMS, pos, mp, out)      # first call: scratch address, module load
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    for _ in range(2):
        sibfa_cluster_elec_noalloc(synth.PARAMS, pos, mp, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == used0
    assert free1 == free0, (free0, free1)
    elec, pen = out.cpu().tolist()
    scale = abs(e_ref) + abs(p_ref)
    assert abs(elec - e_ref) < FP64_E_REL * scale, (elec, e_ref)
    assert abs(pen - p_ref) < FP64_E_REL * scale, (pen, p_ref)


def test_noalloc_rejects_oversized_cluster(torch_cuda):
    from paper_2201_00804_gb300.sibfa import SibfaError

    n = 513
    pos = torch.zeros(n * 9, dtype=torch.float64, device="cuda")
    mp = torch.zeros(n * 50, dtype=torch.float64, device="cuda")
    with pytest.raises(SibfaError, match="exceeds the maximum"):
        _call(pos, mp)


def test_noalloc_rejects_host_and_short_buffers(torch_cuda):
    """The binding refuses CPU arrays and a short mp_local; the C entry point
    itself refuses host addresses (cudaPointerGetAttributes) before any launch."""
    from paper_2201_00804_gb300 import sibfa

    s = synth.make_cluster(4, seed=79)
    pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
    mp = torch.tensor(s.mp_local.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        sibfa.sibfa_cluster_elec_noalloc(synth.PARAMS, np.ascontiguousarray(s.pos.reshape(-1)), mp, out)
    with pytest.raises(ValueError):
        sibfa.sibfa_cluster_elec_noalloc(synth.PARAMS, pos, mp[:-50], out)
    lib = sibfa.load_library()
    P = sibfa.sibfa_params(*[float(synth.PARAMS[n]) for n in sibfa.PARAM_FIELDS])
    host_pos = np.ascontiguousarray(s.pos.reshape(-1))
    host_out = np.zeros(2)
    st = lib.sibfa_cluster_elec_noalloc(ctypes.byref(P), 4, host_pos.ctypes.data, mp.data_ptr(), out.data_ptr(),
                                        None)
    assert st == -1 and b"pos" in lib.sibfa_noalloc_last_error()
    st = lib.sibfa_cluster_elec_noalloc(ctypes.byref(P), 4, pos.data_ptr(), mp.data_ptr(), host_out.ctypes.data,
                                        None)
    assert st == -1 and b"elec_pen" in lib.sibfa_noalloc_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0     # nothing was launched
