"""The library's FP32 elementary kernels against CUDA's functions and against
the exact values, over the ranges the pair kernels use:

- the Newton-refined reciprocal square root (squared distances 1e-2..1e4 A^2)
  within 2 ulp of 1/sqrt(x), no worse than rsqrtf;
- the Newton-refined reciprocal (|x| in 1e-4..1e4) within 2 ulp of 1/x, the
  IEEE division being correctly rounded;
- the erf(alpha r)/r radial kernels g_0..g_3 of the intramolecular Ewald
  exclusions (r 0.05..4 A, alpha 0.4..0.9, across the switch between the
  Maclaurin series and the erfc difference at (alpha r)^2 = 2) within
  relative bounds of the exact derivatives, taken with mpmath at 40 digits
  by numerical differentiation of erf(alpha r)/r, and g_0 within a few ulp of
  erff(alpha r)/r."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()
    return torch


def ulp_err(y, ref):
    """|y - ref| in units of the float32 spacing at ref."""
    ref32 = ref.astype(np.float32)
    sp = np.spacing(np.abs(ref32)).astype(np.float64)
    return np.abs(y.astype(np.float64) - ref) / sp


def test_reciprocal_square_root(torch_cuda):
    torch = torch_cuda
    from paper_2201_00804_gb300.sibfa import sibfa_math_selftest
    x = np.exp(np.random.default_rng(1).uniform(np.log(1e-2), np.log(1e4), 1 << 20)).astype(np.float32)
    out = sibfa_math_selftest(0, torch.tensor(x, device="cuda")).cpu().numpy()
    ref = 1.0 / np.sqrt(x.astype(np.float64))
    ours, cuda = ulp_err(out[:, 0], ref), ulp_err(out[:, 1], ref)
    assert ours.max() <= 2.0, ours.max()
    assert ours.max() <= max(cuda.max(), 1.0), (ours.max(), cuda.max())


def test_reciprocal(torch_cuda):
    torch = torch_cuda
    from paper_2201_00804_gb300.sibfa import sibfa_math_selftest
    rng = np.random.default_rng(2)
    x = (np.exp(rng.uniform(np.log(1e-4), np.log(1e4), 1 << 20)) * rng.choice([-1.0, 1.0], 1 << 20)).astype(np.float32)
    out = sibfa_math_selftest(1, torch.tensor(x, device="cuda")).cpu().numpy()
    ref = 1.0 / x.astype(np.float64)
    ours, ieee = ulp_err(out[:, 0], ref), ulp_err(out[:, 1], ref)
    assert ieee.max() <= 0.5 + 1e-9, ieee.max()
    assert ours.max() <= 2.0, ours.max()


def _erf_kernels_exact(r, alpha):
    import mpmath as mp
    mp.mp.dps = 40
    a = mp.mpf(float(alpha))
    f = lambda t: mp.erf(a * t) / t  # noqa: E731
    t = mp.mpf(float(r))
    d1, d2, d3 = (mp.diff(f, t, k) for k in (1, 2, 3))
    g0 = f(t)
    g1 = d1 / t
    g2 = d2 / t ** 2 - d1 / t ** 3
    g3 = d3 / t ** 3 - 3 * d2 / t ** 4 + 3 * d1 / t ** 5
    return [float(g0), float(g1), float(g2), float(g3)]


@pytest.mark.parametrize("alpha", [0.4, 0.55, 0.9])
def test_erf_radial_kernels(torch_cuda, alpha):
    pytest.importorskip("mpmath")
    torch = torch_cuda
    from paper_2201_00804_gb300.sibfa import sibfa_math_selftest
    r = np.concatenate([np.linspace(0.05, 4.0, 160), [np.sqrt(2.0) / alpha * (1 + e) for e in (-1e-6, 0, 1e-6)]])
    r = r.astype(np.float32)
    out = sibfa_math_selftest(2, torch.tensor(r, device="cuda"), alpha).cpu().numpy().astype(np.float64)
    ref = np.array([_erf_kernels_exact(v, alpha) for v in r])
    rel = np.abs(out[:, :4] - ref) / np.abs(ref)
    # g_0: a few ulp; higher kernels: the recursion adds a few roundings each
    assert rel[:, 0].max() < 5e-7, rel[:, 0].max()
    for n, bound in ((1, 2e-6), (2, 4e-6), (3, 8e-6)):
        assert rel[:, n].max() < bound, (n, rel[:, n].max(), r[rel[:, n].argmax()])
    cuda_rel = np.abs(out[:, 4] - ref[:, 0]) / np.abs(ref[:, 0])
    assert (np.abs(out[:, 0] - out[:, 4]) / np.abs(ref[:, 0])).max() < 1e-6
    assert rel[:, 0].max() <= max(cuda_rel.max(), 2.4e-7) * 2
