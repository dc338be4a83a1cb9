"""Oracle pins for polarization: T is symmetric positive definite, the PCG
solution equals a dense solve of the explicit T, the converged residual is
below 1e-10 D, and E_pol = 1/2 mu T mu - mu E = -1/2 mu E at the solution."""
import numpy as np
import torch

import oracle
import synth

DT = torch.float64


def _dense_T(ops, M):
    n = M * 9
    T = np.zeros((n, n))
    for k in range(n):
        e = torch.zeros(n, dtype=DT)
        e[k] = 1.0
        T[:, k] = ops["matvec"](e.reshape(M, 3, 3)).reshape(-1).numpy()
    return T


def _check(system, opts):
    out = oracle.evaluate(system, opts, forces=False, tol_D=1e-11, keep_operators=True)
    ops = out["pol_ops"]
    M = system.n_mol
    T = _dense_T(ops, M)
    np.testing.assert_allclose(T, T.T, atol=1e-11 * np.abs(T).max())
    assert np.linalg.eigvalsh(0.5 * (T + T.T)).min() > 0
    E = out["efield"].reshape(-1)
    mu_dense = np.linalg.solve(T, E)
    dmu = (out["mu"].reshape(-1) - mu_dense) * 4.80321
    assert np.sqrt((dmu.reshape(-1, 3) ** 2).sum(-1).mean()) < 1e-9
    assert out["resid_D"] < 1e-10
    ke = 332.063713
    e_half = -0.5 * ke * float(out["mu"].reshape(-1) @ E)
    assert abs(out["terms"]["pol"] - e_half) < 1e-12 * abs(e_half)
    e_func = ke * ops["functional"](torch.tensor(out["mu"], dtype=DT))
    assert abs(e_func - e_half) < 1e-9 * abs(e_half)


def test_pcg_matches_dense_gas():
    _check(synth.make_cluster(6, seed=4), None)


def test_pcg_matches_dense_periodic():
    s = synth.make_box(2, 8.0, seed=9, jitter=0.3)
    _check(s, {"rc": 3.2, "grid": 16, "order": 5, "ewald": 0.8})
