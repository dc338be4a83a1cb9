"""Serving (sibfa_server_*): jobs that arrive together share the device (box
jobs in concurrent slots, gas-phase clusters continuously batched), and each
result is the same as the job run alone through a plain context, within the
mixed-precision tolerance; a full queue answers BUSY instead of blocking."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TERMS = ("elec", "pen", "rep", "disp", "xdisp", "pol", "ct")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00804_gb300 import build
    build.build()


def _alone(job):
    """The job through a plain context: n_steps velocity-Verlet steps (or one evaluation)."""
    import torch
    import paper_2201_00804_gb300 as pkg
    s = job["sys"]
    kw = dict(periodic=job["periodic"], precision=pkg.PREC_MIXED, pcg_tol_D=1e-6, warm_start=True)
    if job["periodic"]:
        kw.update(box=s.box, rc=job["rc"], grid=job["grid"], ewald_alpha=job["alpha"])
    ctx = pkg.sibfa_create(synth.PARAMS, s.mp_local, **kw)
    try:
        pos = torch.tensor(s.pos.reshape(-1), dtype=torch.float64, device="cuda")
        if job["n_steps"] == 0:
            F = torch.zeros_like(pos)
            terms = pkg.sibfa_energy_forces(ctx, pos, F)
        else:
            vel = torch.tensor(job["vel"].reshape(-1), dtype=torch.float64, device="cuda")
            m = torch.tensor(s.masses().reshape(-1), dtype=torch.float64, device="cuda")
            terms = pkg.sibfa_md_steps(ctx, pos, vel, m, 0.5, job["n_steps"])
        torch.cuda.synchronize()
        return terms, pos.cpu().numpy()
    finally:
        pkg.sibfa_destroy(ctx)


def _wait(srv, tickets, timeout=300.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "jobs did not finish"
        time.sleep(0.002)
    return out


def test_results_alone_equal_in_the_mix():
    import paper_2201_00804_gb300 as pkg
    jobs = []
    # the first cluster runs alone in the batch for a while; the others join
    # later, so the batch grows between steps
    for k, n in enumerate((2, 7, 12, 20, 31, 5)):
        s = synth.make_cluster(n, seed=300 + k)
        jobs.append(dict(sys=s, periodic=False, n_steps=40 if k == 0 else (0 if k == 5 else 3 + k % 3),
                         vel=synth.maxwell_velocities(s, 300.0, seed=k)))
    s, o = synth.make_config("water216")
    jobs.append(dict(sys=s, periodic=True, rc=o["rc"], grid=o["grid"], alpha=o["ewald"], n_steps=3,
                     vel=synth.maxwell_velocities(s, 300.0, seed=9)))
    s2 = synth.make_box(6, 18.62, seed=11)
    jobs.append(dict(sys=s2, periodic=True, rc=7.0, grid=24, alpha=0.4, n_steps=0, vel=np.zeros_like(s2.pos)))
    srv = pkg.Server(synth.PARAMS, slots=2, batch_waters=512, precision=pkg.PREC_MIXED)
    try:
        tickets = []
        for n, j in enumerate(jobs):
            if n == 1:
                time.sleep(0.3)
            s = j["sys"]
            kw = dict(periodic=j["periodic"], n_steps=j["n_steps"], vel=j["vel"], dt_fs=0.5)
            if j["periodic"]:
                kw.update(box=s.box, rc=j["rc"], grid=j["grid"], ewald_alpha=j["alpha"])
            tickets.append(srv.submit(s.pos, s.mp_local, **kw))
        res = _wait(srv, tickets)
    finally:
        srv.close()
    for j, t in zip(jobs, tickets):
        r = res[t]
        assert r["status"] == 0
        assert r["batched"] == (not j["periodic"])
        terms, pos = _alone(j)
        mag = sum(abs(terms[k]) for k in TERMS)
        for k in TERMS:
            assert abs(r["terms"][k] - terms[k]) <= 1e-6 * mag, (k, r["terms"][k], terms[k])
        assert np.abs(r["pos"] - pos).max() <= 1e-6
        assert r["latency_ms"] >= r["queue_ms"] >= 0.0


def test_slot_context_cache_with_eviction():
    """One box slot and five box shapes (the same 216 waters on five grid
    sizes), submitted as 1, 2, 3, 1, 4, 5, 1: the slot keeps four contexts,
    so shape 1 comes back from its cache once and, after shapes 4 and 5, is
    rebuilt once its context has been evicted as the least recently used;
    every result equals the job run alone."""
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    grids = (24, 25, 27, 30, 32)
    order = (0, 1, 2, 0, 3, 4, 0)
    jobs = []
    for k, g in enumerate(order):
        sk = synth.System(pos=s.pos + 0.01 * k, mp_local=s.mp_local, box=s.box)
        jobs.append(dict(sys=sk, periodic=True, rc=o["rc"], grid=grids[g], alpha=o["ewald"], n_steps=k % 2 * 2,
                         vel=synth.maxwell_velocities(sk, 300.0, seed=40 + k)))
    srv = pkg.Server(synth.PARAMS, slots=1, batch_waters=0, precision=pkg.PREC_MIXED)
    try:
        tickets, res = [], {}
        for j in jobs:
            sk = j["sys"]
            t = srv.submit(sk.pos, sk.mp_local, periodic=True, n_steps=j["n_steps"], vel=j["vel"], dt_fs=0.5,
                           box=sk.box, rc=j["rc"], grid=j["grid"], ewald_alpha=j["alpha"])
            tickets.append(t)
            res.update(_wait(srv, [t]))    # one at a time: the submission order is the run order
    finally:
        srv.close()
    for j, t in zip(jobs, tickets):
        r = res[t]
        assert r["status"] == 0
        terms, pos = _alone(j)
        mag = sum(abs(terms[k]) for k in TERMS)
        for k in TERMS:
            assert abs(r["terms"][k] - terms[k]) <= 1e-6 * mag, (k, r["terms"][k], terms[k])
        assert np.abs(r["pos"] - pos).max() <= 1e-6


def test_full_queue_answers_busy():
    import paper_2201_00804_gb300 as pkg
    s, o = synth.make_config("water216")
    srv = pkg.Server(synth.PARAMS, slots=1, max_pending=2, batch_waters=0, precision=pkg.PREC_MIXED)
    try:
        tickets = [srv.submit(s.pos, s.mp_local, periodic=True, box=s.box, rc=o["rc"], grid=o["grid"],
                              ewald_alpha=o["ewald"], n_steps=5) for _ in range(12)]
        assert any(t is None for t in tickets)
        _wait(srv, [t for t in tickets if t is not None])
    finally:
        srv.close()
