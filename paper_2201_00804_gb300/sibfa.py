"""Thin ctypes binding of the SIBFA C ABI (include/sibfa.h).

Argument marshalling only: every step of an evaluation runs in the CUDA
library.  Arrays may be torch tensors (host or CUDA) or numpy arrays; they
must be float64 and contiguous.  The functions keep the C names.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsibfa.so")

PARAM_FIELDS = (
    "ke debye d_lp lp_half_deg alpha_o alpha_h alpha_m_damp thole z_o z_h b_o b_h "
    "cs_o cp_o cs_h cp_h cs_lp cp_lp g_o g_h nval_o nval_h "
    "rvdw_rep_o rvdw_rep_h rvdw_rep_lp rep_alpha rep_alpha2 rep_c1 rep_c2 rep_f occ_bond n_lp "
    "rvdw_disp_o rvdw_disp_h rvdw_disp_lp disp_alpha beta_o beta_h c6 c8 c10 gamma6 gamma8 gamma10 disp_delta "
    "xd_c1 xd_a1 xd_c2 xd_a2 xd_c3 xd_a3 ct_eta ct_t ct_m ct_ae ct_ah rvdw_ct_o rvdw_ct_h"
).split()
TERMS = ("elec", "pen", "rep", "disp", "xdisp", "pol", "ct", "total")

SIBFA_OK = 0
STATUS = {0: "OK", -1: "INVALID", -2: "OOM", -3: "NOT_CONVERGED", -4: "CUTOFF", -5: "CT_DENOM",
          -6: "TIMEOUT", -7: "CUDA", -8: "BUSY", -9: "NEIGHBOR"}
PREC_FP64, PREC_MIXED = 0, 1


class sibfa_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in PARAM_FIELDS]


class sibfa_topology(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("mp_local", C.POINTER(C.c_double)), ("n_clusters", C.c_int),
                ("cluster_start", C.POINTER(C.c_int))]


class sibfa_run_opts(C.Structure):
    _fields_ = [("periodic", C.c_int), ("box", C.c_double * 3), ("rc", C.c_double), ("grid", C.c_int * 3),
                ("order", C.c_int), ("ewald_alpha", C.c_double), ("pcg_tol_D", C.c_double),
                ("pcg_max_iter", C.c_int), ("precision", C.c_int), ("warm_start", C.c_int),
                ("stream", C.c_void_p), ("md_k_bond", C.c_double), ("md_r0", C.c_double),
                ("md_k_angle", C.c_double), ("md_theta0_deg", C.c_double), ("disp_tail", C.c_int),
                ("md_integrator", C.c_int), ("md_anharmonic", C.c_int), ("md_k_ub", C.c_double),
                ("md_r_ub", C.c_double), ("ct_original", C.c_int)]


class sibfa_energy_terms(C.Structure):
    _fields_ = [(n, C.c_double) for n in TERMS]


class sibfa_server_opts(C.Structure):
    _fields_ = [("params", C.POINTER(sibfa_params)), ("slots", C.c_int), ("device_mem_bytes", C.c_size_t),
                ("max_pending", C.c_int), ("batch_waters", C.c_int), ("batch_max_cluster", C.c_int),
                ("batch_dt_fs", C.c_double), ("precision", C.c_int), ("pcg_tol_D", C.c_double)]


class sibfa_job(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("pos", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
                ("mp_local", C.POINTER(C.c_double)), ("periodic", C.c_int), ("box", C.c_double * 3),
                ("rc", C.c_double), ("grid", C.c_int * 3), ("ewald_alpha", C.c_double), ("n_steps", C.c_int),
                ("dt_fs", C.c_double)]


class sibfa_result(C.Structure):
    _fields_ = [("terms", sibfa_energy_terms), ("forces", C.POINTER(C.c_double)), ("pos", C.POINTER(C.c_double)),
                ("status", C.c_int), ("pcg_iters", C.c_int), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("batched", C.c_int)]


class SibfaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsibfa.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it first (paper_2201_00804_gb300.build.build())")
    lib = C.CDLL(path)
    lib.sibfa_create.argtypes = [C.POINTER(sibfa_params), C.POINTER(sibfa_topology), C.POINTER(sibfa_run_opts),
                                 C.POINTER(C.c_void_p)]
    lib.sibfa_create.restype = C.c_int
    lib.sibfa_energy_forces.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(sibfa_energy_terms),
                                        C.c_void_p, C.c_void_p]
    lib.sibfa_energy_forces.restype = C.c_int
    lib.sibfa_solve_dipoles.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                        C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.sibfa_solve_dipoles.restype = C.c_int
    lib.sibfa_md_steps.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                   C.POINTER(sibfa_energy_terms)]
    lib.sibfa_md_steps.restype = C.c_int
    lib.sibfa_minimize.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(sibfa_energy_terms)]
    lib.sibfa_minimize.restype = C.c_int
    lib.sibfa_last_stats.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.sibfa_last_stats.restype = C.c_int
    lib.sibfa_cluster_terms.argtypes = [C.c_void_p, C.POINTER(sibfa_energy_terms)]
    lib.sibfa_cluster_terms.restype = C.c_int
    lib.sibfa_server_create.argtypes = [C.POINTER(sibfa_server_opts), C.POINTER(C.c_void_p)]
    lib.sibfa_server_create.restype = C.c_int
    lib.sibfa_submit.argtypes = [C.c_void_p, C.POINTER(sibfa_job), C.POINTER(C.c_uint64)]
    lib.sibfa_submit.restype = C.c_int
    lib.sibfa_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(sibfa_result), C.POINTER(C.c_int)]
    lib.sibfa_poll.restype = C.c_int
    lib.sibfa_server_destroy.argtypes = [C.c_void_p]
    lib.sibfa_server_destroy.restype = None
    lib.sibfa_kernel_launches.argtypes = [C.c_void_p]
    lib.sibfa_kernel_launches.restype = C.c_uint64
    lib.sibfa_tuned_shape.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.sibfa_tuned_shape.restype = C.c_int
    lib.sibfa_tuned_schedule.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_double), C.c_int]
    lib.sibfa_tuned_schedule.restype = C.c_int
    lib.sibfa_set_profiling.argtypes = [C.c_void_p, C.c_int]
    lib.sibfa_set_profiling.restype = None
    lib.sibfa_profile_get.argtypes = [C.c_void_p, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.sibfa_profile_get.restype = C.c_int
    lib.sibfa_profile_clear.argtypes = [C.c_void_p]
    lib.sibfa_profile_clear.restype = None
    lib.sibfa_cluster_elec_noalloc.argtypes = [C.POINTER(sibfa_params), C.c_int, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_void_p]
    lib.sibfa_cluster_elec_noalloc.restype = C.c_int
    lib.sibfa_noalloc_last_error.argtypes = []
    lib.sibfa_noalloc_last_error.restype = C.c_char_p
    lib.sibfa_alu_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.sibfa_alu_peak.restype = C.c_int
    lib.sibfa_alu_peak_error.argtypes = []
    lib.sibfa_alu_peak_error.restype = C.c_char_p
    lib.sibfa_math_selftest.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_float, C.c_void_p, C.c_void_p]
    lib.sibfa_math_selftest.restype = C.c_int
    lib.sibfa_destroy.argtypes = [C.c_void_p]
    lib.sibfa_destroy.restype = None
    lib.sibfa_last_error.argtypes = [C.c_void_p]
    lib.sibfa_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a float64 contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(lib, ctx, st):
    if st != SIBFA_OK:
        raise SibfaError(st, lib.sibfa_last_error(ctx).decode())


def sibfa_create(params: dict, mp_local: np.ndarray, *, periodic: bool, box=None, rc=9.0, grid=64, order=5,
                 ewald_alpha=0.4, pcg_tol_D=1e-6, pcg_max_iter=200, precision=PREC_MIXED, warm_start=True,
                 stream=None, md_k_bond=529.6, md_r0=0.9572, md_k_angle=34.05, md_theta0_deg=104.52,
                 cluster_start=None, disp_tail=False, md_integrator="verlet", md_anharmonic=False, md_k_ub=0.0,
                 md_r_ub=1.5326, ct_original=False):
    """Create a context.  mp_local: (n_mol, 5, 10) float64 host array.
    stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None.
    cluster_start: optional (n_clusters + 1) ints splitting a gas-phase batch
    into independent clusters of consecutive molecules.
    warm_start: PCG initial guess, False/0 direct field, True/1 previous
    dipoles, 2..6 extrapolation through the last 2..6 full evaluations."""
    lib = load_library()
    P = sibfa_params(*[float(params[n]) for n in PARAM_FIELDS])
    mp = np.ascontiguousarray(mp_local, dtype=np.float64)
    topo = sibfa_topology(mp.shape[0], mp.ctypes.data_as(C.POINTER(C.c_double)), 0, None)
    if cluster_start is not None:
        cs = np.ascontiguousarray(cluster_start, dtype=np.int32)
        topo.n_clusters = int(cs.size - 1)
        topo.cluster_start = cs.ctypes.data_as(C.POINTER(C.c_int))
    o = sibfa_run_opts()
    o.periodic = 1 if periodic else 0
    if box is not None:
        for k in range(3):
            o.box[k] = float(box[k])
    o.rc = float(rc)
    g = (grid, grid, grid) if np.isscalar(grid) else tuple(grid)
    for k in range(3):
        o.grid[k] = int(g[k])
    o.order = int(order)
    o.ewald_alpha = float(ewald_alpha)
    o.pcg_tol_D = float(pcg_tol_D)
    o.pcg_max_iter = int(pcg_max_iter)
    o.precision = int(precision)
    o.warm_start = int(warm_start)
    if stream is not None:
        o.stream = int(getattr(stream, "cuda_stream", stream))
    o.md_k_bond, o.md_r0, o.md_k_angle, o.md_theta0_deg = md_k_bond, md_r0, md_k_angle, md_theta0_deg
    o.disp_tail = 1 if disp_tail else 0
    o.md_integrator = {"verlet": 0, "beeman": 1}[md_integrator]
    o.md_anharmonic = 1 if md_anharmonic else 0
    o.md_k_ub, o.md_r_ub = float(md_k_ub), float(md_r_ub)
    o.ct_original = 1 if ct_original else 0
    out = C.c_void_p()
    st = lib.sibfa_create(C.byref(P), C.byref(topo), C.byref(o), C.byref(out))
    _check(lib, None, st)
    return out


def _host_box(box):
    """The box as 3 host doubles (the C ABI reads it on the host)."""
    if box is None:
        return None
    if hasattr(box, "detach"):
        box = box.detach().cpu().numpy()
    b = np.ascontiguousarray(box, dtype=np.float64).reshape(-1)
    if b.size != 3:
        raise ValueError("box must have 3 edges")
    return b


def sibfa_energy_forces(ctx, pos, forces=None, box=None, virial=None):
    """One evaluation; returns a dict of energy terms (kcal/mol).  forces (same
    shape as pos) is filled in place when given; virial (a host float64 array
    of 9) receives W_ab = -dE/d eps_ab (row-major) when given.  box (3 edges)
    different from the context's current box changes it (periodic contexts;
    constant-pressure MD)."""
    lib = load_library()
    box = _host_box(box)
    e = sibfa_energy_terms()
    vir = None
    if virial is not None:
        vir = (C.c_double * 9)()
    st = lib.sibfa_energy_forces(ctx, _ptr(pos), _ptr(box), C.byref(e), _ptr(forces),
                                 C.addressof(vir) if vir is not None else None)
    _check(lib, ctx, st)
    if virial is not None:
        virial[...] = np.frombuffer(vir, dtype=np.float64).reshape(np.shape(virial))
    return {n: getattr(e, n) for n in TERMS}


def sibfa_solve_dipoles(ctx, pos, mu=None, tol_D=0.0, box=None):
    """Solve T mu = E only; returns (iterations, residual in D)."""
    lib = load_library()
    box = _host_box(box)
    it = C.c_int()
    res = C.c_double()
    st = lib.sibfa_solve_dipoles(ctx, _ptr(pos), _ptr(box), float(tol_D), _ptr(mu), C.byref(it), C.byref(res))
    _check(lib, ctx, st)
    return it.value, res.value


def sibfa_md_steps(ctx, pos, vel, masses, dt_fs, n_steps):
    """Velocity-Verlet NVE steps on device arrays; returns the last energy terms."""
    lib = load_library()
    e = sibfa_energy_terms()
    st = lib.sibfa_md_steps(ctx, _ptr(pos), _ptr(vel), _ptr(masses), float(dt_fs), int(n_steps), C.byref(e))
    _check(lib, ctx, st)
    return {n: getattr(e, n) for n in TERMS}


def sibfa_minimize(ctx, pos, n_steps, max_disp_A=0.02):
    """Capped steepest-descent relaxation of device positions (in place)."""
    lib = load_library()
    e = sibfa_energy_terms()
    st = lib.sibfa_minimize(ctx, _ptr(pos), int(n_steps), float(max_disp_A), C.byref(e))
    _check(lib, ctx, st)
    return {n: getattr(e, n) for n in TERMS}


def sibfa_cluster_elec_noalloc(params: dict, pos, mp_local, elec_pen, stream=None):
    """Allocation-free cluster electrostatics: pos (n_mol*9), mp_local
    (n_mol*50) and elec_pen (2) are float64 CUDA tensors.  Asynchronous on
    `stream` (a torch.cuda.Stream, raw handle, or None for the legacy default
    stream)."""
    import torch
    for name, t in (("pos", pos), ("mp_local", mp_local), ("elec_pen", elec_pen)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise TypeError(f"sibfa_cluster_elec_noalloc: {name} must be a CUDA tensor")
    if len({t.device for t in (pos, mp_local, elec_pen)}) != 1:
        raise ValueError("sibfa_cluster_elec_noalloc: pos, mp_local and elec_pen must be on one device")
    n_mol = int(pos.numel() // 9)
    if pos.numel() % 9 or mp_local.numel() != n_mol * 50 or elec_pen.numel() < 2:
        raise ValueError("sibfa_cluster_elec_noalloc: need pos of n_mol*9, mp_local of n_mol*50 and elec_pen "
                         f"of >= 2 doubles (got {pos.numel()}, {mp_local.numel()}, {elec_pen.numel()})")
    lib = load_library()
    P = sibfa_params(*[float(params[n]) for n in PARAM_FIELDS])
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    st = lib.sibfa_cluster_elec_noalloc(C.byref(P), n_mol, _ptr(pos), _ptr(mp_local), _ptr(elec_pen), s)
    if st != SIBFA_OK:
        raise SibfaError(st, lib.sibfa_noalloc_last_error().decode())


def sibfa_alu_peak(fp64: bool = False, iters: int = 4096, blocks: int = 0):
    """FMA-chain rate of the current device: returns (flops, milliseconds).
    blocks = 0 launches 8 blocks of 256 threads per SM."""
    lib = load_library()
    if blocks <= 0:
        import torch
        blocks = 8 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ms, fl = C.c_double(), C.c_double()
    st = lib.sibfa_alu_peak(1 if fp64 else 0, int(iters), int(blocks), C.byref(ms), C.byref(fl))
    if st != SIBFA_OK:
        raise SibfaError(st, lib.sibfa_alu_peak_error().decode())
    return fl.value, ms.value


def sibfa_math_selftest(fn: int, x, alpha: float = 0.0):
    """The library's FP32 elementary kernels beside CUDA's on a float32 CUDA
    tensor x: returns a float32 CUDA tensor of shape (n, 2) (fn 0, 1) or
    (n, 5) (fn 2), see include/sibfa.h."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError("x must be a contiguous float32 CUDA tensor")
    lib = load_library()
    w = 5 if fn == 2 else 2
    out = torch.empty((x.numel(), w), dtype=torch.float32, device=x.device)
    st = lib.sibfa_math_selftest(int(fn), x.numel(), x.data_ptr(), float(alpha), out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    if st != SIBFA_OK:
        raise SibfaError(st, "sibfa_math_selftest failed")
    return out


def sibfa_cluster_terms(ctx, n_clusters: int):
    """Energy terms per cluster of the last evaluation: list of dicts."""
    lib = load_library()
    arr = (sibfa_energy_terms * max(1, int(n_clusters)))()
    _check(lib, ctx, lib.sibfa_cluster_terms(ctx, arr))
    return [{k: getattr(t, k) for k, _ in sibfa_energy_terms._fields_} for t in arr]


def sibfa_last_stats(ctx):
    lib = load_library()
    it = C.c_int()
    res = C.c_double()
    _check(lib, ctx, lib.sibfa_last_stats(ctx, C.byref(it), C.byref(res)))
    return it.value, res.value


def sibfa_kernel_launches(ctx) -> int:
    return int(load_library().sibfa_kernel_launches(ctx))


def sibfa_tuned_schedule(ctx):
    """(short-range blocks per SM, joined before the solve, True once tuning
    fixed it, the five candidates' fastest timed evaluations in ms)."""
    lib = load_library()
    b, j, dn = C.c_int(), C.c_int(), C.c_int()
    ms = (C.c_double * 5)()
    st = lib.sibfa_tuned_schedule(ctx, C.byref(b), C.byref(j), C.byref(dn), ms, 5)
    _check(lib, ctx, st)
    return b.value, bool(j.value), bool(dn.value), list(ms)


def sibfa_tuned_shape(ctx):
    """(short-range resident blocks per SM, 0 = uncapped; True once tuning fixed it)."""
    lib = load_library()
    b, dn = C.c_int(), C.c_int()
    st = lib.sibfa_tuned_shape(ctx, C.byref(b), C.byref(dn))
    _check(lib, ctx, st)
    return b.value, bool(dn.value)


def sibfa_set_profiling(ctx, on):
    """on: False/0 off, True/1 phase spans with the usual stream overlap,
    2 serial (every phase alone on the GPU)."""
    load_library().sibfa_set_profiling(ctx, int(on))


def sibfa_profile_get(ctx, name: str):
    """(milliseconds summed, span count) of one phase since its last read."""
    lib = load_library()
    ms = C.c_double()
    n = C.c_int()
    _check(lib, ctx, lib.sibfa_profile_get(ctx, name.encode(), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def sibfa_profile_clear(ctx):
    load_library().sibfa_profile_clear(ctx)


def sibfa_destroy(ctx):
    if ctx:
        load_library().sibfa_destroy(ctx)


def sibfa_last_error(ctx=None) -> str:
    return load_library().sibfa_last_error(ctx).decode()


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------
SIBFA_E_BUSY = -8


class Server:
    """Request server (sibfa_server_*): submit MD/energy jobs, poll results."""

    def __init__(self, params: dict, *, slots=2, device_mem_bytes=8 << 30, max_pending=4096, batch_waters=8192,
                 batch_max_cluster=32, batch_dt_fs=0.5, precision=PREC_MIXED, pcg_tol_D=1e-6):
        self._lib = load_library()
        self._h = None
        self._P = sibfa_params(*[float(params[n]) for n in PARAM_FIELDS])
        o = sibfa_server_opts(C.pointer(self._P), int(slots), int(device_mem_bytes), int(max_pending),
                              int(batch_waters), int(batch_max_cluster), float(batch_dt_fs), int(precision),
                              float(pcg_tol_D))
        h = C.c_void_p()
        st = self._lib.sibfa_server_create(C.byref(o), C.byref(h))
        if st != SIBFA_OK:
            raise SibfaError(st, "sibfa_server_create failed")
        self._h = h
        self._n = {}

    def submit(self, pos, mp_local, *, vel=None, periodic=False, box=None, rc=9.0, grid=64, ewald_alpha=0.4,
               n_steps=0, dt_fs=0.5):
        """Queue a job; returns its ticket, or None when the server is busy."""
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
        mp = np.ascontiguousarray(mp_local, dtype=np.float64).reshape(-1)
        n = pos.size // 9
        j = sibfa_job()
        j.n_mol = n
        j.pos = pos.ctypes.data_as(C.POINTER(C.c_double))
        v = None
        if vel is not None:
            v = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1)
            j.vel = v.ctypes.data_as(C.POINTER(C.c_double))
        j.mp_local = mp.ctypes.data_as(C.POINTER(C.c_double))
        j.periodic = 1 if periodic else 0
        if box is not None:
            for k in range(3):
                j.box[k] = float(box[k])
        g = (grid, grid, grid) if np.isscalar(grid) else tuple(grid)
        for k in range(3):
            j.grid[k] = int(g[k])
        j.rc, j.ewald_alpha, j.n_steps, j.dt_fs = float(rc), float(ewald_alpha), int(n_steps), float(dt_fs)
        t = C.c_uint64()
        st = self._lib.sibfa_submit(self._h, C.byref(j), C.byref(t))
        if st == SIBFA_E_BUSY:
            return None
        if st != SIBFA_OK:
            raise SibfaError(st, "sibfa_submit refused the job")
        self._n[t.value] = n
        return t.value

    def poll(self, ticket):
        """None while the job waits or runs; then a dict with terms, forces,
        final positions, status, pcg_iters, queue_ms, latency_ms, batched."""
        n = self._n[ticket]
        F = np.zeros(n * 9)
        X = np.zeros(n * 9)
        r = sibfa_result()
        r.forces = F.ctypes.data_as(C.POINTER(C.c_double))
        r.pos = X.ctypes.data_as(C.POINTER(C.c_double))
        done = C.c_int()
        st = self._lib.sibfa_poll(self._h, C.c_uint64(ticket), C.byref(r), C.byref(done))
        if st != SIBFA_OK:
            raise SibfaError(st, "sibfa_poll: unknown ticket")
        if not done.value:
            return None
        del self._n[ticket]
        return {"terms": {k: getattr(r.terms, k) for k in TERMS}, "forces": F, "pos": X, "status": r.status,
                "pcg_iters": r.pcg_iters, "queue_ms": r.queue_ms, "latency_ms": r.latency_ms,
                "batched": bool(r.batched)}

    def close(self):
        if self._h:
            self._lib.sibfa_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
