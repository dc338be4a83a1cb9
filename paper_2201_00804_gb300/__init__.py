"""GB300-native SIBFA21 water energy + force library (sm_103a CUDA behind a C ABI).

The compute path is libsibfa.so (csrc/, include/sibfa.h); this package holds
the ctypes binding (sibfa.py) and the in-tree build (build.py).  There is no
CPU fallback: the binding raises if the library is missing.
"""
from .sibfa import (  # noqa: F401
    PREC_FP64,
    PREC_MIXED,
    Server,
    SibfaError,
    load_library,
    sibfa_alu_peak,
    sibfa_cluster_terms,
    sibfa_math_selftest,
    sibfa_create,
    sibfa_destroy,
    sibfa_energy_forces,
    sibfa_kernel_launches,
    sibfa_tuned_schedule,
    sibfa_tuned_shape,
    sibfa_last_error,
    sibfa_last_stats,
    sibfa_md_steps,
    sibfa_minimize,
    sibfa_profile_clear,
    sibfa_profile_get,
    sibfa_set_profiling,
    sibfa_solve_dipoles,
)
