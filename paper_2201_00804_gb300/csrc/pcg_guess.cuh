// PCG initial guess extrapolated from stored solutions of earlier evaluations.
#pragma once
#include "sibfa_internal.cuh"

namespace sibfa {

// sum_j c[j] h[j] over n stored dipole vectors (n = 0: no stored guess)
constexpr int MU_HIST = 6;   // stored solutions at most (quintic extrapolation)
struct MuGuess {
    const double *h[MU_HIST];
    double c[MU_HIST];
    int n;
};

// k_pcg_init with the dipoles set to the combination g (n >= 1) instead of
// alpha E or the previous dipoles
template <typename R> void launch_pcg_init_guess(const KParams &p, DevState<R> &d, MuGuess g, Launch L);

}  // namespace sibfa
