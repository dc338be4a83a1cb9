// Internal hooks between the context code (capi.cu) and the request server
// (server.cu); not part of the C ABI.
#pragma once
#include <cstddef>

#include <cuda_runtime.h>

#include "sibfa.h"

namespace sibfa {

// Device arrays of a gas-phase context that the server rearranges between
// steps of a batch (molecule-major, the layouts of the C ABI).
struct BatchArrays {
    double *mp_local;   // capacity * 50 local-frame multipoles
    double *mu;         // capacity * 9 induced dipoles (warm start of the next solve)
    double *forces;     // capacity * 9 forces of the last evaluation
    int capacity;       // molecules the arrays hold
};

// Regroup a gas-phase context to n_mol <= capacity molecules in n_cl clusters
// (cluster_start: host, n_cl + 1 ints); the caller has placed the molecules'
// multipoles (and warm-start dipoles) in the device arrays.
sibfa_status ctx_set_batch(sibfa_ctx *ctx, int n_mol, int n_cl, const int *cluster_start);
BatchArrays ctx_batch_arrays(sibfa_ctx *ctx);
cudaStream_t ctx_stream(sibfa_ctx *ctx);
size_t ctx_device_bytes(const sibfa_ctx *ctx);

}  // namespace sibfa
