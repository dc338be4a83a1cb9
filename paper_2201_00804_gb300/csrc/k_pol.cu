// Polarization solve (Technical Appendix: T mu = E, Jacobi-preconditioned
// conjugate gradient with FP64 vectors and dot products), intramolecular
// Ewald corrections, the chain rule from point gradients and multipole
// sensitivities to atom forces, energy totals and the velocity-Verlet kick.
#include <cooperative_groups.h>

#include <algorithm>

#include "sibfa_internal.cuh"
#include "pcg_guess.cuh"

namespace sibfa {

// scal[] layout
enum { S_RZ = 0, S_PAP = 1, S_ALPHA = 2, S_BETA = 3, S_RES = 4, S_RZN = 5, S_IT = 6, S_DONE = 7, S_TOL = 8 };
constexpr int PB = 256;   // threads per block of the vector kernels

__device__ inline double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;   // valid in thread 0
}

// Two block partials reduced by the last block to finish, in fixed order.
// Returns true in thread 0 of the last block, with the two totals.
// *is_last (optional) tells every thread of the block whether it is the last one.
__device__ inline bool last_block_sum2(double a, double b, double *partial, unsigned *counter, double &ta,
                                       double &tb, bool *is_last = nullptr) {
    __shared__ double sh[32];
    __shared__ bool s_last;
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
        __threadfence();
        unsigned k = atomicAdd(counter, 1u);
        s_last = (k == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) *is_last = s_last;
    if (!s_last) return false;
    __threadfence();
    double x = 0, y = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        x += __ldcg(&partial[2 * i]);
        y += __ldcg(&partial[2 * i + 1]);
    }
    x = block_sum(x, sh);
    y = block_sum(y, sh);
    if (threadIdx.x == 0) {
        ta = x;
        tb = y;
        *counter = 0;
        return true;
    }
    return false;
}

__device__ inline double apol(const KParams &p, int k) { return p.a_pol[(k / 3) % 3]; }
__device__ inline double apol_inv(const KParams &p, int k) { return p.a_pol_inv[(k / 3) % 3]; }

// Zero the real SPME grid (input of the next spread of the PCG product).
template <typename R>
__device__ inline void zero_grid(const KParams &p, const DevState<R> &d, size_t tid, size_t nth) {
    if (!p.periodic) return;
    const size_t ng = (size_t)p.K[0] * p.K[1] * p.K[2];
    for (size_t k = tid; k < ng; k += nth) d.grid[k] = R(0);
}

template <typename R>
__global__ void k_pcg_init(KParams p, DevState<R> d, int warm, MuGuess g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    zero_grid(p, d, k, (size_t)gridDim.x * blockDim.x);
    if (p.n_cl > 1 && k < p.n_cl) d.cl_rr[k] = 0.0;
    if (k >= p.M * 9) return;
    if (g.n > 0) {
        double m = 0;
        for (int j = 0; j < g.n; ++j) m += g.c[j] * g.h[j][k];
        d.mu[k] = m;
    } else if (!warm) {
        d.mu[k] = apol(p, k) * d.efield[k];
    }
    d.vecR[k] = R(d.mu[k]);
    d.efp[k] = 0.0;
    d.efp_r[k] = 0.0;
}

// r = E - T mu0, z = alpha r, p = z
template <typename R>
__global__ void k_pcg_first(KParams p, DevState<R> d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    zero_grid(p, d, k, (size_t)gridDim.x * blockDim.x);
    double rz = 0, rr = 0;
    if (k < p.M * 9) {
        const double a = apol(p, k);
        const double r = d.efield[k] - (d.mu[k] * apol_inv(p, k) - (d.efp[k] + d.efp_r[k]));
        d.res[k] = r;
        d.zv[k] = a * r;
        d.pv[k] = a * r;
        d.vecR[k] = R(a * r);
        d.efp[k] = 0.0;
        d.efp_r[k] = 0.0;
        rz = r * a * r;
        rr = a * r * a * r;
    }
    if (p.n_cl > 1) cluster_rr_add(d, k, k < p.M * 9, rr);
    double trz, trr;
    bool last = false;
    const bool lead = last_block_sum2(rz, rr, d.partial, d.counter, trz, trr, &last);
    double cres = 0;
    if (last && p.n_cl > 1) cres = cluster_res_max(p, d);   // the whole last block
    if (lead) {
        d.scal[S_RZ] = trz;
        const double res = p.n_cl > 1 ? cres : sqrt(trr / (p.M * 3)) * 4.80321;
        d.scal[S_RES] = res;
        d.scal[S_IT] = 0;
        d.scal[S_DONE] = (res < d.scal[S_TOL]) ? 1.0 : 0.0;
        d.flags[1] = res < d.scal[S_TOL];
    }
}

// Cluster batches: the largest per-cluster RMS preconditioned residual (D)
// from the per-cluster sums of squares.  Block-wide (all threads call it);
// every block gets the same value (a maximum does not depend on order).
template <typename R>
__device__ inline double cluster_res_max(const KParams &p, const DevState<R> &d) {
    __shared__ double smx[32];
    double mx = 0;
    for (int c = threadIdx.x; c < p.n_cl; c += blockDim.x) {
        const int n = d.cl_start[c + 1] - d.cl_start[c];
        mx = fmax(mx, __ldcg(d.cl_rr + c) / (3.0 * n));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) smx[threadIdx.x >> 5] = mx;
    __syncthreads();
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, smx[w]);
    __syncthreads();
    return sqrt(r) * 4.80321;
}

// Cluster batches: add v (element k of the PCG vectors, valid or not) to the
// sum of squares of its cluster.  Warp-collective: a warp whose elements lie
// in one cluster adds its total with one atomic.
template <typename R>
__device__ inline void cluster_rr_add(const DevState<R> &d, int k, bool valid, double v) {
    const int c = valid ? d.cl_of[k / 9] : -1;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    if (__all_sync(0xffffffffu, c == c0 || c < 0)) {
        const double s = warp_sum(valid ? v : 0.0);
        if ((threadIdx.x & 31) == 0 && c0 >= 0) atomicAdd(d.cl_rr + c0, s);
    } else if (valid) {
        atomicAdd(d.cl_rr + c, v);
    }
}

// Block sums of two values at once (valid in thread 0): the two FP64 add
// chains interleave, and the second stage runs over the 8 warp totals only.
__device__ inline void block_sum2(double a, double b, double *sh, double &ra, double &rb) {
    static_assert(PB == 256, "8 warps per block");
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sh[w] = a;
        sh[16 + w] = b;
    }
    __syncthreads();
    ra = rb = 0;
    if (w == 0) {
        double x = l < 8 ? sh[l] : 0.0, y = l < 8 ? sh[16 + l] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        ra = x;
        rb = y;
    }
}

// Sums of nb pairs of block partials (part[2b], part[2b + 1]) in a fixed
// order, both in one pass: every block obtains bit-identical totals.
__device__ inline void sum_partials2(const double *part, int nb, double *sh, double &ta, double &tb) {
    if (threadIdx.x < 32) {
        double a = 0, b = 0;
        for (int k = threadIdx.x; k < nb; k += 32) {
            a += __ldcg(part + 2 * k);
            b += __ldcg(part + 2 * k + 1);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        if (threadIdx.x == 0) {
            sh[0] = a;
            sh[1] = b;
        }
    }
    __syncthreads();
    ta = sh[0];
    tb = sh[1];
    __syncthreads();
}

// Sum of the nb block partials at part[0], part[stride], ... in a fixed
// order (lane l takes l, l+32, ...; then a fixed tree): every block obtains
// the bit-identical total.
__device__ inline double sum_partials(const double *part, int nb, int stride, double *sh) {
    if (threadIdx.x < 32) {
        double v = 0;
        for (int b = threadIdx.x; b < nb; b += 32) v += __ldcg(part + (size_t)b * stride);
        v = warp_sum(v);
        if (threadIdx.x == 0) sh[0] = v;
    }
    __syncthreads();
    const double t = sh[0];
    __syncthreads();
    return t;
}

// One PCG iteration after the product T p (cooperative launch, grid-stride):
//   (a) ap = p / alpha - E(p), alpha_k = rz / p.ap
//   (b) mu += alpha_k p, r -= alpha_k ap, z = alpha r, beta = rz_new / rz,
//       residual check
//   (c) p = z + beta p, working-precision copy of p, clear the field
//       accumulators and the SPME grid for the next product.
// Inside the solver graph (maxit > 0) it also sets the while-node's
// condition: another iteration while not converged and below maxit.
template <typename R>
__global__ void __launch_bounds__(PB) k_pcg_step(KParams p, DevState<R> d, cudaGraphConditionalHandle loop,
                                                 int maxit) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ double sh[32];
    if (d.flags[1]) {   // converged before this launch: uniform over the grid
        if (maxit > 0 && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(loop, 0u);
        return;
    }
    const int n = p.M * 9;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int nb = gridDim.x;
    const double rz_old = d.scal[S_RZ], tol = d.scal[S_TOL];
    double pap = 0;
    unsigned long long *rmax = reinterpret_cast<unsigned long long *>(d.partial + 3 * nb);   // cluster max slot
    if (p.n_cl > 1) {
        for (int c = tid; c < p.n_cl; c += nth) d.cl_rr[c] = 0.0;
        if (tid == 0) *rmax = 0ull;
    }
    for (int k = tid; k < n; k += nth) {
        const double ap = d.pv[k] * apol_inv(p, k) - (d.efp[k] + d.efp_r[k]);
        d.ap[k] = ap;
        pap += d.pv[k] * ap;
    }
    pap = block_sum(pap, sh);
    if (threadIdx.x == 0) d.partial[blockIdx.x] = pap;
    grid.sync();
    const double tpap = sum_partials(d.partial, nb, 1, sh);
    const double al = rz_old / tpap;
    double rz = 0, rr = 0;
    for (int k0 = tid - (threadIdx.x & 31); k0 < n; k0 += nth) {   // warp-uniform trip count
        const int k = k0 + (threadIdx.x & 31);
        double q = 0;
        if (k < n) {
            const double a = apol(p, k);
            d.mu[k] += al * d.pv[k];
            const double r = d.res[k] - al * d.ap[k];
            d.res[k] = r;
            d.zv[k] = a * r;
            rz += r * a * r;
            q = a * r * a * r;
            rr += q;
        }
        if (p.n_cl > 1) cluster_rr_add(d, k, k < n, q);
    }
    double brz, brr;
    block_sum2(rz, rr, sh, brz, brr);
    if (threadIdx.x == 0) {
        d.partial[nb + 2 * blockIdx.x] = brz;
        d.partial[nb + 2 * blockIdx.x + 1] = brr;
    }
    grid.sync();
    double trz, trr;
    sum_partials2(d.partial + nb, nb, sh, trz, trr);
    const double beta = trz / rz_old;
    double res = sqrt(trr / (p.M * 3)) * 4.80321;
    if (p.n_cl > 1) {
        // largest per-cluster mean square: each block a slice, combined by an
        // atomic maximum (non-negative doubles order like their bit patterns)
        double mx = 0;
        for (int c = tid; c < p.n_cl; c += nth)
            mx = fmax(mx, __ldcg(d.cl_rr + c) / (3.0 * (d.cl_start[c + 1] - d.cl_start[c])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(rmax, (unsigned long long)__double_as_longlong(mx));
        grid.sync();
        res = sqrt(__longlong_as_double((long long)__ldcg(rmax))) * 4.80321;
    }
    const bool done = res < tol;
    if (tid == 0) {
        d.scal[S_PAP] = tpap;
        d.scal[S_ALPHA] = al;
        d.scal[S_BETA] = beta;
        d.scal[S_RZ] = trz;
        d.scal[S_RES] = res;
        d.scal[S_IT] += 1.0;
        if (done) {
            d.scal[S_DONE] = 1.0;
            d.flags[1] = 1;
        }
        if (maxit > 0) cudaGraphSetConditional(loop, (!done && d.scal[S_IT] < (double)maxit) ? 1u : 0u);
    }
    if (done) return;   // uniform: every block computed the same residual
    for (int k = tid; k < n; k += nth) {
        const double pk = d.zv[k] + beta * d.pv[k];
        d.pv[k] = pk;
        d.vecR[k] = R(pk);
        d.efp[k] = 0.0;
        d.efp_r[k] = 0.0;
    }
    zero_grid(p, d, tid, nth);
}

static inline unsigned nblk(int n) { return (unsigned)((n + PB - 1) / PB); }

// start of an evaluation: clear the solver scalars and the converged flag,
// set the tolerance (error flags accumulate over the evaluations of one call)
__global__ void k_begin(double *scal, int *flags, double tol_D) {
    if (threadIdx.x < 16) scal[threadIdx.x] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        scal[S_TOL] = tol_D;
        flags[1] = 0;   // PCG converged (integer copy of scal[S_DONE] for the loop kernels)
    }
}
// after the solve: record a solve that stopped at the iteration limit
__global__ void k_pcg_check(const double *scal, int *flags) {
    if (scal[S_DONE] == 0.0) atomicOr(flags, F_NOCONV);
}
void launch_pcg_check(const double *scal, int *flags, Launch L) {
    k_pcg_check<<<1, 1, 0, L.s>>>(scal, flags);
    count(L);
}

void launch_begin(double *scal, int *flags, double tol_D, Launch L) {
    k_begin<<<1, 32, 0, L.s>>>(scal, flags, tol_D);
    count(L);
}

template <typename R>
void launch_pcg_init(const KParams &p, DevState<R> &d, int warm, Launch L) {
    k_pcg_init<R><<<nblk(p.M * 9), PB, 0, L.s>>>(p, d, warm, MuGuess{});
    count(L);
}
template <typename R>
void launch_pcg_init_guess(const KParams &p, DevState<R> &d, MuGuess g, Launch L) {
    k_pcg_init<R><<<nblk(p.M * 9), PB, 0, L.s>>>(p, d, 1, g);
    count(L);
}
template <typename R>
void launch_pcg_first(const KParams &p, DevState<R> &d, Launch L) {
    k_pcg_first<R><<<nblk(p.M * 9), PB, 0, L.s>>>(p, d);
    count(L);
}
// Cooperative launch of the PCG step: a grid-stride kernel with as many
// blocks as can be resident at once (at most one per 256 vector entries).
template <typename R>
void launch_pcg_step(const KParams &p, DevState<R> &d, Launch L, cudaGraphConditionalHandle loop, int maxit) {
    static int per_sm[2] = {0, 0}, n_sm = 0;
    int &ps = per_sm[sizeof(R) == 8];
    if (ps == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_pcg_step<R>, PB, 0);
        if (ps < 1) ps = 1;
    }
    // at most two blocks per SM: the grid must be co-resident while the
    // short-range kernels occupy part of every SM on their own stream
    const unsigned grid = (unsigned)std::min<long long>(nblk(p.M * 9), (long long)std::min(ps, 2) * n_sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PB);
    cfg.stream = L.s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_pcg_step<R>, p, d, loop, maxit);
    count(L);
}

// E_pol = -1/2 ke mu . E (value at the solution); working-precision copies
// of mu and of the CT lambdas for the force pass
template <typename R>
__global__ void k_pol_energy(KParams p, DevState<R> d) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    double e = 0;
    for (int k = 0; k < 9; ++k) {
        e += d.mu[m * 9 + k] * d.efield[m * 9 + k];
        d.muR[m * 9 + k] = R(d.mu[m * 9 + k]);
    }
    d.lamR[m * 2] = R(d.lam[m * 2]);
    d.lamR[m * 2 + 1] = R(d.lam[m * 2 + 1]);
    if (p.ct_orig)
        for (int a = 0; a < 3; ++a) d.lamaR[m * 3 + a] = R(d.lama[m * 3 + a]);
    d.epart[m * NTERM + T_POL] = -0.5 * p.ke * e;
    // real-space multipole and penetration energies of the five target sites
    double el = 0, pe = 0;
    for (int w = 0; w < NS; ++w) el += d.epw[(m * NS + w) * 2], pe += d.epw[(m * NS + w) * 2 + 1];
    d.epart[m * NTERM + T_ELEC] += el;
    d.epart[m * NTERM + T_PEN] += pe;
}
template <typename R>
void launch_pol_energy(const KParams &p, DevState<R> &d, Launch L) {
    k_pol_energy<R><<<(p.M + 127) / 128, 128, 0, L.s>>>(p, d);
    count(L);
}

// ---------------------------------------------------------------------------
// Chain rule to atom forces.  Frame construction: z along zv, x in the
// (z, xv) plane, y = z x x; its vector-Jacobian product maps gradients of the
// axes back to zv and xv.
// ---------------------------------------------------------------------------
template <typename W>
__device__ inline void frame_vjp(V3<W> zv, V3<W> xv, V3<W> gx, V3<W> gy, V3<W> gz, V3<W> &gzv, V3<W> &gxv) {
    const W iz = rsqrt_<W>(dot(zv, zv));
    const V3<W> ez = iz * zv;
    const V3<W> xp = xv - dot(xv, ez) * ez;
    const W ix = rsqrt_<W>(dot(xp, xp));
    const V3<W> ex = ix * xp;
    // y = z x x
    gz = gz + cross(ex, gy);
    gx = gx + cross(gy, ez);
    // x = xp / |xp|
    const V3<W> gxp = ix * (gx - dot(gx, ex) * ex);
    // xp = xv - (xv.z) z
    gxv = gxp - dot(gxp, ez) * ez;
    gz = gz - dot(xv, ez) * gxp - dot(gxp, ez) * xv;
    // z = zv / |zv|
    gzv = iz * (gz - dot(gz, ez) * ez);
}

// Four lanes per molecule.  Lane f < 3 carries the multipole sensitivities
// of the sites in frame f (frame 0: O and the lone pairs; frame 1: H1, M1;
// frame 2: H2, M2) back through that frame's construction; lane 3 takes the
// point gradients (lone-pair charge-transfer term, V_int chain rule,
// midpoints, lone-pair carrier).  The four partial atom gradients are summed
// with shuffles.  The accumulated gradients are summed in FP64 and the chain
// rule runs in the working precision R, on the same frames as the site
// kernel.
template <typename R>
__global__ void __launch_bounds__(128) k_finalize(KParams p, DevState<R> d, double *forces) {
    const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = gidx >> 2, t = gidx & 3;
    const bool live = m < p.M;
    V3<R> gO = mk(R(0), R(0), R(0)), gH1 = gO, gH2 = gO;
    R W[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // virial (p.vir)
    if (live) {
        V3<R> r1, r2;
        bond_vectors(d.pos + m * 9, r1, r2);
        const R s1 = rsqrt_<R>(dot(r1, r1)), s2 = rsqrt_<R>(dot(r2, r2));
        auto sum2 = [&](const double *a, const double *b, int o) {
            return mk(R(a[o] + b[o]), R(a[o + 1] + b[o + 1]), R(a[o + 2] + b[o + 2]));
        };
        auto gpt = [&](int k) {
            const int o = (m * NP + k) * 3;
            return mk(R(d.gpt[o] + d.gpt_r[o] + d.gpt_s[o]), R(d.gpt[o + 1] + d.gpt_r[o + 1] + d.gpt_s[o + 1]),
                      R(d.gpt[o + 2] + d.gpt_r[o + 2] + d.gpt_s[o + 2]));
        };
        // lone-pair point gradient including the charge-transfer dependence through its potential
        auto glp = [&](int l) {
            return gpt(5 + l) + R(d.lam[m * 2 + l]) * sum2(d.dvlp, d.dvlp_r, (m * 2 + l) * 3);
        };
        if (t < 3) {
            const int f = t;
            V3<R> zv, xv, E[3];
            frame_generators(f, r1, r2, s1, s2, zv, xv);
            frame_axes(zv, xv, E[0], E[1], E[2]);
            V3<R> gE[3] = {mk(R(0), R(0), R(0)), mk(R(0), R(0), R(0)), mk(R(0), R(0), R(0))};
            for (int s = 0; s < NS; ++s) {
                if (site_frame(s) != f) continue;
                const double *ml = d.mp_local + (m * NS + s) * NMP;
                const int ot = (m * NS + s) * 6;
                const V3<R> gmu = sum2(d.gmu, d.gmu_r, (m * NS + s) * 3);
                const double *gt6 = d.gth + ot, *gr6 = d.gth_r + ot;
                const Sym<R> D{R(gt6[0] + gr6[0]), R(gt6[1] + gr6[1]), R(gt6[2] + gr6[2]),
                               R(gt6[3] + gr6[3]), R(gt6[4] + gr6[4]), R(gt6[5] + gr6[5])};
                const R tl[3][3] = {{R(ml[4]), R(ml[7]), R(ml[8])}, {R(ml[7]), R(ml[5]), R(ml[9])},
                                    {R(ml[8]), R(ml[9]), R(ml[6])}};
                for (int k = 0; k < 3; ++k) {
                    const V3<R> acc = tl[k][0] * E[0] + tl[k][1] * E[1] + tl[k][2] * E[2];
                    gE[k] = gE[k] + R(ml[1 + k]) * gmu + R(2) * symv(D, acc);
                }
            }
            if (f == 0)   // lone pairs: X = O + d (-c z_O +/- s y_O)
                for (int l = 0; l < 2; ++l) {
                    const V3<R> G = glp(l);
                    gE[2] = gE[2] + R(-p.d_lp * p.lp_cos) * G;
                    gE[1] = gE[1] + R(l == 0 ? p.d_lp * p.lp_sin : -p.d_lp * p.lp_sin) * G;
                }
            V3<R> gzv, gxv;
            frame_vjp(zv, xv, gE[0], gE[1], gE[2], gzv, gxv);
            if (f == 0) {
                // zv = u1 + u2, u_k = r_k/|r_k|; xv = r1
                const V3<R> u1 = s1 * r1, u2 = s2 * r2;
                const V3<R> gr1 = s1 * (gzv - dot(gzv, u1) * u1) + gxv;
                const V3<R> gr2 = s2 * (gzv - dot(gzv, u2) * u2);
                gH1 = gr1;
                gH2 = gr2;
                gO = -(gr1 + gr2);
            } else if (f == 1) {
                // zv = O - H1, xv = H2 - H1
                gO = gzv;
                gH1 = -(gzv + gxv);
                gH2 = gxv;
            } else {
                // zv = O - H2, xv = H1 - H2
                gO = gzv;
                gH2 = -(gzv + gxv);
                gH1 = gxv;
            }
            if (p.vir) {   // the frame's atoms move affinely: sum_a g_a (x) (x_a - O)
                vir_add(W, gH1, r1, R(1));
                vir_add(W, gH2, r2, R(1));
            }
        } else {
            V3<R> G[NS], X[NS];
            for (int k = 0; k < NS; ++k) {
                G[k] = gpt(k);
                const R *o = d.off + (m * NP + k) * 3;
                X[k] = mk(o[0], o[1], o[2]);
            }
            // charge-transfer dependence through the intramolecular potentials V_int(O, H1, H2)
            for (int a = 0; a < 3; ++a) {
                const double k = d.kap[m * 3 + a];
                if (k == 0.0) continue;
                const R kk = R(k * p.ke);
                for (int s = 0; s < NS; ++s) {
                    if (s == a) continue;
                    const V3<R> dd = X[a] - X[s];
                    const R ir = rsqrt_<R>(dot(dd, dd));
                    const R c = kk * d.gmp[(m * NS + s) * GMP] * ir * ir * ir;
                    G[a] = G[a] - c * dd;
                    G[s] = G[s] + c * dd;
                    if (p.vir) vir_add(W, dd, dd, -c);   // the (a, s) pair's gradient on a is -c dd
                }
            }
            // The pair kernels counted the lone pairs as points moving with
            // the strain; they follow the frame of O instead, which lane 0's
            // chain rule has taken: remove their point share g_lp (x) off_lp.
            if (p.vir)
                for (int l = 0; l < 2; ++l) {
                    const R *o = d.off + (m * NP + 5 + l) * 3;
                    vir_add(W, glp(l), mk(o[0], o[1], o[2]), R(-1));
                }
            // midpoints and the lone pairs' carrier
            gO = G[0] + R(0.5) * (G[3] + G[4]) + glp(0) + glp(1);
            gH1 = G[1] + R(0.5) * G[3];
            gH2 = G[2] + R(0.5) * G[4];
        }
    }
    R v[9] = {gO.x, gO.y, gO.z, gH1.x, gH1.y, gH1.z, gH2.x, gH2.y, gH2.z};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 1, 4);
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 2, 4);
    }
    if (live && t == 0 && forces) {
        double *F = forces + m * 9;
        for (int k = 0; k < 9; ++k) F[k] = -(double)v[k];
    }
    if (p.vir) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            W[k] += __shfl_xor_sync(0xffffffffu, W[k], 1, 4);
            W[k] += __shfl_xor_sync(0xffffffffu, W[k], 2, 4);
        }
        if (live && t == 0)
            for (int k = 0; k < 9; ++k) d.vir[m * 9 + k] += (double)W[k];
    }
}

// Virial total: out[3a + b] = -dE/d eps_ab = -(sum over molecules of both
// chains' dE/d eps + the k-space sums of npass convolution passes), summed
// in a fixed order by one block.
template <typename R>
__global__ void __launch_bounds__(256) k_virial_total(int M, DevState<R> d, int npass, double *out) {
    __shared__ double sh[8][9];
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = threadIdx.x; m < M; m += blockDim.x)
        for (int k = 0; k < 9; ++k) v[k] += d.vir[m * 9 + k] + d.vir_r[m * 9 + k];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 9; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[9];
        for (int k = 0; k < 9; ++k) {
            t[k] = 0;
            for (int j = 0; j < 8; ++j) t[k] += sh[j][k];
        }
        double ks[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < npass * VK_BLOCKS; ++b)
            for (int k = 0; k < 7; ++k) ks[k] += d.virk[(size_t)b * 8 + k];
        // dE/d eps_ab from the k-space sums: -delta_ab sum e + sum e f m_a m_b
        const int ia[6] = {0, 4, 8, 1, 2, 5}, ib[6] = {0, 4, 8, 3, 6, 7};
        for (int k = 0; k < 3; ++k) t[4 * k] -= ks[0];
        for (int k = 0; k < 6; ++k) {
            t[ia[k]] += ks[1 + k];
            if (ib[k] != ia[k]) t[ib[k]] += ks[1 + k];
        }
        for (int k = 0; k < 9; ++k) out[k] = -t[k];
    }
}

template <typename R>
void launch_virial_total(const KParams &p, DevState<R> &d, double *out, Launch L) {
    k_virial_total<R><<<1, 256, 0, L.s>>>(p.M, d, p.periodic ? 2 : 0, out);
    count(L);
}

// Join of the reciprocal chain into the permanent field that the
// polarization solve reads (the charge transfer reads both lone-pair
// potential arrays itself).
template <typename R>
__global__ void k_merge_rec(int M, DevState<R> d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M * 9) d.efield[k] += d.efield_r[k];
}
template <typename R>
void launch_merge_rec(const KParams &p, DevState<R> &d, Launch L) {
    k_merge_rec<R><<<(p.M * 9 + 255) / 256, 256, 0, L.s>>>(p.M, d);
    count(L);
}

template <typename R>
void launch_finalize(const KParams &p, DevState<R> &d, double *forces_out, Launch L) {
    const long long n = (long long)p.M * 4;
    k_finalize<R><<<(unsigned)((n + 127) / 128), 128, 0, L.s>>>(p, d, forces_out);
    count(L);
}

// energy totals: out[k] = sum_m epart[m*NTERM + k], out[NTERM] = total, in a
// fixed order: ER_BLOCKS blocks each sum a contiguous slice of molecules
// (threads take independent chains, then a shared-memory tree per term) into
// partials; one small block sums the partials in block order.
constexpr int ER_BLOCKS = 128, ER_THREADS = 256;
__global__ void __launch_bounds__(ER_THREADS) k_energy_partial(int M, const double *epart, const double *epart_r,
                                                              const double *eintra, double *partial) {
    __shared__ double sh[ER_THREADS / 32][NTERM];
    const int per = (M + ER_BLOCKS - 1) / ER_BLOCKS;
    const int m0 = blockIdx.x * per, m1 = min(M, m0 + per);
    double v[NTERM];
#pragma unroll
    for (int k = 0; k < NTERM; ++k) v[k] = 0.0;
    for (int m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NTERM; ++k) v[k] += epart[m * NTERM + k] + epart_r[m * NTERM + k];
        if (eintra) v[T_ELEC] += eintra[m];
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NTERM; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0) sh[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NTERM) {
        double x = 0.0;
        for (int j = 0; j < ER_THREADS / 32; ++j) x += sh[j][threadIdx.x];
        partial[blockIdx.x * NTERM + threadIdx.x] = x;
    }
}
__global__ void k_energy_final(const double *partial, double *out) {
    __shared__ double sh[NTERM];
    if (threadIdx.x < NTERM) {
        double x = 0.0;
        for (int b = 0; b < ER_BLOCKS; ++b) x += partial[b * NTERM + threadIdx.x];
        out[threadIdx.x] = x;
        sh[threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < NTERM; ++k) tot += sh[k];
        out[NTERM] = tot;
    }
}

void launch_energy_reduce(int M, const double *epart, const double *epart_r, const double *eintra, double *partial,
                          double *out, Launch L) {
    k_energy_partial<<<ER_BLOCKS, ER_THREADS, 0, L.s>>>(M, epart, epart_r, eintra, partial);
    k_energy_final<<<1, 32, 0, L.s>>>(partial, out);
    count(L, 2);
}

// Cluster batches: terms per cluster (one block per cluster, fixed order),
// then their sums over the clusters into out (NTERM terms and the total).
template <typename R>
__global__ void k_cluster_energy(KParams p, DevState<R> d) {
    __shared__ double sh[32];
    const int c = blockIdx.x;
    const int m0 = d.cl_start[c], m1 = d.cl_start[c + 1];
    double tot = 0;
    for (int k = 0; k < NTERM; ++k) {
        double v = 0;
        for (int m = m0 + threadIdx.x; m < m1; m += blockDim.x) v += d.epart[m * NTERM + k] + d.epart_r[m * NTERM + k];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) {
            d.cl_energy[c * (NTERM + 1) + k] = v;
            tot += v;
        }
    }
    if (threadIdx.x == 0) d.cl_energy[c * (NTERM + 1) + NTERM] = tot;
}
__global__ void k_cluster_total(int n_cl, const double *cl_energy, double *out) {
    __shared__ double sh[32];
    for (int k = 0; k <= NTERM; ++k) {
        double v = 0;
        for (int c = threadIdx.x; c < n_cl; c += blockDim.x) v += cl_energy[c * (NTERM + 1) + k];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) out[k] = v;
    }
}
template <typename R>
void launch_cluster_energy(const KParams &p, DevState<R> &d, double *out, Launch L) {
    k_cluster_energy<R><<<p.n_cl, 64, 0, L.s>>>(p, d);
    k_cluster_total<<<1, 512, 0, L.s>>>(p.n_cl, d.cl_energy, out);
    count(L, 2);
}

// velocity-Verlet half kick (and drift): v += dt/2 F/m ; x += dt v
__global__ void k_md_kick(int M, double *pos, double *vel, const double *inv_mass, const double *F, double dt,
                          int drift) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M * 9) return;
    const double conv = 4.184e-4;   // (kcal/mol/A)/amu -> A/fs^2
    double v = vel[k] + 0.5 * dt * F[k] * inv_mass[k / 3] * conv;
    vel[k] = v;
    if (drift) pos[k] += dt * v;
}

// Intramolecular support potential for the MD driver (not part of the
// intermolecular energy): O-H bonds and the H-O-H angle, harmonic or with the
// MM3-style anharmonic factors (anh = 1), and an optional Urey-Bradley H-H
// term; forces added to F in place.
//   bond  E = kb dr^2 (1 - cs dr + (7/12) cs^2 dr^2), cs = 2.55 / A
//   angle E = ka dth^2 (1 - 0.014 D + 5.6e-5 D^2 - 7e-7 D^3 + 9e-10 D^4), D = dth in degrees
//   UB    E = kub (r_HH - rub)^2
__device__ inline double bond_dEdr(double kb, double dr, int anh) {
    if (!anh) return 2.0 * kb * dr;
    const double cs = 2.55, c4 = (7.0 / 12.0) * cs * cs;
    // d/dr [dr^2 - cs dr^3 + c4 dr^4]
    return kb * (2.0 * dr - 3.0 * cs * dr * dr + 4.0 * c4 * dr * dr * dr);
}
__device__ inline double angle_dEdth(double ka, double dth, int anh) {
    if (!anh) return 2.0 * ka * dth;
    const double g = 180.0 / M_PI;   // degrees per radian
    const double D = dth * g;
    const double f = 1.0 - 0.014 * D + 5.6e-5 * D * D - 7.0e-7 * D * D * D + 9.0e-10 * D * D * D * D;
    const double dfdD = -0.014 + 2.0 * 5.6e-5 * D - 3.0 * 7.0e-7 * D * D + 4.0 * 9.0e-10 * D * D * D;
    return ka * (2.0 * dth * f + dth * dth * dfdD * g);
}

__global__ void k_water_intra(int M, const double *pos, double *F, double kb, double r0, double ka, double th0,
                              int anh, double kub, double rub) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double *x = pos + m * 9;
    const V3<double> O = mk(x[0], x[1], x[2]), H1 = mk(x[3], x[4], x[5]), H2 = mk(x[6], x[7], x[8]);
    const V3<double> a = H1 - O, b = H2 - O;
    const double ra = sqrt(dot(a, a)), rb = sqrt(dot(b, b));
    // bonds
    const V3<double> fa = (-bond_dEdr(kb, ra - r0, anh) / ra) * a;   // force on H1
    const V3<double> fb = (-bond_dEdr(kb, rb - r0, anh) / rb) * b;
    // angle
    const double c = fmax(-1.0, fmin(1.0, dot(a, b) / (ra * rb)));
    const double th = acos(c);
    const double s = fmax(sqrt(1.0 - c * c), 1e-8);
    const double dEdth = angle_dEdth(ka, th - th0, anh);
    // dtheta/da = -(b/(ra rb) - c a/ra^2)/sin
    const V3<double> dca = (1.0 / (ra * rb)) * b - (c / (ra * ra)) * a;
    const V3<double> dcb = (1.0 / (ra * rb)) * a - (c / (rb * rb)) * b;
    const V3<double> ga = (dEdth / s) * dca;     // -dE/da  (dtheta = -dc/sin)
    const V3<double> gb = (dEdth / s) * dcb;
    V3<double> f1 = fa + ga, f2 = fb + gb;
    if (kub > 0.0) {   // Urey-Bradley: force on H1 along H2 -> H1
        const V3<double> hh = H1 - H2;
        const double rhh = sqrt(dot(hh, hh));
        const V3<double> fu = (-2.0 * kub * (rhh - rub) / rhh) * hh;
        f1 = f1 + fu;
        f2 = f2 - fu;
    }
    double *f = F + m * 9;
    f[0] -= f1.x + f2.x; f[1] -= f1.y + f2.y; f[2] -= f1.z + f2.z;
    f[3] += f1.x; f[4] += f1.y; f[5] += f1.z;
    f[6] += f2.x; f[7] += f2.y; f[8] += f2.z;
}

// Capped steepest-descent update used to relax a starting structure:
// x += F * min(gamma, cap / |F|) per atom.
__global__ void k_sd_step(int M, double *pos, const double *F, double gamma, double cap) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= M * 3) return;
    const double fx = F[a * 3], fy = F[a * 3 + 1], fz = F[a * 3 + 2];
    const double f = sqrt(fx * fx + fy * fy + fz * fz);
    const double s = (f * gamma > cap) ? cap / f : gamma;
    pos[a * 3] += s * fx;
    pos[a * 3 + 1] += s * fy;
    pos[a * 3 + 2] += s * fz;
}

void launch_sd_step(int M, double *pos, const double *F, double gamma, double cap, Launch L) {
    k_sd_step<<<(M * 3 + 127) / 128, 128, 0, L.s>>>(M, pos, F, gamma, cap);
    count(L);
}

void launch_water_intra(int M, const double *pos, double *F, double kb, double r0, double ka, double th0, int anh,
                        double kub, double rub, Launch L) {
    k_water_intra<<<(M + 127) / 128, 128, 0, L.s>>>(M, pos, F, kb, r0, ka, th0, anh, kub, rub);
    count(L);
}

// Beeman integrator, first half: x += v dt + (4 a - a_prev) dt^2 / 6,
// v += (5 a - a_prev) dt / 6, then a_prev <- a (stored as forces).
__global__ void k_beeman1(int M, double *pos, double *vel, const double *inv_mass, const double *F, double *Fprev,
                          double dt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M * 9) return;
    const double conv = 4.184e-4;   // (kcal/mol/A)/amu -> A/fs^2
    const double im = inv_mass[k / 3] * conv;
    const double a = F[k] * im, ap = Fprev[k] * im;
    const double v = vel[k];
    pos[k] += v * dt + (4.0 * a - ap) * dt * dt * (1.0 / 6.0);
    vel[k] = v + (5.0 * a - ap) * dt * (1.0 / 6.0);
    Fprev[k] = F[k];
}
// second half, after the forces at t + dt: v += 2 a(t + dt) dt / 6
__global__ void k_beeman2(int M, double *vel, const double *inv_mass, const double *F, double dt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M * 9) return;
    vel[k] += 2.0 * F[k] * inv_mass[k / 3] * 4.184e-4 * dt * (1.0 / 6.0);
}
void launch_beeman(int M, double *pos, double *vel, const double *inv_mass, double *F, double *Fprev, double dt,
                   int half, Launch L) {
    if (half == 1) k_beeman1<<<(M * 9 + 255) / 256, 256, 0, L.s>>>(M, pos, vel, inv_mass, F, Fprev, dt);
    else k_beeman2<<<(M * 9 + 255) / 256, 256, 0, L.s>>>(M, vel, inv_mass, F, dt);
    count(L);
}

void launch_md_kick(int M, double *pos, double *vel, const double *inv_mass, const double *forces, double dt,
                    int drift, Launch L) {
    k_md_kick<<<(M * 9 + 255) / 256, 256, 0, L.s>>>(M, pos, vel, inv_mass, forces, dt, drift);
    count(L);
}

#define INST(R)                                                                                        \
    template void launch_pcg_init<R>(const KParams &, DevState<R> &, int, Launch);                     \
    template void launch_pcg_init_guess<R>(const KParams &, DevState<R> &, MuGuess, Launch);           \
    template void launch_pcg_first<R>(const KParams &, DevState<R> &, Launch);                         \
    template void launch_pcg_step<R>(const KParams &, DevState<R> &, Launch, cudaGraphConditionalHandle, int); \
    template void launch_pol_energy<R>(const KParams &, DevState<R> &, Launch);                        \
    template void launch_finalize<R>(const KParams &, DevState<R> &, double *, Launch);                \
    template void launch_merge_rec<R>(const KParams &, DevState<R> &, Launch);                         \
    template void launch_cluster_energy<R>(const KParams &, DevState<R> &, double *, Launch);           \
    template void launch_virial_total<R>(const KParams &, DevState<R> &, double *, Launch);
INST(float)
INST(double)

}  // namespace sibfa
