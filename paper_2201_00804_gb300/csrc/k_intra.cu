// Intramolecular Ewald corrections: the reciprocal sum contains every pair of
// sites, including those of the same molecule, and every site with itself;
// the intermolecular potential (Eq. 1) removes the erf part of those pairs
// and the Gaussian self terms.  Arithmetic in the working precision R with
// the cancellation-free erf kernel (g_erf_s); displacements come from the
// per-molecule point offsets, so no large coordinates enter.  One warp per
// molecule, one lane per site-pair task; vector contributions meet through
// shared-memory atomics, energies through warp sums in FP64.
#include "sibfa_internal.cuh"

namespace sibfa {

constexpr int IW = 4;   // molecules (warps) per block

template <typename R>
struct IntraAcc {
    R gpt[NS][3];
    R gmu[NS][3];
    R gth[NS][6];
    R ef[3][3];
    R dvlp[2][3];
    R va[3], dva[3][3];   // original charge transfer: potential and gradient at O, H1, H2
};

template <typename R>
__device__ inline void sadd3(R *a, V3<R> v, R s) {
    atomicAdd(a, s * v.x);
    atomicAdd(a + 1, s * v.y);
    atomicAdd(a + 2, s * v.z);
}
template <typename R>
__device__ inline void sadd6(R *a, const Sym<R> &v, R s) {
    atomicAdd(a, s * v.xx);
    atomicAdd(a + 1, s * v.yy);
    atomicAdd(a + 2, s * v.zz);
    atomicAdd(a + 3, s * v.xy);
    atomicAdd(a + 4, s * v.xz);
    atomicAdd(a + 5, s * v.yz);
}

template <typename R>
__device__ inline void zero_acc(IntraAcc<R> &A, int lane) {
    R *z = (R *)&A;
    for (int k = lane; k < (int)(sizeof(IntraAcc<R>) / sizeof(R)); k += 32) z[k] = R(0);
    __syncwarp();
}

// position of point k of molecule m relative to its O
template <typename R>
__device__ inline V3<R> opt(const DevState<R> &d, int m, int k) {
    const R *o = d.off + (m * NP + k) * 3;
    return mk(o[0], o[1], o[2]);
}

// warp sum of the per-lane virials into vir[m] (scaled by ke)
template <typename R>
__device__ inline void vir_warp_out(const DevState<R> &d, int m, R (&W)[9], double ke, int lane) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        R v = W[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        W[k] = v;
    }
    if (lane < 9) {
        R v = W[0];
#pragma unroll
        for (int k = 1; k < 9; ++k)
            if (k == lane) v = W[k];
        d.vir[m * 9 + lane] += ke * double(v);
    }
}

__constant__ int c_pair10[10][2] = {{0, 1}, {0, 2}, {0, 3}, {0, 4}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}};

// Permanent pass.  Lanes 0-9: the 10 site pairs (energy, gradients and
// sensitivities of both sites); lanes 10-21: field on O/H1/H2 from the other
// 4 sites (with the original charge transfer also the potential and its
// gradient there, removed from the acceptor potentials together with the
// atom's own Gaussian self terms: the charge's potential 2 alpha / sqrt(pi)
// q and the dipole's potential gradient (4/3) alpha^3 / sqrt(pi) mu); lanes 22-31:
// lone-pair potential from the 5 sites.  Lanes 0-4 add the Gaussian self
// energy of their site, lanes 10/14/18 the self field.
template <typename R>
__global__ void __launch_bounds__(128) k_intra_perm(KParams p, DevState<R> d) {
    __shared__ IntraAcc<R> acc[IW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * IW + w;
    if (m >= p.M) return;
    IntraAcc<R> &A = acc[w];
    zero_acc(A, lane);
    const R al = sc<R>(p).alpha;
    const R spi = R(0.56418958354775628695);   // 1 / sqrt(pi)
    const R cself = R(4.0 / 3.0) * al * al * al * spi;
    R e = R(0), vl = R(0);
    R W[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // virial (p.vir)
    if (lane < 10) {
        const int t = c_pair10[lane][0], s = c_pair10[lane][1];
        const Mp<R> Mt = load_mp(d.gmp + (m * NS + t) * GMP), Ms = load_mp(d.gmp + (m * NS + s) * GMP);
        const V3<R> x = opt(d, m, t) - opt(d, m, s);
        R g[6];
        g_erf_s<R, 5>(dot(x, x), al, g);
        FieldTerms<R> f;
        source_field<R, 3>(Ms, x, g, f);
        e -= Mt.q * f.phi + dot(Mt.mu, f.d1) + symdd(Mt.th, f.d2) * R(1.0 / 3.0);
        const V3<R> gt = target_grad(Mt, Ms, x, g, f);
        sadd3(A.gpt[t], gt, R(-1));
        sadd3(A.gpt[s], gt, R(1));
        if (p.vir) vir_add(W, gt, x, R(-1));
        sadd3(A.gmu[t], f.d1, R(-1));
        sadd6(A.gth[t], f.d2, R(-1.0 / 3.0));
        FieldTerms<R> f2;
        source_field<R, 2>(Mt, -x, g, f2);
        sadd3(A.gmu[s], f2.d1, R(-1));
        sadd6(A.gth[s], f2.d2, R(-1.0 / 3.0));
    } else if (lane < 22) {
        const int a = (lane - 10) / 4, k = (lane - 10) % 4;
        const int s = k < a ? k : k + 1;
        const Mp<R> Ms = load_mp(d.gmp + (m * NS + s) * GMP);
        const V3<R> x = opt(d, m, a) - opt(d, m, s);
        R g[4];
        g_erf_s<R, 3>(dot(x, x), al, g);
        FieldTerms<R> f;
        source_field<R, 1>(Ms, x, g, f);
        V3<R> E = f.d1;
        R va = -f.phi;
        V3<R> dva = R(-1) * f.d1;
        if (k == 0) {
            const Mp<R> Ma = load_mp(d.gmp + (m * NS + a) * GMP);
            E = E + cself * Ma.mu;
            va -= R(2) * al * spi * Ma.q;
            // the own Gaussian dipole's potential gradient at its centre, cself mu
            dva = dva - cself * Ma.mu;
        }
        sadd3(A.ef[a], E, R(1));
        if (p.ct_orig) {
            atomicAdd(&A.va[a], va);
            sadd3(A.dva[a], dva, R(1));
        }
    } else {
        const int l = (lane - 22) / 5, s = (lane - 22) % 5;
        const Mp<R> Ms = load_mp(d.gmp + (m * NS + s) * GMP);
        const V3<R> x = opt(d, m, 5 + l) - opt(d, m, s);
        R g[4];
        g_erf_s<R, 3>(dot(x, x), al, g);
        FieldTerms<R> f;
        source_field<R, 1>(Ms, x, g, f);
        vl = -f.phi;
        sadd3(A.dvlp[l], f.d1, R(-1));
    }
    if (lane < NS) {
        const Mp<R> M = load_mp(d.gmp + (m * NS + lane) * GMP);
        const R self = M.q * M.q + (R(2.0 / 3.0) * al * al) * dot(M.mu, M.mu) +
                       (R(8.0 / 45.0) * al * al * al * al) * symdd(M.th, M.th);
        e -= self * al * spi;
    }
    const double ke = p.ke;
    // FP32 path: the energy comes from k_intra_energy64
    const double esum = sizeof(R) == 8 ? warp_sum(double(e)) : 0.0;
    // lanes 22-26 carry lone pair 0, lanes 27-31 lone pair 1
    const double v0 = warp_sum(lane < 27 ? double(vl) : 0.0);
    const double v1 = warp_sum(lane >= 27 ? double(vl) : 0.0);
    __syncwarp();
    for (int k = lane; k < NS * 3; k += 32) d.gpt[m * NP * 3 + k] += ke * double((&A.gpt[0][0])[k]);
    for (int k = lane; k < NS * 3; k += 32) d.gmu[m * NS * 3 + k] += ke * double((&A.gmu[0][0])[k]);
    for (int k = lane; k < NS * 6; k += 32) d.gth[m * NS * 6 + k] += ke * double((&A.gth[0][0])[k]);
    if (lane < 9) d.efield[m * 9 + lane] += double((&A.ef[0][0])[lane]);
    if (lane < 6) d.dvlp[m * 6 + lane] += ke * double((&A.dvlp[0][0])[lane]);
    if (p.ct_orig) {
        if (lane < 3) d.va[m * 3 + lane] += ke * double(A.va[lane]);
        if (lane < 9) d.dva[m * 9 + lane] += ke * double((&A.dva[0][0])[lane]);
    }
    if (lane == 0) {
        d.vlp[m * 2] += ke * v0;
        d.vlp[m * 2 + 1] += ke * v1;
        d.epart[m * NTERM + T_ELEC] += ke * esum;
    }
    // the lone pairs' share of the lambda-weighted virial is taken in the force pass
    if (p.vir) vir_warp_out(d, m, W, ke, lane);
}

// Mixed path: the intramolecular Ewald energy (erf part of the 10 site pairs
// of each molecule and the five Gaussian self terms) in FP64.  These terms
// are ~50 kcal/mol per molecule and cancel against the reciprocal sum; the
// same geometry repeats in every rigid molecule, so FP32 rounding of them
// adds up coherently over the box (about 1e-6 of the total energy at a few
// hundred waters).  The multipoles are the working-precision global ones the
// reciprocal grid was spread from (converted exactly to FP64), the site
// offsets FP64 differences of the positions; the radial kernels, products
// and sums are FP64 (the FP64 pipe bounds this kernel).  Sixteen lanes per
// molecule: lanes 0-4 stage the five sites in shared memory, then lanes 0-9
// take the pairs and lanes 10-14 the self terms.  It reads only positions
// and multipoles, so it runs on the lowest-priority stream beside the other
// kernels, and writes its own per-molecule array.
constexpr int IE_MOL = 8;   // molecules per 128-thread block
template <typename R>
__global__ void __launch_bounds__(128) k_intra_energy64(KParams p, const double *pos, const R *gmp, double *eintra) {
    __shared__ double sq[IE_MOL][NS], smu[IE_MOL][NS][3], sth[IE_MOL][NS][6], soff[IE_MOL][NS][3];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int lm = threadIdx.x >> 4, m = g >> 4, t = g & 15;
    const bool live = m < p.M;
    const double al = p.alpha, spi = 0.56418958354775628695;
    if (live && t < NS) {
        const R *gm = gmp + (m * NS + t) * GMP;
        sq[lm][t] = double(gm[0]);
        for (int k = 0; k < 3; ++k) smu[lm][t][k] = double(gm[1 + k]);
        for (int k = 0; k < 6; ++k) sth[lm][t][k] = double(gm[4 + k]);   // xx yy zz xy xz yz
        const double *x = pos + m * 9;
        // offsets from O: O, H1, H2, and the O-H midpoints
        const int h = t == 0 ? 0 : (t == 1 || t == 3 ? 1 : 2);
        const double f = t >= 3 ? 0.5 : 1.0;
        for (int k = 0; k < 3; ++k) soff[lm][t][k] = h ? f * (x[3 * h + k] - x[k]) : 0.0;
    }
    __syncthreads();
    auto site = [&](int k) {
        Mp<double> M;
        M.q = sq[lm][k];
        M.mu = mk(smu[lm][k][0], smu[lm][k][1], smu[lm][k][2]);
        M.th.xx = sth[lm][k][0]; M.th.yy = sth[lm][k][1]; M.th.zz = sth[lm][k][2];
        M.th.xy = sth[lm][k][3]; M.th.xz = sth[lm][k][4]; M.th.yz = sth[lm][k][5];
        return M;
    };
    double e = 0.0;
    if (live) {
        if (t < 10) {
            const int a = c_pair10[t][0], b = c_pair10[t][1];
            const Mp<double> Ma = site(a), Mb = site(b);
            const V3<double> xv = mk(soff[lm][a][0] - soff[lm][b][0], soff[lm][a][1] - soff[lm][b][1],
                                     soff[lm][a][2] - soff[lm][b][2]);
            double gg[5];   // source_field to second derivatives reads g_0..g_4
            g_erf_s<double, 4>(dot(xv, xv), al, gg);
            FieldTerms<double> f;
            source_field<double, 2>(Mb, xv, gg, f);
            e = -(Ma.q * f.phi + dot(Ma.mu, f.d1) + symdd(Ma.th, f.d2) * (1.0 / 3.0));
        } else if (t < 10 + NS) {
            const Mp<double> M = site(t - 10);
            const double self = M.q * M.q + (2.0 / 3.0) * al * al * dot(M.mu, M.mu) +
                                (8.0 / 45.0) * al * al * al * al * symdd(M.th, M.th);
            e = -self * al * spi;
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o, 16);
    if (live && t == 0) eintra[m] = p.ke * e;
}

template <typename R>
void launch_intra_energy64(const KParams &p, DevState<R> &d, Launch L) {
    k_intra_energy64<R><<<(p.M + IE_MOL - 1) / IE_MOL, 128, 0, L.s>>>(p, d.pos, d.gmp, d.eintra);
    count(L);
}

template <typename R>
void launch_intra_perm(const KParams &p, DevState<R> &d, Launch L) {
    k_intra_perm<R><<<(p.M + IW - 1) / IW, 32 * IW, 0, L.s>>>(p, d);
    count(L);
}

__constant__ int c_pair3[3][2] = {{0, 1}, {0, 2}, {1, 2}};

// Force pass at fixed induced dipoles and lambda charges.  Lanes 0-11:
// induced dipole a with site s != a; lanes 12-14: induced-induced pairs;
// lanes 15-24: lambda charge l with site s; lanes 25-27: the self cross term
// (sensitivity of the permanent dipole of O/H1/H2).
template <typename R>
__global__ void __launch_bounds__(128) k_intra_polforce(KParams p, DevState<R> d) {
    __shared__ IntraAcc<R> acc[IW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * IW + w;
    if (m >= p.M) return;
    IntraAcc<R> &A = acc[w];
    zero_acc(A, lane);
    const R al = sc<R>(p).alpha;
    R W[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // virial (p.vir)
    auto mu_of = [&](int a) {
        return mk(R(d.mu[m * 9 + a * 3]), R(d.mu[m * 9 + a * 3 + 1]), R(d.mu[m * 9 + a * 3 + 2]));
    };
    if (lane < 12) {
        const int a = lane / 4, k = lane % 4;
        const int s = k < a ? k : k + 1;
        const Mp<R> Ms = load_mp(d.gmp + (m * NS + s) * GMP);
        const V3<R> mua = mu_of(a);
        const V3<R> x = opt(d, m, a) - opt(d, m, s);
        R g[5];
        g_erf_s<R, 4>(dot(x, x), al, g);
        FieldTerms<R> f;
        source_field<R, 2>(Ms, x, g, f);
        const V3<R> ga = symv(f.d2, mua);
        sadd3(A.gpt[a], ga, R(-1));
        sadd3(A.gpt[s], ga, R(1));
        if (p.vir) vir_add(W, ga, x, R(-1));
        Mp<R> dip{};
        dip.mu = mua;
        FieldTerms<R> f2;
        source_field<R, 2>(dip, -x, g, f2);
        sadd3(A.gmu[s], f2.d1, R(-1));
        sadd6(A.gth[s], f2.d2, R(-1.0 / 3.0));
    } else if (lane < 15) {
        const int a = c_pair3[lane - 12][0], b = c_pair3[lane - 12][1];
        const V3<R> x = opt(d, m, a) - opt(d, m, b);
        R g[5];
        g_erf_s<R, 4>(dot(x, x), al, g);
        Mp<R> dip{};
        dip.mu = mu_of(b);
        FieldTerms<R> f;
        source_field<R, 2>(dip, x, g, f);
        const V3<R> ga = symv(f.d2, mu_of(a));
        sadd3(A.gpt[a], ga, R(-1));
        sadd3(A.gpt[b], ga, R(1));
        if (p.vir) vir_add(W, ga, x, R(-1));
    } else if (lane < 25) {
        const int l = (lane - 15) / 5, s = (lane - 15) % 5;
        const double lq = d.lam[m * 2 + l];
        if (lq != 0.0) {
            const Mp<R> Ms = load_mp(d.gmp + (m * NS + s) * GMP);
            const V3<R> x = opt(d, m, s) - opt(d, m, 5 + l);
            R g[6];
            g_erf_s<R, 5>(dot(x, x), al, g);
            Mp<R> c{};
            c.q = R(lq);
            FieldTerms<R> f;
            source_field<R, 3>(c, x, g, f);
            const V3<R> tg = target_grad(Ms, c, x, g, f);
            sadd3(A.gpt[s], tg, R(-1));
            if (p.vir) vir_add(W, tg, x, R(-1));   // the whole (site, lambda) pair
            sadd3(A.gmu[s], f.d1, R(-1));
            sadd6(A.gth[s], f.d2, R(-1.0 / 3.0));
        }
    } else if (lane < 28) {
        const int a = lane - 25;
        const R cself = R(4.0 / 3.0) * al * al * al * R(0.56418958354775628695);
        sadd3(A.gmu[a], mu_of(a), -cself);
    }
    // original charge transfer: the charges dE/dV(a) on O, H1, H2 were spread
    // with the lone-pair lambdas; remove their erf part at the molecule's
    // other four sites, and at the atom's own site the gradient d2 . mu that
    // the charge's own Gaussian (field gradient -(4/3) alpha^3 / sqrt(pi) I at
    // its centre) gives its dipole
    if (p.ct_orig && lane >= 25 && lane < 28) {
        const int a = lane - 25;
        const R cself = R(4.0 / 3.0) * al * al * al * R(0.56418958354775628695);
        const Mp<R> Ma = load_mp(d.gmp + (m * NS + a) * GMP);
        sadd3(A.gpt[a], Ma.mu, cself * R(d.lama[m * 3 + a]));
    }
    if (p.ct_orig && lane < 12) {
        const int a = lane / 4, k = lane % 4;
        const int s = k < a ? k : k + 1;
        const double lq = d.lama[m * 3 + a];
        if (lq != 0.0) {
            const Mp<R> Ms = load_mp(d.gmp + (m * NS + s) * GMP);
            const V3<R> x = opt(d, m, s) - opt(d, m, a);
            R g[6];
            g_erf_s<R, 5>(dot(x, x), al, g);
            Mp<R> c{};
            c.q = R(lq);
            FieldTerms<R> f;
            source_field<R, 3>(c, x, g, f);
            sadd3(A.gpt[s], target_grad(Ms, c, x, g, f), R(-1));
            sadd3(A.gmu[s], f.d1, R(-1));
            sadd6(A.gth[s], f.d2, R(-1.0 / 3.0));
        }
    }
    const double ke = p.ke;
    __syncwarp();
    for (int k = lane; k < NS * 3; k += 32) d.gpt[m * NP * 3 + k] += ke * double((&A.gpt[0][0])[k]);
    for (int k = lane; k < NS * 3; k += 32) d.gmu[m * NS * 3 + k] += ke * double((&A.gmu[0][0])[k]);
    for (int k = lane; k < NS * 6; k += 32) d.gth[m * NS * 6 + k] += ke * double((&A.gth[0][0])[k]);
    if (p.vir) vir_warp_out(d, m, W, ke, lane);
}

template <typename R>
void launch_intra_polforce(const KParams &p, DevState<R> &d, Launch L) {
    k_intra_polforce<R><<<(p.M + IW - 1) / IW, 32 * IW, 0, L.s>>>(p, d);
    count(L);
}

#define INST(R)                                                                                         \
    template void launch_intra_perm<R>(const KParams &, DevState<R> &, Launch);                         \
    template void launch_intra_polforce<R>(const KParams &, DevState<R> &, Launch);                     \
    template void launch_intra_energy64<R>(const KParams &, DevState<R> &, Launch);
INST(float)
INST(double)

}  // namespace sibfa
