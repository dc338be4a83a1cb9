// Intramolecular Ewald corrections (FP64): the reciprocal sum contains every
// pair of sites, including those of the same molecule, and every site with
// itself; the intermolecular potential (Eq. 1) removes the erf part of those
// pairs and the Gaussian self terms.  One warp per molecule, one lane per
// site-pair task; contributions meet in shared memory.
#include "sibfa_internal.cuh"

namespace sibfa {

constexpr int IW = 4;   // molecules (warps) per block

struct IntraAcc {
    double gpt[NS][3];
    double gmu[NS][3];
    double gth[NS][6];
    double ef[3][3];
    double vlp[2];
    double dvlp[2][3];
    double e;
};
constexpr int IA_N = sizeof(IntraAcc) / sizeof(double);

__device__ inline void sadd3(double *a, V3<double> v, double s) {
    atomicAdd(a, s * v.x);
    atomicAdd(a + 1, s * v.y);
    atomicAdd(a + 2, s * v.z);
}
__device__ inline void sadd6(double *a, const Sym<double> &v, double s) {
    atomicAdd(a, s * v.xx);
    atomicAdd(a + 1, s * v.yy);
    atomicAdd(a + 2, s * v.zz);
    atomicAdd(a + 3, s * v.xy);
    atomicAdd(a + 4, s * v.xz);
    atomicAdd(a + 5, s * v.yz);
}

__device__ inline void zero_acc(IntraAcc &A, int lane) {
    double *z = (double *)&A;
    for (int k = lane; k < IA_N; k += 32) z[k] = 0.0;
}

// lane 0 builds the FP64 point positions of the molecule in shared memory
template <typename R>
__device__ inline void load_points(const KParams &p, const DevState<R> &d, int m, int lane, double (*sX)[3]) {
    if (lane == 0) {
        V3<double> X[NP];
        points_d(p, d, m, X);
        for (int k = 0; k < NP; ++k) {
            sX[k][0] = X[k].x;
            sX[k][1] = X[k].y;
            sX[k][2] = X[k].z;
        }
    }
    __syncwarp();
}

__device__ inline V3<double> pt(double (*sX)[3], int k) { return mk(sX[k][0], sX[k][1], sX[k][2]); }

__constant__ int c_pair10[10][2] = {{0, 1}, {0, 2}, {0, 3}, {0, 4}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}};

// Permanent pass.  Lanes 0-9: the 10 site pairs (energy, gradients and
// sensitivities of both sites); lanes 10-21: field on O/H1/H2 from the other
// 4 sites; lanes 22-31: lone-pair potential from the 5 sites.  Lanes 0-4 add
// the Gaussian self energy of their site, lanes 10/14/18 the self field.
template <typename R>
__global__ void __launch_bounds__(128) k_intra_perm(KParams p, DevState<R> d) {
    __shared__ IntraAcc acc[IW];
    __shared__ double sX[IW][NP][3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * IW + w;
    if (m >= p.M) return;
    IntraAcc &A = acc[w];
    zero_acc(A, lane);
    load_points(p, d, m, lane, sX[w]);
    const double ke = p.ke, al = p.alpha;
    const double cself = 4.0 * al * al * al / (3.0 * sqrt(M_PI));
    if (lane < 10) {
        const int t = c_pair10[lane][0], s = c_pair10[lane][1];
        const Mp<double> Mt = mp_d(d, m, t), Ms = mp_d(d, m, s);
        const V3<double> x = pt(sX[w], t) - pt(sX[w], s);
        double g[6];
        g_erf_d(sqrt(dot(x, x)), al, g);
        FieldTerms<double> f;
        source_field<double, 3>(Ms, x, g, f);
        atomicAdd(&A.e, -(Mt.q * f.phi + dot(Mt.mu, f.d1) + symdd(Mt.th, f.d2) / 3.0));
        const V3<double> gt = target_grad(Mt, Ms, x, g, f);
        sadd3(A.gpt[t], gt, -1.0);
        sadd3(A.gpt[s], gt, 1.0);
        sadd3(A.gmu[t], f.d1, -1.0);
        sadd6(A.gth[t], f.d2, -1.0 / 3.0);
        FieldTerms<double> f2;
        source_field<double, 2>(Mt, -x, g, f2);
        sadd3(A.gmu[s], f2.d1, -1.0);
        sadd6(A.gth[s], f2.d2, -1.0 / 3.0);
    } else if (lane < 22) {
        const int a = (lane - 10) / 4, k = (lane - 10) % 4;
        const int s = k < a ? k : k + 1;
        const Mp<double> Ms = mp_d(d, m, s);
        const V3<double> x = pt(sX[w], a) - pt(sX[w], s);
        double g[6];
        g_erf_d(sqrt(dot(x, x)), al, g);
        FieldTerms<double> f;
        source_field<double, 1>(Ms, x, g, f);
        V3<double> E = f.d1;
        if (k == 0) E = E + cself * mp_d(d, m, a).mu;
        sadd3(A.ef[a], E, 1.0);
    } else {
        const int l = (lane - 22) / 5, s = (lane - 22) % 5;
        const Mp<double> Ms = mp_d(d, m, s);
        const V3<double> x = pt(sX[w], 5 + l) - pt(sX[w], s);
        double g[6];
        g_erf_d(sqrt(dot(x, x)), al, g);
        FieldTerms<double> f;
        source_field<double, 1>(Ms, x, g, f);
        atomicAdd(&A.vlp[l], -f.phi);
        sadd3(A.dvlp[l], f.d1, -1.0);
    }
    if (lane < NS) {
        const Mp<double> M = mp_d(d, m, lane);
        const double self = M.q * M.q + (2.0 * al * al / 3.0) * dot(M.mu, M.mu) +
                            (8.0 * al * al * al * al / 45.0) * symdd(M.th, M.th);
        atomicAdd(&A.e, -self * al / sqrt(M_PI));
    }
    __syncwarp();
    for (int k = lane; k < NS * 3; k += 32) d.gpt[m * NP * 3 + k] += ke * (&A.gpt[0][0])[k];
    for (int k = lane; k < NS * 3; k += 32) d.gmu[m * NS * 3 + k] += ke * (&A.gmu[0][0])[k];
    for (int k = lane; k < NS * 6; k += 32) d.gth[m * NS * 6 + k] += ke * (&A.gth[0][0])[k];
    if (lane < 9) d.efield[m * 9 + lane] += (&A.ef[0][0])[lane];
    if (lane < 2) d.vlp[m * 2 + lane] += ke * A.vlp[lane];
    if (lane < 6) d.dvlp[m * 6 + lane] += ke * (&A.dvlp[0][0])[lane];
    if (lane == 0) d.epart[m * NTERM + T_ELEC] += ke * A.e;
}

template <typename R>
void launch_intra_perm(const KParams &p, DevState<R> &d, Launch L) {
    k_intra_perm<R><<<(p.M + IW - 1) / IW, 32 * IW, 0, L.s>>>(p, d);
    count(L);
}

// PCG product, intramolecular part: one thread per polarizable atom, out +=
// field from the other two atoms' dipoles minus its erf part, plus the self
// term of its own dipole.
template <typename R>
__global__ void k_intra_tmu(KParams p, DevState<R> d, const double *vec, double *out) {
    if (d.scal[7] != 0.0) return;   // solver already converged
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.M * 3) return;
    const int m = t / 3, a = t % 3;
    const double al = p.alpha;
    const double cself = 4.0 * al * al * al / (3.0 * sqrt(M_PI));
    const double *x = d.pos + m * 9;
    const V3<double> Xa = mk(x[a * 3], x[a * 3 + 1], x[a * 3 + 2]);
    V3<double> E = cself * mk(vec[m * 9 + a * 3], vec[m * 9 + a * 3 + 1], vec[m * 9 + a * 3 + 2]);
    for (int b = 0; b < 3; ++b) {
        if (b == a) continue;
        const V3<double> xv = Xa - mk(x[b * 3], x[b * 3 + 1], x[b * 3 + 2]);
        double g[6];
        g_erf_d(sqrt(dot(xv, xv)), al, g);
        Mp<double> s{};
        s.mu = mk(vec[m * 9 + b * 3], vec[m * 9 + b * 3 + 1], vec[m * 9 + b * 3 + 2]);
        FieldTerms<double> f;
        source_field<double, 1>(s, xv, g, f);
        E = E + f.d1;
    }
    out[m * 9 + a * 3] += E.x;
    out[m * 9 + a * 3 + 1] += E.y;
    out[m * 9 + a * 3 + 2] += E.z;
}

template <typename R>
void launch_intra_tmu(const KParams &p, DevState<R> &d, const double *vec, double *out, Launch L) {
    const int n = p.M * 3;
    k_intra_tmu<R><<<(n + 127) / 128, 128, 0, L.s>>>(p, d, vec, out);
    count(L);
}

__constant__ int c_pair3[3][2] = {{0, 1}, {0, 2}, {1, 2}};

// Force pass at fixed induced dipoles and lambda charges.  Lanes 0-11:
// induced dipole a with site s != a; lanes 12-14: induced-induced pairs;
// lanes 15-24: lambda charge l with site s; lanes 25-27: the self cross term
// (sensitivity of the permanent dipole of O/H1/H2).
template <typename R>
__global__ void __launch_bounds__(128) k_intra_polforce(KParams p, DevState<R> d) {
    __shared__ IntraAcc acc[IW];
    __shared__ double sX[IW][NP][3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * IW + w;
    if (m >= p.M) return;
    IntraAcc &A = acc[w];
    zero_acc(A, lane);
    load_points(p, d, m, lane, sX[w]);
    const double ke = p.ke, al = p.alpha;
    auto mu_of = [&](int a) { return mk(d.mu[m * 9 + a * 3], d.mu[m * 9 + a * 3 + 1], d.mu[m * 9 + a * 3 + 2]); };
    if (lane < 12) {
        const int a = lane / 4, k = lane % 4;
        const int s = k < a ? k : k + 1;
        const Mp<double> Ms = mp_d(d, m, s);
        const V3<double> mua = mu_of(a);
        const V3<double> x = pt(sX[w], a) - pt(sX[w], s);
        double g[6];
        g_erf_d(sqrt(dot(x, x)), al, g);
        FieldTerms<double> f;
        source_field<double, 2>(Ms, x, g, f);
        const V3<double> ga = symv(f.d2, mua);
        sadd3(A.gpt[a], ga, -1.0);
        sadd3(A.gpt[s], ga, 1.0);
        Mp<double> dip{};
        dip.mu = mua;
        FieldTerms<double> f2;
        source_field<double, 2>(dip, -x, g, f2);
        sadd3(A.gmu[s], f2.d1, -1.0);
        sadd6(A.gth[s], f2.d2, -1.0 / 3.0);
    } else if (lane < 15) {
        const int a = c_pair3[lane - 12][0], b = c_pair3[lane - 12][1];
        const V3<double> x = pt(sX[w], a) - pt(sX[w], b);
        double g[6];
        g_erf_d(sqrt(dot(x, x)), al, g);
        Mp<double> dip{};
        dip.mu = mu_of(b);
        FieldTerms<double> f;
        source_field<double, 2>(dip, x, g, f);
        const V3<double> ga = symv(f.d2, mu_of(a));
        sadd3(A.gpt[a], ga, -1.0);
        sadd3(A.gpt[b], ga, 1.0);
    } else if (lane < 25) {
        const int l = (lane - 15) / 5, s = (lane - 15) % 5;
        const double lq = d.lam[m * 2 + l];
        if (lq != 0.0) {
            const Mp<double> Ms = mp_d(d, m, s);
            const V3<double> x = pt(sX[w], s) - pt(sX[w], 5 + l);
            double g[6];
            g_erf_d(sqrt(dot(x, x)), al, g);
            Mp<double> c{};
            c.q = lq;
            FieldTerms<double> f;
            source_field<double, 3>(c, x, g, f);
            sadd3(A.gpt[s], target_grad(Ms, c, x, g, f), -1.0);
            sadd3(A.gmu[s], f.d1, -1.0);
            sadd6(A.gth[s], f.d2, -1.0 / 3.0);
        }
    } else if (lane < 28) {
        const int a = lane - 25;
        const double cself = 4.0 * al * al * al / (3.0 * sqrt(M_PI));
        sadd3(A.gmu[a], mu_of(a), -cself);
    }
    __syncwarp();
    for (int k = lane; k < NS * 3; k += 32) d.gpt[m * NP * 3 + k] += ke * (&A.gpt[0][0])[k];
    for (int k = lane; k < NS * 3; k += 32) d.gmu[m * NS * 3 + k] += ke * (&A.gmu[0][0])[k];
    for (int k = lane; k < NS * 6; k += 32) d.gth[m * NS * 6 + k] += ke * (&A.gth[0][0])[k];
}

template <typename R>
void launch_intra_polforce(const KParams &p, DevState<R> &d, Launch L) {
    k_intra_polforce<R><<<(p.M + IW - 1) / IW, 32 * IW, 0, L.s>>>(p, d);
    count(L);
}

#define INST(R)                                                                                         \
    template void launch_intra_perm<R>(const KParams &, DevState<R> &, Launch);                         \
    template void launch_intra_tmu<R>(const KParams &, DevState<R> &, const double *, double *, Launch); \
    template void launch_intra_polforce<R>(const KParams &, DevState<R> &, Launch);
INST(float)
INST(double)

}  // namespace sibfa
