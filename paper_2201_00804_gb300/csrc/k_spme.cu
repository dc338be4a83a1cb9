// Smooth particle mesh Ewald of order 5 for point multipoles (Computational
// Details: SPME for multipoles and polarization).  Spread applies the
// multipole operator q + mu.grad + (1/3) Theta:grad grad to the B-spline
// weights, the FFT is cuFFT, the convolution multiplies by the FP64
// influence function, and the gather returns the potential and its first
// three derivatives from the same weights.
#include "sibfa_internal.cuh"

namespace sibfa {

// Per-dimension spline data of one point: grid indices and weights with
// Cartesian derivatives up to NDER.
template <typename R, int NDER>
struct Spl {
    int idx[3][ORDER];
    R w[NDER + 1][3][ORDER];
};

template <typename R, int NDER>
__device__ inline void spline_point(const KParams &p, double x, double y, double z, Spl<R, NDER> &s) {
    const double xyz[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double u = xyz[d] * (double)p.K[d] / p.box[d];
        const double fl = floor(u);
        const R w = R(u - fl);
        int base = (int)fl;
        base %= p.K[d];
        if (base < 0) base += p.K[d];
        R m0[ORDER], m1[ORDER], m2[ORDER], m3[ORDER];
        bspline5<R, NDER>(w, m0, m1, m2, m3);
        const R sc = R((double)p.K[d] / p.box[d]);
#pragma unroll
        for (int j = 0; j < ORDER; ++j) {
            int g = base - j;
            if (g < 0) g += p.K[d];
            s.idx[d][j] = g;
            s.w[0][d][j] = m0[j];
            if constexpr (NDER >= 1) s.w[1][d][j] = m1[j] * sc;
            if constexpr (NDER >= 2) s.w[2][d][j] = m2[j] * sc * sc;
            if constexpr (NDER >= 3) s.w[3][d][j] = m3[j] * sc * sc * sc;
        }
    }
}

// absolute position of point pt of molecule m
template <typename R>
__device__ inline void abs_point(const DevState<R> &d, int m, int pt, double &x, double &y, double &z) {
    x = d.pos[m * 9 + 0] + (double)d.off[(m * NP + pt) * 3 + 0];
    y = d.pos[m * 9 + 1] + (double)d.off[(m * NP + pt) * 3 + 1];
    z = d.pos[m * 9 + 2] + (double)d.off[(m * NP + pt) * 3 + 2];
}

// kind PERM: 5 sites per molecule with their multipoles;
// kind DIP: 3 polarizable atoms with dipoles vec[m*9 + a*3 + c];
// kind LAMBDA: 2 lone pairs with charges d.lam.
template <typename R>
__global__ void k_spread(KParams p, DevState<R> d, int kind, const double *vec, R *grid) {
    if (kind == SPREAD_DIP_PCG) {
        if (d.scal[7] != 0.0) return;   // solver already converged
        kind = SPREAD_DIP;
    }
    const int per = kind == SPREAD_PERM ? NS : (kind == SPREAD_DIP ? 3 : 2);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.M * per) return;
    const int m = t / per, a = t % per;
    const int pt = kind == SPREAD_LAMBDA ? 5 + a : a;
    Mp<R> mp{};
    if (kind == SPREAD_PERM) mp = load_mp(d.gmp + (m * NS + a) * NMP);
    else if (kind == SPREAD_DIP) mp.mu = mk(R(vec[m * 9 + a * 3]), R(vec[m * 9 + a * 3 + 1]), R(vec[m * 9 + a * 3 + 2]));
    else mp.q = R(d.lam[m * 2 + a]);
    double x, y, z;
    abs_point(d, m, pt, x, y, z);
    Spl<R, 2> s;
    spline_point<R, 2>(p, x, y, z, s);
    const R third = R(1) / R(3);
    const int K1 = p.K[1], K2 = p.K[2];
    for (int i = 0; i < ORDER; ++i) {
        const R wx0 = s.w[0][0][i], wx1 = s.w[1][0][i], wx2 = s.w[2][0][i];
        for (int j = 0; j < ORDER; ++j) {
            const R wy0 = s.w[0][1][j], wy1 = s.w[1][1][j], wy2 = s.w[2][1][j];
            // coefficients of the z weights (0th, 1st, 2nd derivative)
            const R c0 = mp.q * wx0 * wy0 + mp.mu.x * wx1 * wy0 + mp.mu.y * wx0 * wy1 +
                         third * (mp.th.xx * wx2 * wy0 + mp.th.yy * wx0 * wy2 + R(2) * mp.th.xy * wx1 * wy1);
            const R c1 = mp.mu.z * wx0 * wy0 + third * R(2) * (mp.th.xz * wx1 * wy0 + mp.th.yz * wx0 * wy1);
            const R c2 = third * mp.th.zz * wx0 * wy0;
            const size_t row = ((size_t)s.idx[0][i] * K1 + s.idx[1][j]) * K2;
            for (int k = 0; k < ORDER; ++k) {
                const R v = c0 * s.w[0][2][k] + c1 * s.w[1][2][k] + c2 * s.w[2][2][k];
                atomicAdd(&grid[row + s.idx[2][k]], v);
            }
        }
    }
}

template <typename R>
void launch_spread(const KParams &p, DevState<R> &d, int kind, const double *vec, R *grid, Launch L) {
    const int per = kind == SPREAD_PERM ? NS : ((kind == SPREAD_DIP || kind == SPREAD_DIP_PCG) ? 3 : 2);
    const int n = p.M * per;
    k_spread<R><<<(n + 127) / 128, 128, 0, L.s>>>(p, d, kind, vec, grid);
    count(L);
}

// multiply the half-complex spectrum (ngrid grids back to back) by the influence function
template <typename R, typename C>
__global__ void k_convolve(KParams p, const double *infl, C *cg, int ngrid, const double *scal, int check) {
    if (check && scal[7] != 0.0) return;
    const size_t nh = (size_t)p.K[0] * p.K[1] * (p.K[2] / 2 + 1);
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nh * ngrid) return;
    const double g = infl[t % nh];
    C c = cg[t];
    c.x = R(double(c.x) * g);
    c.y = R(double(c.y) * g);
    cg[t] = c;
}

template <typename R>
void launch_convolve(const KParams &p, DevState<R> &d, void *cgrid, int ngrid, int check, Launch L) {
    const size_t nh = (size_t)p.K[0] * p.K[1] * (p.K[2] / 2 + 1);
    const size_t n = nh * ngrid;
    if (sizeof(R) == 4)
        k_convolve<float, cufftComplex><<<(unsigned)((n + 255) / 256), 256, 0, L.s>>>(p, d.infl, (cufftComplex *)cgrid,
                                                                                    ngrid, d.scal, check);
    else
        k_convolve<double, cufftDoubleComplex><<<(unsigned)((n + 255) / 256), 256, 0, L.s>>>(
            p, d.infl, (cufftDoubleComplex *)cgrid, ngrid, d.scal, check);
    count(L);
}

// Influence function G(m) = ke exp(-pi^2 m~^2/alpha^2) B(m) / (pi V m~^2), G(0) = 0, with the
// Euler-spline moduli B(m) = prod_d |b_d(m_d)|^2; a vanishing modulus denominator
// (m = K/2 for odd orders) takes the mean of its neighbours.
__device__ inline double bmod_den(int m, int K) {
    // sum_{k=0}^{3} M_5(k+1) exp(2 pi i m k / K), M_5(1..4) = (1, 11, 11, 1)/24
    const double Mk[4] = {1.0 / 24, 11.0 / 24, 11.0 / 24, 1.0 / 24};
    double re = 0, im = 0;
    for (int k = 0; k < 4; ++k) {
        double ph = 2.0 * M_PI * (double)m * k / K;
        re += Mk[k] * cos(ph);
        im += Mk[k] * sin(ph);
    }
    return re * re + im * im;
}
__device__ inline double bmod(int m, int K) {
    double den = bmod_den(m, K);
    if (den < 1e-7) den = 0.5 * (bmod_den((m + K - 1) % K, K) + bmod_den((m + 1) % K, K));
    return 1.0 / den;
}

__global__ void k_influence(KParams p, double *infl) {
    const int nz = p.K[2] / 2 + 1;
    const size_t n = (size_t)p.K[0] * p.K[1] * nz;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int kz = t % nz, ky = (t / nz) % p.K[1], kx = t / ((size_t)nz * p.K[1]);
    const int mx = kx <= p.K[0] / 2 ? kx : kx - p.K[0];
    const int my = ky <= p.K[1] / 2 ? ky : ky - p.K[1];
    const int mz = kz;
    const double fx = mx / p.box[0], fy = my / p.box[1], fz = mz / p.box[2];
    const double m2 = fx * fx + fy * fy + fz * fz;
    if (m2 == 0.0) {
        infl[t] = 0.0;
        return;
    }
    const double V = p.box[0] * p.box[1] * p.box[2];
    const double B = bmod(kx, p.K[0]) * bmod(ky, p.K[1]) * bmod(kz, p.K[2]);
    infl[t] = p.ke * exp(-M_PI * M_PI * m2 / (p.alpha * p.alpha)) * B / (M_PI * V * m2);
}

void launch_influence(const KParams &p, double *infl, Launch L) {
    const size_t n = (size_t)p.K[0] * p.K[1] * (p.K[2] / 2 + 1);
    k_influence<<<(unsigned)((n + 255) / 256), 256, 0, L.s>>>(p, infl);
    count(L);
}

// ---------------------------------------------------------------------------
// Gather: potential derivatives at a point from a convolved grid.
// ---------------------------------------------------------------------------
template <typename R>
struct Derivs {
    R phi;
    R d1[3];
    R d2[6];    // xx yy zz xy xz yz
    R d3[10];   // xxx yyy zzz xxy xxz xyy yyz xzz yzz xyz
};

template <typename R, int NDER>
__device__ inline void gather_point(const KParams &p, const R *grid, const Spl<R, NDER> &s, Derivs<R> &D) {
    D = Derivs<R>{};
    const int K1 = p.K[1], K2 = p.K[2];
    for (int i = 0; i < ORDER; ++i) {
        for (int j = 0; j < ORDER; ++j) {
            const size_t row = ((size_t)s.idx[0][i] * K1 + s.idx[1][j]) * K2;
            R t0 = 0, t1 = 0, t2 = 0, t3 = 0;   // sums over z with z-derivative order 0..3
            for (int k = 0; k < ORDER; ++k) {
                const R g = grid[row + s.idx[2][k]];
                t0 += g * s.w[0][2][k];
                if constexpr (NDER >= 1) t1 += g * s.w[1][2][k];
                if constexpr (NDER >= 2) t2 += g * s.w[2][2][k];
                if constexpr (NDER >= 3) t3 += g * s.w[3][2][k];
            }
            const R x0 = s.w[0][0][i], y0 = s.w[0][1][j];
            D.phi += x0 * y0 * t0;
            if constexpr (NDER >= 1) {
                const R x1 = s.w[1][0][i], y1 = s.w[1][1][j];
                D.d1[0] += x1 * y0 * t0;
                D.d1[1] += x0 * y1 * t0;
                D.d1[2] += x0 * y0 * t1;
                if constexpr (NDER >= 2) {
                    const R x2 = s.w[2][0][i], y2 = s.w[2][1][j];
                    D.d2[0] += x2 * y0 * t0;
                    D.d2[1] += x0 * y2 * t0;
                    D.d2[2] += x0 * y0 * t2;
                    D.d2[3] += x1 * y1 * t0;
                    D.d2[4] += x1 * y0 * t1;
                    D.d2[5] += x0 * y1 * t1;
                    if constexpr (NDER >= 3) {
                        const R x3 = s.w[3][0][i], y3 = s.w[3][1][j];
                        D.d3[0] += x3 * y0 * t0;
                        D.d3[1] += x0 * y3 * t0;
                        D.d3[2] += x0 * y0 * t3;
                        D.d3[3] += x2 * y1 * t0;
                        D.d3[4] += x2 * y0 * t1;
                        D.d3[5] += x1 * y2 * t0;
                        D.d3[6] += x0 * y2 * t1;
                        D.d3[7] += x1 * y0 * t2;
                        D.d3[8] += x0 * y1 * t2;
                        D.d3[9] += x1 * y1 * t1;
                    }
                }
            }
        }
    }
}

// full third-derivative tensor entry (a, b, c) from the 10 unique components
template <typename R>
__device__ inline R d3at(const Derivs<R> &D, int a, int b, int c) {
    int n[3] = {0, 0, 0};
    n[a]++; n[b]++; n[c]++;
    if (n[0] == 3) return D.d3[0];
    if (n[1] == 3) return D.d3[1];
    if (n[2] == 3) return D.d3[2];
    if (n[0] == 2 && n[1] == 1) return D.d3[3];
    if (n[0] == 2 && n[2] == 1) return D.d3[4];
    if (n[1] == 2 && n[0] == 1) return D.d3[5];
    if (n[1] == 2 && n[2] == 1) return D.d3[6];
    if (n[2] == 2 && n[0] == 1) return D.d3[7];
    if (n[2] == 2 && n[1] == 1) return D.d3[8];
    return D.d3[9];
}

template <typename R>
__device__ inline R sym_at(const R *s6, int a, int b) {
    if (a == b) return s6[a];
    int k = a + b;   // 1: xy, 2: xz, 3: yz
    return s6[2 + k];
}

// dU/dr for a multipole sitting in the gathered potential:
// q d1 + d2 . mu + (1/3) Theta : d3
template <typename R>
__device__ inline void mp_grad(const Mp<R> &m, const Derivs<R> &D, R out[3]) {
    const R th[6] = {m.th.xx, m.th.yy, m.th.zz, m.th.xy, m.th.xz, m.th.yz};
    const R mu[3] = {m.mu.x, m.mu.y, m.mu.z};
    for (int a = 0; a < 3; ++a) {
        R v = m.q * D.d1[a];
        for (int b = 0; b < 3; ++b) v += sym_at(D.d2, a, b) * mu[b];
        R t = 0;
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) t += sym_at(th, b, c) * d3at(D, a, b, c);
        out[a] = v + t / R(3);
    }
}

template <typename R>
__device__ inline R mp_energy(const Mp<R> &m, const Derivs<R> &D) {
    const Sym<R> d2{D.d2[0], D.d2[1], D.d2[2], D.d2[3], D.d2[4], D.d2[5]};
    return m.q * D.phi + m.mu.x * D.d1[0] + m.mu.y * D.d1[1] + m.mu.z * D.d1[2] + symdd(m.th, d2) / R(3);
}

// Permanent pass: 8 threads per molecule (points 0..6 used).  Sites: energy,
// gradient, multipole sensitivities; O/H1/H2 also their field and Hessian;
// lone pairs: potential and its gradient.
template <typename R>
__global__ void k_gather_perm(KParams p, DevState<R> d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = t >> 3, pt = t & 7;
    double e = 0.0;
    if (m < p.M && pt < NP) {
        double x, y, z;
        abs_point(d, m, pt, x, y, z);
        Derivs<R> D;
        if (pt < NS) {
            Spl<R, 3> s;
            spline_point<R, 3>(p, x, y, z, s);
            gather_point<R, 3>(p, d.grid, s, D);
            const Mp<R> mp = load_mp(d.gmp + (m * NS + pt) * NMP);
            e = 0.5 * (double)mp_energy(mp, D);
            R g[3];
            mp_grad(mp, D, g);
            double *gp = d.gpt + (m * NP + pt) * 3;
            double *gm = d.gmu + (m * NS + pt) * 3;
            double *gt = d.gth + (m * NS + pt) * 6;
            for (int a = 0; a < 3; ++a) {
                gp[a] += (double)g[a];
                gm[a] += (double)D.d1[a];
            }
            for (int k = 0; k < 6; ++k) gt[k] += (double)D.d2[k] / 3.0;
            if (pt < 3) {
                for (int a = 0; a < 3; ++a) d.efield[m * 9 + pt * 3 + a] -= (double)D.d1[a] / p.ke;
                for (int k = 0; k < 6; ++k) d.d2rec[m * 18 + pt * 6 + k] = (double)D.d2[k];
            }
        } else {
            Spl<R, 1> s;
            spline_point<R, 1>(p, x, y, z, s);
            gather_point<R, 1>(p, d.grid, s, D);
            const int l = pt - NS;
            d.vlp[m * 2 + l] += (double)D.phi;
            for (int a = 0; a < 3; ++a) d.dvlp[(m * 2 + l) * 3 + a] += (double)D.d1[a];
        }
    }
    // sum the 8 lanes of this molecule
    for (int o = 4; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o, 8);
    if (m < p.M && pt == 0) d.epart[m * NTERM + T_ELEC] += e;
}

template <typename R>
void launch_gather_perm(const KParams &p, DevState<R> &d, Launch L) {
    const int n = p.M * 8;
    k_gather_perm<R><<<(n + 127) / 128, 128, 0, L.s>>>(p, d);
    count(L);
}

// Field on the polarizable atoms from the dipole grid: out += -grad phi / ke.
template <typename R>
__global__ void k_gather_field(KParams p, DevState<R> d, double *out) {
    if (d.scal[7] != 0.0) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.M * 3) return;
    const int m = t / 3, a = t % 3;
    double x, y, z;
    abs_point(d, m, a, x, y, z);
    Spl<R, 1> s;
    spline_point<R, 1>(p, x, y, z, s);
    Derivs<R> D;
    gather_point<R, 1>(p, d.grid, s, D);
    for (int c = 0; c < 3; ++c) out[m * 9 + a * 3 + c] -= (double)D.d1[c] / p.ke;
}

template <typename R>
void launch_gather_field(const KParams &p, DevState<R> &d, double *out, Launch L) {
    const int n = p.M * 3;
    k_gather_field<R><<<(n + 127) / 128, 128, 0, L.s>>>(p, d, out);
    count(L);
}

// Force pass: grid 0 holds the induced dipoles, grid 1 the lambda charges.
// Sites: gradient and sensitivities of the permanent multipoles in the sum of
// both potentials.  O/H1/H2: gradient of the induced dipole in the induced
// (grid 0) and permanent (stored Hessian) reciprocal potentials.
template <typename R>
__global__ void k_gather_polforce(KParams p, DevState<R> d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.M * NS) return;
    const int m = t / NS, pt = t % NS;
    const size_t ng = (size_t)p.K[0] * p.K[1] * p.K[2];
    double x, y, z;
    abs_point(d, m, pt, x, y, z);
    Spl<R, 3> s;
    spline_point<R, 3>(p, x, y, z, s);
    Derivs<R> A, B;
    gather_point<R, 3>(p, d.grid, s, A);
    gather_point<R, 3>(p, d.grid + ng, s, B);
    Derivs<R> S;
    S.phi = A.phi + B.phi;
    for (int k = 0; k < 3; ++k) S.d1[k] = A.d1[k] + B.d1[k];
    for (int k = 0; k < 6; ++k) S.d2[k] = A.d2[k] + B.d2[k];
    for (int k = 0; k < 10; ++k) S.d3[k] = A.d3[k] + B.d3[k];
    const Mp<R> mp = load_mp(d.gmp + (m * NS + pt) * NMP);
    R g[3];
    mp_grad(mp, S, g);
    double *gp = d.gpt + (m * NP + pt) * 3;
    double *gm = d.gmu + (m * NS + pt) * 3;
    double *gt = d.gth + (m * NS + pt) * 6;
    for (int a = 0; a < 3; ++a) {
        gp[a] += (double)g[a];
        gm[a] += (double)S.d1[a];
    }
    for (int k = 0; k < 6; ++k) gt[k] += (double)S.d2[k] / 3.0;
    if (pt < 3) {
        const double mu[3] = {d.mu[m * 9 + pt * 3], d.mu[m * 9 + pt * 3 + 1], d.mu[m * 9 + pt * 3 + 2]};
        const double *h = d.d2rec + m * 18 + pt * 6;
        for (int a = 0; a < 3; ++a) {
            double v = 0;
            for (int b = 0; b < 3; ++b) v += ((double)sym_at(A.d2, a, b) + sym_at(h, a, b)) * mu[b];
            gp[a] += v;
        }
    }
}

template <typename R>
void launch_gather_polforce(const KParams &p, DevState<R> &d, Launch L) {
    const int n = p.M * NS;
    k_gather_polforce<R><<<(n + 127) / 128, 128, 0, L.s>>>(p, d);
    count(L);
}

#define INST(R)                                                                                         \
    template void launch_spread<R>(const KParams &, DevState<R> &, int, const double *, R *, Launch);    \
    template void launch_convolve<R>(const KParams &, DevState<R> &, void *, int, int, Launch);               \
    template void launch_gather_perm<R>(const KParams &, DevState<R> &, Launch);                         \
    template void launch_gather_field<R>(const KParams &, DevState<R> &, double *, Launch);              \
    template void launch_gather_polforce<R>(const KParams &, DevState<R> &, Launch);
INST(float)
INST(double)

}  // namespace sibfa
