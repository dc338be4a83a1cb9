// Smooth particle mesh Ewald of order 5 for point multipoles (Computational
// Details: SPME for multipoles and polarization).  Spread applies the
// multipole operator q + mu.grad + (1/3) Theta:grad grad to the B-spline
// weights, the FFT is cuFFT, the convolution multiplies by the FP64
// influence function, and the gather returns the potential and its first
// three derivatives from the same weights.
#include "sibfa_internal.cuh"

namespace sibfa {

// B-spline weights of one point along one axis at the 5 grid lines
// base - j (j = 0..4), with Cartesian derivatives up to NDER (scaled by K/L).
template <typename R, int NDER>
struct Axis {
    int g[ORDER];
    R w[NDER + 1][ORDER];
};

template <typename R, int NDER>
__device__ inline void axis_weights(const KParams &p, const DevState<R> &d, int m, int pt, int c, Axis<R, NDER> &A) {
    const int K = p.K[c];
    const int b = d.sbase[(m * NP + pt) * 3 + c];
    const R u = d.sfrac[(m * NP + pt) * 3 + c];
    R m0[ORDER], m1[ORDER], m2[ORDER], m3[ORDER];
    bspline5<R, NDER>(u, m0, m1, m2, m3);
    const R scl = sc<R>(p).kl[c];
#pragma unroll
    for (int j = 0; j < ORDER; ++j) {
        const int g = b - j;
        A.g[j] = g < 0 ? g + K : g;
        A.w[0][j] = m0[j];
        if constexpr (NDER >= 1) A.w[1][j] = m1[j] * scl;
        if constexpr (NDER >= 2) A.w[2][j] = m2[j] * scl * scl;
        if constexpr (NDER >= 3) A.w[3][j] = m3[j] * scl * scl * scl;
    }
}

// weights of stencil line i only (x or y axis of a lane's row)
template <typename R, int NDER>
__device__ inline void line_weight(const Axis<R, NDER> &A, int i, int &g, R (&w)[NDER + 1]) {
    g = A.g[0];
#pragma unroll
    for (int n = 0; n <= NDER; ++n) w[n] = A.w[n][0];
#pragma unroll
    for (int j = 1; j < ORDER; ++j)
        if (j == i) {
            g = A.g[j];
#pragma unroll
            for (int n = 0; n <= NDER; ++n) w[n] = A.w[n][j];
        }
}

// Spread and PCG-gather layout: a group of PG = 8 lanes per point (4 points
// per warp).  Lanes 0-4 of a group own the x-lines i = 0..4 of the 5x5x5
// stencil (25 grid points each); lanes 5-7 take per-point work that does
// not touch the grid.  The lanes of a group reduce with shuffles.
constexpr int PG = 8;

// Adds v[k] at the grid points row + zg[k] (k = 0..4, zg[k] = b - k modulo
// K2).  In FP32, when the row length is a multiple of 4 and the five points
// do not wrap, the values go as two aligned 4-wide vector reductions over the
// 8 points from the 4-aligned index at or below b - 4 (the three free slots
// add zero): 2 atomic operations instead of 5.
template <typename R>
__device__ inline void add_zline(R *grid, size_t row, int K2, const int (&zg)[ORDER], const R (&v)[ORDER]) {
    if constexpr (sizeof(R) == 4) {
        if ((K2 & 3) == 0 && zg[0] >= ORDER - 1) {
            const int zlo = zg[0] - (ORDER - 1), a0 = zlo & ~3, r = zlo - a0;
            // u: values at increasing z from zlo, then shifted up by r (0..3)
            float u[8] = {v[4], v[3], v[2], v[1], v[0], 0.f, 0.f, 0.f};
            float t[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) t[o] = (r & 1) ? (o >= 1 ? u[o - 1] : 0.f) : u[o];
#pragma unroll
            for (int o = 0; o < 8; ++o) u[o] = (r & 2) ? (o >= 2 ? t[o - 2] : 0.f) : t[o];
            float4 *g4 = reinterpret_cast<float4 *>(grid + row + a0);
            atomicAdd(g4, make_float4(u[0], u[1], u[2], u[3]));
            atomicAdd(g4 + 1, make_float4(u[4], u[5], u[6], u[7]));
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < ORDER; ++k) atomicAdd(&grid[row + zg[k]], v[k]);
}

// Spread: lane i < 5 of a point's group adds the multipole operator
// q + mu.grad + (1/3) Theta:grad grad applied to the B-spline weights at the
// 25 grid points of x-line i.
// kind PERM: 5 sites per molecule with their multipoles;
// kind DIP: 3 polarizable atoms with the induced dipoles (d.muR);
// kind DIP_PCG: the same from the working-precision PCG vector;
// kind LAMBDA: 2 lone pairs with the charge-transfer lambdas (d.lamR), and
// with the original charge transfer also O, H1, H2 with dE/dV(a) (d.lamaR).
// NDER: derivative order the multipoles need (2: quadrupoles, 1: dipoles, 0: charges).
template <typename R, int NDER>
__global__ void __launch_bounds__(256) k_spread(KParams p, DevState<R> d, int kind, const double *vec, R *grid) {
    const bool pcg = kind == SPREAD_DIP_PCG;
    if (pcg) {
        if (d.flags[1]) return;   // solver already converged
        kind = SPREAD_DIP;
    }
    const int per = kind == SPREAD_PERM ? NS : (kind == SPREAD_DIP ? 3 : (p.ct_orig ? 5 : 2));
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / PG, xi = gt % PG;
    if (t >= p.M * per || xi >= ORDER) return;
    const int m = t / per, a = t % per;
    const int pt = kind == SPREAD_LAMBDA ? (a < 2 ? 5 + a : a - 2) : a;
    Mp<R> mp{};
    if (kind == SPREAD_PERM) mp = load_mp(d.gmp + (m * NS + a) * GMP);
    else if (kind == SPREAD_DIP) {
        const R *v = pcg ? d.vecR : d.muR;
        mp.mu = mk(v[m * 9 + a * 3], v[m * 9 + a * 3 + 1], v[m * 9 + a * 3 + 2]);
    } else mp.q = a < 2 ? d.lamR[m * 2 + a] : d.lamaR[m * 3 + a - 2];
    Axis<R, NDER> X, Y, Z;
    axis_weights<R, NDER>(p, d, m, pt, 0, X);
    axis_weights<R, NDER>(p, d, m, pt, 1, Y);
    axis_weights<R, NDER>(p, d, m, pt, 2, Z);
    int gx;
    R wx[NDER + 1];
    line_weight<R, NDER>(X, xi, gx, wx);
    const R third = R(1) / R(3);
#pragma unroll
    for (int jy = 0; jy < ORDER; ++jy) {
        R wy[NDER + 1];
#pragma unroll
        for (int n = 0; n <= NDER; ++n) wy[n] = Y.w[n][jy];
        // coefficients of the z weights (0th, 1st, 2nd derivative)
        R c0 = mp.q * wx[0] * wy[0], c1 = R(0), c2 = R(0);
        if constexpr (NDER >= 1) {
            c0 += mp.mu.x * wx[1] * wy[0] + mp.mu.y * wx[0] * wy[1];
            c1 = mp.mu.z * wx[0] * wy[0];
        }
        if constexpr (NDER >= 2) {
            c0 += third * (mp.th.xx * wx[2] * wy[0] + mp.th.yy * wx[0] * wy[2] + R(2) * mp.th.xy * wx[1] * wy[1]);
            c1 += third * R(2) * (mp.th.xz * wx[1] * wy[0] + mp.th.yz * wx[0] * wy[1]);
            c2 = third * mp.th.zz * wx[0] * wy[0];
        }
        R v[ORDER];
#pragma unroll
        for (int k = 0; k < ORDER; ++k) {
            v[k] = c0 * Z.w[0][k];
            if constexpr (NDER >= 1) v[k] += c1 * Z.w[1][k];
            if constexpr (NDER >= 2) v[k] += c2 * Z.w[2][k];
        }
        add_zline<R>(grid, ((size_t)gx * p.K[1] + Y.g[jy]) * p.K[2], p.K[2], Z.g, v);
    }
}

template <typename R>
void launch_spread(const KParams &p, DevState<R> &d, int kind, const double *vec, R *grid, Launch L) {
    const int per = kind == SPREAD_PERM ? NS : ((kind == SPREAD_DIP || kind == SPREAD_DIP_PCG) ? 3 : (p.ct_orig ? 5 : 2));
    const long long threads = (long long)p.M * per * PG;
    const unsigned nb = (unsigned)((threads + 255) / 256);
    if (kind == SPREAD_PERM) k_spread<R, 2><<<nb, 256, 0, L.s>>>(p, d, kind, vec, grid);
    else if (kind == SPREAD_LAMBDA) k_spread<R, 0><<<nb, 256, 0, L.s>>>(p, d, kind, vec, grid);
    else k_spread<R, 1><<<nb, 256, 0, L.s>>>(p, d, kind, vec, grid);
    count(L);
}

// multiply the half-complex spectrum (ngrid grids back to back) by the influence function
template <typename R, typename C>
__global__ void k_convolve(KParams p, const R *infl, C *cg, int ngrid, const int *done, int check) {
    if (check && *done) return;
    const size_t nh = (size_t)p.K[0] * p.K[1] * (p.K[2] / 2 + 1);
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nh * ngrid) return;
    const R g = infl[t % nh];
    C c = cg[t];
    c.x *= g;
    c.y *= g;
    cg[t] = c;
}

// working-precision copy of the FP64 influence function
template <typename R>
__global__ void k_infl_copy(size_t n, const double *infl, R *out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = R(infl[t]);
}
template <typename R>
void launch_influence_copy(const KParams &p, DevState<R> &d, Launch L) {
    const size_t nh = (size_t)p.K[0] * p.K[1] * (p.K[2] / 2 + 1);
    k_infl_copy<R><<<(unsigned)((nh + 255) / 256), 256, 0, L.s>>>(nh, d.infl, d.inflR);
    count(L);
}

template <typename R>
void launch_convolve(const KParams &p, DevState<R> &d, void *cgrid, int ngrid, int check, Launch L) {
    const size_t nh = (size_t)p.K[0] * p.K[1] * (p.K[2] / 2 + 1);
    const size_t n = nh * ngrid;
    if (sizeof(R) == 4)
        k_convolve<float, cufftComplex><<<(unsigned)((n + 255) / 256), 256, 0, L.s>>>(
            p, (const float *)d.inflR, (cufftComplex *)cgrid, ngrid, d.flags + 1, check);
    else
        k_convolve<double, cufftDoubleComplex><<<(unsigned)((n + 255) / 256), 256, 0, L.s>>>(
            p, (const double *)d.inflR, (cufftDoubleComplex *)cgrid, ngrid, d.flags + 1, check);
    count(L);
}

// Convolution with the k-space virial sums.  E_rec = sum over the full
// spectrum of e(k) = G(k) (...); a half-spectrum point with 0 < kz < K2/2
// also stands for its conjugate -k (same e, folded vector below).  Under the
// strain the reciprocal vectors m and the volume change, dG/d eps_ab =
// G [-delta_ab + 2 (1/m^2 + pi^2/alpha^2) m_a m_b].  Per block: sum e, and
// sum e f m_a m_b (xx yy zz xy xz yz), f = 2 (1/m^2 + pi^2/alpha^2).
// pass 0: the permanent spectrum, e = 1/2 |Q_p|^2 G; it is kept in qp.
// pass 1: grids of the induced dipoles (Q_m) and the lambda charges (Q_l),
//         e = G [Re(Q_p^* (Q_m + Q_l)) + 1/2 |Q_m|^2].
template <typename R, typename C>
__global__ void __launch_bounds__(256) k_convolve_vir(KParams p, const R *infl, C *cg, C *qp, double *part, int pass) {
    const int K0 = p.K[0], K1 = p.K[1], K2 = p.K[2], nz = K2 / 2 + 1;
    const size_t nh = (size_t)K0 * K1 * nz;
    const double pa2 = M_PI * M_PI / (p.alpha * p.alpha);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nh; t += (size_t)gridDim.x * blockDim.x) {
        const int kz = (int)(t % nz), ky = (int)((t / nz) % K1), kx = (int)(t / ((size_t)nz * K1));
        const double fx = (kx <= K0 / 2 ? kx : kx - K0) * p.ibox[0];
        const double fy = (ky <= K1 / 2 ? ky : ky - K1) * p.ibox[1];
        const double fz = kz * p.ibox[2];
        const double m2 = fx * fx + fy * fy + fz * fz;
        const R g = infl[t];
        C a = cg[t];
        double e;
        if (pass == 0) {
            e = 0.5 * (double)g * ((double)a.x * a.x + (double)a.y * a.y);
            qp[t] = a;
        } else {
            C b = cg[t + nh];
            const C q = qp[t];
            e = (double)g * ((double)q.x * ((double)a.x + b.x) + (double)q.y * ((double)a.y + b.y) +
                             0.5 * ((double)a.x * a.x + (double)a.y * a.y));
            b.x *= g;
            b.y *= g;
            cg[t + nh] = b;
        }
        a.x *= g;
        a.y *= g;
        cg[t] = a;
        if (m2 > 0.0) {
            const double f = 2.0 * (1.0 / m2 + pa2) * e;
            acc[0] += e;
            acc[1] += f * fx * fx;
            acc[2] += f * fy * fy;
            acc[3] += f * fz * fz;
            acc[4] += f * fx * fy;
            acc[5] += f * fx * fz;
            acc[6] += f * fy * fz;
            if (!(kz == 0 || (K2 % 2 == 0 && kz == K2 / 2))) {
                // the conjugate point -k of the full spectrum, same e; its
                // folded vector flips every component except on a Nyquist
                // row (k = K/2 folds onto itself)
                const double gx = 2 * kx == K0 ? fx : -fx, gy = 2 * ky == K1 ? fy : -fy, gz = -fz;
                acc[0] += e;
                acc[1] += f * gx * gx;
                acc[2] += f * gy * gy;
                acc[3] += f * gz * gz;
                acc[4] += f * gx * gy;
                acc[5] += f * gx * gz;
                acc[6] += f * gy * gz;
            }
        }
    }
    __shared__ double sh[8][7];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0;
        for (int k = 0; k < 8; ++k) v += sh[k][threadIdx.x];
        part[((size_t)pass * VK_BLOCKS + blockIdx.x) * 8 + threadIdx.x] = v;
    }
}

template <typename R>
void launch_convolve_vir(const KParams &p, DevState<R> &d, int pass, Launch L) {
    if (sizeof(R) == 4)
        k_convolve_vir<float, cufftComplex><<<VK_BLOCKS, 256, 0, L.s>>>(
            p, (const float *)d.inflR, (cufftComplex *)d.cgrid, (cufftComplex *)d.qhat_p, d.virk, pass);
    else
        k_convolve_vir<double, cufftDoubleComplex><<<VK_BLOCKS, 256, 0, L.s>>>(
            p, (const double *)d.inflR, (cufftDoubleComplex *)d.cgrid, (cufftDoubleComplex *)d.qhat_p, d.virk, pass);
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
// Gather: potential derivatives at a point from a convolved grid, one warp
// per point; lane (i, j) < 25 sums its stencil row, the warp reduces.
// ---------------------------------------------------------------------------
template <typename R>
struct Derivs {
    R phi;
    R d1[3];
    R d2[6];    // xx yy zz xy xz yz
    R d3[10];   // xxx yyy zzz xxy xxz xyy yyz xzz yzz xyz
};
constexpr int ND_VALS = 20;

// this lane's row contribution to the derivatives up to NDER, packed as
// phi, d1[3], d2[6], d3[10]
template <typename R, int NDER>
__device__ inline void gather_row(const KParams &p, const R *grid, const Axis<R, NDER> &X, const Axis<R, NDER> &Y,
                                  const Axis<R, NDER> &Z, int lane, R *v) {
    int gx, gy;
    R x[NDER + 1], y[NDER + 1];
    line_weight<R, NDER>(X, lane / 5, gx, x);
    line_weight<R, NDER>(Y, lane % 5, gy, y);
    const size_t row = ((size_t)gx * p.K[1] + gy) * p.K[2];
    R t[4] = {R(0), R(0), R(0), R(0)};   // sums over z with z-derivative order 0..3
#pragma unroll
    for (int k = 0; k < ORDER; ++k) {
        const R g = grid[row + Z.g[k]];
#pragma unroll
        for (int n = 0; n <= NDER; ++n) t[n] += g * Z.w[n][k];
    }
    v[0] = x[0] * y[0] * t[0];
    if constexpr (NDER >= 1) {
        v[1] = x[1] * y[0] * t[0];
        v[2] = x[0] * y[1] * t[0];
        v[3] = x[0] * y[0] * t[1];
    }
    if constexpr (NDER >= 2) {
        v[4] = x[2] * y[0] * t[0];
        v[5] = x[0] * y[2] * t[0];
        v[6] = x[0] * y[0] * t[2];
        v[7] = x[1] * y[1] * t[0];
        v[8] = x[1] * y[0] * t[1];
        v[9] = x[0] * y[1] * t[1];
    }
    if constexpr (NDER >= 3) {
        v[10] = x[3] * y[0] * t[0];
        v[11] = x[0] * y[3] * t[0];
        v[12] = x[0] * y[0] * t[3];
        v[13] = x[2] * y[1] * t[0];
        v[14] = x[2] * y[0] * t[1];
        v[15] = x[1] * y[2] * t[0];
        v[16] = x[0] * y[2] * t[1];
        v[17] = x[1] * y[0] * t[2];
        v[18] = x[0] * y[1] * t[2];
        v[19] = x[1] * y[1] * t[1];
    }
}

// Group gather of one point (PG lanes; lanes 0-4 sum x-lines 0-4 of the
// stencil): the derivatives up to NDER, complete in every lane of the group
// after a shuffle reduction.  All 32 lanes of the warp must call it; a group
// with live = false returns zeros.
template <typename R, int NDER>
__device__ inline void group_gather(const KParams &p, const DevState<R> &d, const R *grid, int m, int pt, int sub,
                                    bool live, Derivs<R> &D) {
    constexpr int NV = NDER >= 3 ? 20 : (NDER == 2 ? 10 : (NDER == 1 ? 4 : 1));
    R v[ND_VALS];
#pragma unroll
    for (int k = 0; k < ND_VALS; ++k) v[k] = R(0);
    if (live && sub < ORDER) {
        Axis<R, NDER> X, Y, Z;
        axis_weights<R, NDER>(p, d, m, pt, 0, X);
        axis_weights<R, NDER>(p, d, m, pt, 1, Y);
        axis_weights<R, NDER>(p, d, m, pt, 2, Z);
#pragma unroll
        for (int jy = 0; jy < ORDER; ++jy) {
            R u[ND_VALS];
            gather_row<R, NDER>(p, grid, X, Y, Z, sub * ORDER + jy, u);
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] += u[k];
        }
    }
#pragma unroll
    for (int o = PG / 2; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    R *out = reinterpret_cast<R *>(&D);
#pragma unroll
    for (int k = 0; k < ND_VALS; ++k) out[k] = k < NV ? v[k] : R(0);
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

// dU/dr component a for a multipole sitting in the gathered potential:
// q d1 + d2 . mu + (1/3) Theta : d3
template <typename R>
__device__ inline R mp_grad(const Mp<R> &m, const Derivs<R> &D, int a) {
    const R th[6] = {m.th.xx, m.th.yy, m.th.zz, m.th.xy, m.th.xz, m.th.yz};
    const R mu[3] = {m.mu.x, m.mu.y, m.mu.z};
    R v = m.q * D.d1[a];
    for (int b = 0; b < 3; ++b) v += sym_at(D.d2, a, b) * mu[b];
    R t = 0;
    for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) t += sym_at(th, b, c) * d3at(D, a, b, c);
    return v + t / R(3);
}

template <typename R>
__device__ inline R mp_energy(const Mp<R> &m, const Derivs<R> &D) {
    const Sym<R> d2{D.d2[0], D.d2[1], D.d2[2], D.d2[3], D.d2[4], D.d2[5]};
    return m.q * D.phi + m.mu.x * D.d1[0] + m.mu.y * D.d1[1] + m.mu.z * D.d1[2] + symdd(m.th, d2) / R(3);
}

// Strain derivative of a multipole's reciprocal energy through the
// reciprocal vectors at fixed Cartesian multipoles: entry (a, b) of
// d1_a mu_b + (2/3) sum_c d2_ac Theta_cb (its negative adds to dE/d eps_ab;
// the Ewald structure factor's k-dependence of mu.k and k.Theta.k)
template <typename R>
__device__ inline R mp_strain(const Mp<R> &m, const Derivs<R> &D, int k) {
    const int a = k / 3, b = k % 3;
    const R th[6] = {m.th.xx, m.th.yy, m.th.zz, m.th.xy, m.th.xz, m.th.yz};
    const R mu[3] = {m.mu.x, m.mu.y, m.mu.z};
    R t = R(0);
    for (int c = 0; c < 3; ++c) t += sym_at(D.d2, a, c) * sym_at(th, c, b);
    return D.d1[a] * mu[b] + R(2.0 / 3.0) * t;
}

// Permanent pass: a group of PG lanes per point, the 5 sites of every
// molecule first (points t < 5 M), then the 2 lone pairs.  Sites: energy,
// gradient, multipole sensitivities; O/H1/H2 also their field and Hessian;
// lone pairs: potential and its gradient.  The group's lanes then share the
// outputs.
template <typename R>
__global__ void __launch_bounds__(256, 2) k_gather_perm(KParams p, DevState<R> d) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / PG, sub = gt % PG;
    const int nsite = p.M * NS;
    const bool live = t < p.M * NP;
    const bool site = t < nsite;
    const int m = site ? t / NS : (t - nsite) / 2;
    const int pt = site ? t % NS : NS + (t - nsite) % 2;
    Derivs<R> D;
    // groups of one warp are all sites except in one warp
    const bool any_site = __any_sync(0xffffffffu, live && site), any_lp = __any_sync(0xffffffffu, live && !site);
    if (any_site) group_gather<R, 3>(p, d, d.grid, m, pt, sub, live && site, D);
    if (any_lp) {
        Derivs<R> Dl;
        group_gather<R, 1>(p, d, d.grid, m, pt, sub, live && !site, Dl);
        if (!site) D = Dl;
    }
    if (!live) return;
    if (site) {
        const Mp<R> mp = load_mp(d.gmp + (m * NS + pt) * GMP);
        // original charge transfer: also the potential and its gradient at the atoms
        const int nout = (p.ct_orig && pt < 3) ? 26 : 22;
        for (int o = sub; o < nout; o += PG) {
            if (o < 3) {
                d.gpt[(m * NP + pt) * 3 + o] += (double)mp_grad(mp, D, o);
                d.gmu[(m * NS + pt) * 3 + o] += (double)D.d1[o];
                if (pt < 3) d.efield[m * 9 + pt * 3 + o] -= (double)D.d1[o] * p.sd.ike;
            } else if (o < 9) {
                d.gth[(m * NS + pt) * 6 + o - 3] += (double)D.d2[o - 3] * (1.0 / 3.0);
                if (pt < 3) d.d2rec[m * 18 + pt * 6 + o - 3] = (double)D.d2[o - 3];
            } else if (o == 9) {
                atomicAdd(&d.epart[m * NTERM + T_ELEC], 0.5 * (double)mp_energy(mp, D));
            } else if (o < 22) {
                if (p.vir) {
                    if (o < 19) atomicAdd(&d.vir[m * 9 + o - 10], -(double)mp_strain(mp, D, o - 10));
                    else if (pt < 3) d.vphi[m * 9 + pt * 3 + o - 19] = D.d1[o - 19];
                }
            } else if (o == 22) {
                d.va[m * 3 + pt] += (double)D.phi;
            } else {
                d.dva[(m * 3 + pt) * 3 + o - 23] += (double)D.d1[o - 23];
            }
        }
    } else {
        const int l = pt - NS;
        if (sub < 3) d.dvlp[(m * 2 + l) * 3 + sub] += (double)D.d1[sub];
        else if (sub == 3) d.vlp[m * 2 + l] += (double)D.phi;
    }
}

template <typename R>
void launch_gather_perm(const KParams &p, DevState<R> &d, Launch L) {
    const long long threads = (long long)p.M * NP * PG;
    k_gather_perm<R><<<(unsigned)((threads + 255) / 256), 256, 0, L.s>>>(p, d);
    count(L);
}

// PCG product, reciprocal and intramolecular part at each polarizable atom:
// out += -grad phi / ke from the dipole grid plus the self term of the atom's
// own dipole minus the erf part of the field of the other two atoms' dipoles
// (dipoles: the working-precision PCG vector).  A group of PG lanes per atom:
// lanes 0-4 sum the 25 grid points of their x-line, lane 5 the self term,
// lanes 6 and 7 the erf field of one other atom each.
template <typename R>
__global__ void __launch_bounds__(256) k_gather_field(KParams p, DevState<R> d, double *out) {
    if (d.flags[1]) return;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / PG, sub = gt % PG;
    const bool live = t < p.M * 3;   // the whole group is live or not
    const int m = live ? t / 3 : 0, a = live ? t % 3 : 0;
    const Scal<R> &S = sc<R>(p);
    V3<R> E = mk(R(0), R(0), R(0));
    if (live && sub < ORDER) {
        Axis<R, 1> X, Y, Z;
        axis_weights<R, 1>(p, d, m, a, 0, X);
        axis_weights<R, 1>(p, d, m, a, 1, Y);
        axis_weights<R, 1>(p, d, m, a, 2, Z);
        int gx;
        R wx[2];
        line_weight<R, 1>(X, sub, gx, wx);
        R v1 = R(0), v2 = R(0), v3 = R(0);
#pragma unroll
        for (int jy = 0; jy < ORDER; ++jy) {
            const R *row = d.grid + ((size_t)gx * p.K[1] + Y.g[jy]) * p.K[2];
            R t0 = R(0), t1 = R(0);
#pragma unroll
            for (int k = 0; k < ORDER; ++k) {
                const R g = row[Z.g[k]];
                t0 += g * Z.w[0][k];
                t1 += g * Z.w[1][k];
            }
            v1 += wx[1] * Y.w[0][jy] * t0;
            v2 += wx[0] * Y.w[1][jy] * t0;
            v3 += wx[0] * Y.w[0][jy] * t1;
        }
        E = mk(-v1 * S.ike, -v2 * S.ike, -v3 * S.ike);
    } else if (live) {
        const R al = S.alpha;
        const R *v = d.vecR + m * 9;
        if (sub == ORDER) {
            const R cself = R(4.0 / 3.0) * al * al * al * R(0.56418958354775628695);
            E = cself * mk(v[a * 3], v[a * 3 + 1], v[a * 3 + 2]);
        } else {
            const int b = (a + sub - ORDER) % 3;   // the two atoms b != a
            const V3<R> xv = my_pt(d, m, a) - my_pt(d, m, b);
            R g[4];
            g_erf_s<R, 3>(dot(xv, xv), al, g);
            Mp<R> s{};
            s.mu = mk(v[b * 3], v[b * 3 + 1], v[b * 3 + 2]);
            FieldTerms<R> f;
            source_field<R, 1>(s, xv, g, f);
            E = f.d1;
        }
    }
#pragma unroll
    for (int o = PG / 2; o > 0; o >>= 1) {
        E.x += __shfl_xor_sync(0xffffffffu, E.x, o);
        E.y += __shfl_xor_sync(0xffffffffu, E.y, o);
        E.z += __shfl_xor_sync(0xffffffffu, E.z, o);
    }
    if (live && sub < 3) out[m * 9 + a * 3 + sub] += (double)(sub == 0 ? E.x : (sub == 1 ? E.y : E.z));
}

template <typename R>
void launch_gather_field(const KParams &p, DevState<R> &d, double *out, Launch L) {
    const long long threads = (long long)p.M * 3 * PG;
    k_gather_field<R><<<(unsigned)((threads + 255) / 256), 256, 0, L.s>>>(p, d, out);
    count(L);
}

// Force pass: grid 0 holds the induced dipoles, grid 1 the lambda charges.
// Sites: gradient and sensitivities of the permanent multipoles in the sum of
// both potentials.  O/H1/H2: gradient of the induced dipole in the induced
// (grid 0) and permanent (stored Hessian) reciprocal potentials.
template <typename R>
__global__ void __launch_bounds__(256, 2) k_gather_polforce(KParams p, DevState<R> d) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / PG, sub = gt % PG;
    const bool live = t < p.M * NS;
    const int m = live ? t / NS : 0, pt = live ? t % NS : 0;
    const size_t ng = (size_t)p.K[0] * p.K[1] * p.K[2];
    Derivs<R> A, B;
    group_gather<R, 3>(p, d, d.grid, m, pt, sub, live, A);
    group_gather<R, 3>(p, d, d.grid + ng, m, pt, sub, live, B);
    if (!live) return;
    Derivs<R> S;
    S.phi = A.phi + B.phi;
    for (int k = 0; k < 3; ++k) S.d1[k] = A.d1[k] + B.d1[k];
    for (int k = 0; k < 6; ++k) S.d2[k] = A.d2[k] + B.d2[k];
    for (int k = 0; k < 10; ++k) S.d3[k] = A.d3[k] + B.d3[k];
    const Mp<R> mp = load_mp(d.gmp + (m * NS + pt) * GMP);
    for (int o = sub; o < 19; o += PG) {
        if (o < 3) {
            double g = (double)mp_grad(mp, S, o);
            if (pt < 3) {
                // induced dipole in the induced (grid 0) and permanent (stored Hessian) potentials
                const double *mu = d.mu + m * 9 + pt * 3;
                const double *h = d.d2rec + m * 18 + pt * 6;
                for (int b = 0; b < 3; ++b) g += ((double)sym_at(A.d2, o, b) + sym_at(h, o, b)) * mu[b];
            }
            d.gpt[(m * NP + pt) * 3 + o] += g;
            d.gmu[(m * NS + pt) * 3 + o] += (double)S.d1[o];
        } else if (o < 9) {
            d.gth[(m * NS + pt) * 6 + o - 3] += (double)S.d2[o - 3] * (1.0 / 3.0);
        } else if (p.vir && o >= 10) {
            // permanent multipoles in the induced + lambda potential; induced
            // dipole in the permanent + induced potential
            const int k = o - 10, a = k / 3, b = k % 3;
            double c = (double)mp_strain(mp, S, k);
            if (pt < 3) c += ((double)d.vphi[m * 9 + pt * 3 + a] + (double)A.d1[a]) * d.mu[m * 9 + pt * 3 + b];
            atomicAdd(&d.vir[m * 9 + k], -c);
        }
    }
}

template <typename R>
void launch_gather_polforce(const KParams &p, DevState<R> &d, Launch L) {
    const long long threads = (long long)p.M * NS * PG;
    k_gather_polforce<R><<<(unsigned)((threads + 255) / 256), 256, 0, L.s>>>(p, d);
    count(L);
}

#define INST(R)                                                                                         \
    template void launch_spread<R>(const KParams &, DevState<R> &, int, const double *, R *, Launch);    \
    template void launch_convolve<R>(const KParams &, DevState<R> &, void *, int, int, Launch);               \
    template void launch_influence_copy<R>(const KParams &, DevState<R> &, Launch);                      \
    template void launch_gather_perm<R>(const KParams &, DevState<R> &, Launch);                         \
    template void launch_gather_field<R>(const KParams &, DevState<R> &, double *, Launch);              \
    template void launch_gather_polforce<R>(const KParams &, DevState<R> &, Launch);                     \
    template void launch_convolve_vir<R>(const KParams &, DevState<R> &, int, Launch);
INST(float)
INST(double)

}  // namespace sibfa
