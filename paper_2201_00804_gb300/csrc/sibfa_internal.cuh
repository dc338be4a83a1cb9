// Internal declarations of the SIBFA CUDA library: device state, kernel
// parameters, vector helpers, radial kernels and the multipole field
// evaluation shared by the pair and grid kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cufft.h>

#include "../../include/sibfa.h"

namespace sibfa {

constexpr int NS = 5;          // multipole sites per water: O, H1, H2, M1, M2
constexpr int NP = 7;          // points per water: 5 sites + 2 lone pairs
constexpr int NMP = 10;        // q, mu(3), theta(6: xx yy zz xy xz yz)
constexpr int GMP = 12;        // row stride of the global multipoles: NMP values + 2 pad (48-byte FP32 rows)
constexpr int MAXN = 384;      // neighbour slots per molecule
constexpr int NTERM = 7;       // elec pen rep disp xdisp pol ct
enum { T_ELEC = 0, T_PEN, T_REP, T_DISP, T_XDISP, T_POL, T_CT };
constexpr int ORDER = 5;       // B-spline order of the SPME
constexpr int VK_BLOCKS = 304;  // blocks of the virial convolution (fixed, so its partial sums have a fixed layout)

// error flags (bitwise, device side)
enum { F_CUTOFF = 1, F_NEIGHBOR = 2, F_CTDEN = 4, F_NAN = 8, F_NOCONV = 16 };

// Scalars read inside pair loops, rounded once per precision on the host so
// that the FP32 kernels do no FP64 conversion in their loops.
template <typename R>
struct Scal {
    R rc2, alpha, thole;
    R cs_o, cp_o, cs_h, cp_h, cs_lp, cp_lp, g_o, g_h, inv_nval_o, inv_nval_h;
    R rep_f, rep_c1, rep_c2, occ, nlp;
    R c6, c8, c10, g6, g8, g10, delta, xd_c1, xd_c2, xd_c3;
    R ct_t, ct_m, ct_ae, ct_ah;
    R kl[3];   // SPME grid points per unit length, K / L
    R ike;     // 1 / ke
};

// ---------------------------------------------------------------------------
// Kernel parameters (by value).
// ---------------------------------------------------------------------------
// Verlet skin of the periodic neighbour list (A): the list keeps the pairs
// within rc + 2 * site extent + skin of its build and is rebuilt once an O
// has moved by half the skin (less any growth of the extent) since then.
constexpr double LIST_SKIN = 0.4;

struct KParams {
    int M;
    int periodic;
    int n_cl;              // clusters (1: one system)
    int tls;               // T-pair list slots per polarizable atom: 3 x the most neighbours a molecule can have
    int vir;               // 1: this evaluation also accumulates the virial
    int ct_orig;           // 1: the original many-body charge transfer (acceptor potentials kept)
    double box[3];
    double ibox[3];        // 1 / box
    double rc, rc2;
    double skin;           // Verlet skin of the periodic neighbour list (0: rebuilt every evaluation)
    double alpha;          // Ewald
    int K[3];
    double ke;
    double d_lp, lp_cos, lp_sin;
    double a_pol[3];       // O, H, H polarizabilities
    double a_pol_inv[3];   // their reciprocals
    double a_damp[5];      // site polarizabilities used in Thole damping
    double thole;
    double z[5], b[5];     // nuclear charge and valence damping per site (0 on midpoints)
    // repulsion
    double cs_o, cp_o, cs_h, cp_h, cs_lp, cp_lp, g_o, g_h, nval_o, nval_h;
    double rv_rep_o, rv_rep_h, rv_rep_lp, rep_a1, rep_a2, rep_c1, rep_c2, rep_f, occ, nlp;
    // dispersion
    double rv_d[5];        // O, H, H, LP, LP
    double beta[5];
    double disp_alpha, c6, c8, c10, g6, g8, g10, delta;
    double xd_c1, xd_a1, xd_c2, xd_a2, xd_c3, xd_a3;
    // charge transfer
    double ct_eta, ct_t, ct_m, ct_ae, ct_ah, rv_ct_o, rv_ct_h;
    // Pair-type coefficients precomputed in FP64 on the host (kinds: 0 = O,
    // 1 = H, 2 = lone pair).  In the FP32 path each is used as a hi + lo pair
    // of floats so that large exponent arguments keep FP64-rounded constants.
    struct Coef {
        double d;
        float hi, lo;   // hi = float(d), lo = float(d - hi)
    };
    Coef rep_k1[3][3], rep_k2[3][3];     // rep_alpha / (4 sqrt(rv_a rv_b)), same with rep_alpha2
    Coef disp_km[3][3];                  // 1 / (2 sqrt(rv_a rv_b))   (dispersion radii)
    Coef disp_gS[3][3][3];               // gamma_n (rv_a + rv_b) disp_alpha, n = 6, 8, 10
    Coef xd_k[3][3];                     // A_type / (2 sqrt(rv_a rv_b)) for exchange-dispersion
    Coef ct_k1, ct_k2;                   // eta / (2 sqrt(rv_O rv_O)), eta / (2 sqrt(rv_O rv_H))
    Coef pen_b[5];                       // valence damping exponents per site
    // Single-precision copies of per-pair indexed constants (no FP64 work in
    // the FP32 inner loops); the FP64 path uses the double tables.
    float zf[5];                         // nuclear charge per site
    float ainv3f[5][5];                  // Thole 1 / sqrt(alpha_s alpha_t) over the site damping polarizabilities
    double ainv3[5][5];
    float betaf[5];                      // dispersion beta per point (O, H, H, LP, LP)
    Scal<float> sf;
    Scal<double> sd;
    float fxs[3];                        // box / 2^32: length of one fixed-point unit per axis
};

template <typename R>
__device__ inline const Scal<R> &sc(const KParams &p);
template <>
__device__ inline const Scal<float> &sc<float>(const KParams &p) { return p.sf; }
template <>
__device__ inline const Scal<double> &sc<double>(const KParams &p) { return p.sd; }

template <typename R>
__device__ inline R zsite(const KParams &p, int s);
template <>
__device__ inline float zsite<float>(const KParams &p, int s) { return p.zf[s]; }
template <>
__device__ inline double zsite<double>(const KParams &p, int s) { return p.z[s]; }
template <typename R>
__device__ inline R ainv3(const KParams &p, int a, int b);
template <>
__device__ inline float ainv3<float>(const KParams &p, int a, int b) { return p.ainv3f[a][b]; }
template <>
__device__ inline double ainv3<double>(const KParams &p, int a, int b) { return p.ainv3[a][b]; }
template <typename R>
__device__ inline R betap(const KParams &p, int a);
template <>
__device__ inline float betap<float>(const KParams &p, int a) { return p.betaf[a]; }
template <>
__device__ inline double betap<double>(const KParams &p, int a) { return p.beta[a]; }

// x * c for a coefficient precomputed in FP64: in FP32 the product keeps the
// FP64 rounding of c (x * hi + x * lo).
template <typename R>
__device__ inline R mulc(R x, const KParams::Coef &c);
template <>
__device__ inline double mulc<double>(double x, const KParams::Coef &c) { return x * c.d; }
template <>
__device__ inline float mulc<float>(float x, const KParams::Coef &c) { return fmaf(x, c.hi, x * c.lo); }
template <typename R>
__device__ inline R cval(const KParams::Coef &c);
template <>
__device__ inline double cval<double>(const KParams::Coef &c) { return c.d; }
template <>
__device__ inline float cval<float>(const KParams::Coef &c) { return c.hi; }

// ---------------------------------------------------------------------------
// Device state.  Per-molecule arrays are SoA-by-molecule: index m*stride+k.
// ---------------------------------------------------------------------------
template <typename R>
struct DevState {
    int M;
    double *pos;        // M*9 working positions (O, H1, H2)
    double *mp_local;   // M*50
    R *off;             // M*NP*3 point offsets from own O (5 sites + 2 LPs)
    R *gmp;             // M*NS*GMP global multipoles (rows of NMP values, padded)
    double *vint;       // M*3 intramolecular potential on O, H1, H2 (charge-transfer V_int)
    int *nbr;           // M*MAXN neighbour molecules (full list)
    R *ndo;             // M*MAXN*3 minimum-image displacement O_j - O_i of each entry
    int *nnbr;          // M
    int *cl_of;         // M    cluster of each molecule
    int *cl_start;      // n_cl+1 first molecule of each cluster
    double *cl_rr;      // n_cl  PCG: sum of squared preconditioned residuals per cluster
    double *cl_energy;  // n_cl*(NTERM+1) energy terms and total per cluster
    float *ofw;         // M*3 O positions wrapped into the box (single precision, cell binning)
    unsigned *ufx;      // M*3 O fractional coordinates in units of 2^-32 of the box (periodic list build)
    int *sbase;         // M*NP*3 SPME: floor(u) mod K of every point (u = fractional coordinate x K)
    R *sfrac;           // M*NP*3 SPME: u - floor(u)
    // cell list
    int *cell_of;       // M
    int *cell_start;    // ncell+1
    int *cell_cursor;   // ncell
    int *cell_mol;      // M
    // gradients dE/dx (double) and multipole sensitivities
    double *gpt;        // M*NP*3 dE/d(point)
    double *gmu;        // M*NS*3 dE/dmu_global
    double *gth;        // M*NS*6 dE/dTheta_global (symmetric, components as stored)
    double *efield;     // M*9 permanent field on O, H1, H2 (Thole-damped real + recip - excl + self)
    double *d2rec;      // M*3*6 reciprocal Hessian of the permanent potential at O, H1, H2
    double *vlp;        // M*2 potential on lone pairs (undamped, own molecule excluded)
    double *dvlp;       // M*2*3 its gradient
    double *lam;        // M*2 dE_ct/dV_lp
    double *kap;        // M*3 dE_ct/dV_int
    double *epart;      // M*NTERM per-molecule energy partials
    double *eintra;     // M  mixed periodic path: FP64 intramolecular Ewald energy per molecule
    double *epartial;   // 128*NTERM per-block partial energy sums
    double *epw;        // M*NS*2 multipole and penetration energy of each target site (k_real_perm)
    // Virial: per-molecule dE/d eps (row-major 3x3) for the affine strain
    // x -> (I + eps) x of atoms and cell, and the reciprocal-space parts
    double *vir;        // M*9
    double *vir_r;      // M*9 (reciprocal chain)
    double *virk;       // 2 passes x VK_BLOCKS x 8: k-space sums per convolution block
    void *qhat_p;       // K0*K1*(K2/2+1) complex: spectrum of the permanent grid (kept for the force pass)
    R *vphi;            // M*9 gradient of the reciprocal permanent potential at O, H1, H2
    // Accumulators of the reciprocal-space chain (SPME and intramolecular
    // Ewald corrections), which runs on a second stream concurrently with the
    // real-space kernels; same layouts as the arrays above, merged where used.
    double *gpt_r, *gmu_r, *gth_r, *efield_r, *vlp_r, *dvlp_r, *epart_r, *efp_r;
    // point gradients of the short-range kernels, which run on a third stream
    // concurrently with the permanent pass and the polarization solve
    double *gpt_s;
    // polarization solve
    double *mu, *res, *zv, *pv, *ap, *efp;   // M*9 each
    R *vecR;            // M*9 the vector of the current T product in the working precision
    R *muR, *lamR;      // M*9, M*2 induced dipoles and CT lambdas in the working precision (force pass)
    // Real-space T pairs recorded by the permanent pass: for polarizable atom
    // t = 3 m + a, entries [t*tls, t*tls + tl_n[t]) hold the partner atom
    // (3 j + b), the displacement x = r_t - r_jb and the Thole-damped kernel
    // weights g1, g2 of the dipole field (E = g2 (mu.x) x + g1 mu).
    // original charge transfer: potential and its gradient at O, H1, H2 from
    // the other molecules (real space / reciprocal chain), dE/dV(a) of the
    // acceptor atoms (FP64 and working-precision copy), and per neighbour
    // slot the sensitivities dE/dV*(a) at the partner's atoms (i donor, 0-2)
    // and at the molecule's own atoms (j donor, 3-5)
    double *va, *va_r, *dva, *dva_r, *lama;
    R *lamaR, *cvs;
    R *ctin;            // M*8 working-precision charge-transfer inputs (V_lp, V_int, V(a))
    R *spk;             // M*20 short-range point data (offset from O, valence factor) x 5 points
    int *tl_n, *tl_j;                   // polarization pair list: count per atom; partner | sgn(g2) << 31
    R *tl_x, *tl_y, *tl_z, *tl_g1;      // sqrt|g2| x (x the pair displacement) and g1
    double *partial;    // reduction partials
    double *scal;       // device scalars (see pcg kernels)
    unsigned int *counter;
    int *flags;         // [0] error flags, [1] PCG converged
    float *ext;         // maximum point distance from own O (float bits, atomicMax)
    double *oref;       // M*3 O positions at the last neighbour-list build
    float *lst;         // list state: [0] extent at the build, [1] skin of the build, [2] max squared O move (bits)
    int *lflag;         // [0] rebuild the list this evaluation, [1] a list has been built
    // grids
    R *grid;            // 2 * K0*K1*K2 (two real grids for the force pass)
    void *cgrid;        // 2 * K0*K1*(K2/2+1) complex
    double *infl;       // K0*K1*(K2/2+1) influence function / (K0 K1 K2)
    R *inflR;           // the same in the working precision
};

// ---------------------------------------------------------------------------
// Small vector helpers
// ---------------------------------------------------------------------------
template <typename R>
struct V3 {
    R x, y, z;
};
template <typename R>
__host__ __device__ inline V3<R> mk(R a, R b, R c) { return V3<R>{a, b, c}; }
template <typename R>
__host__ __device__ inline V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R>
__host__ __device__ inline V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R>
__host__ __device__ inline V3<R> operator-(V3<R> a) { return {-a.x, -a.y, -a.z}; }
template <typename R>
__host__ __device__ inline V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename R>
__host__ __device__ inline R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R>
__host__ __device__ inline V3<R> cross(V3<R> a, V3<R> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

template <typename R> __device__ inline R rsqrt_(R x);
// FP32: the hardware reciprocal square root refined by one Newton step
// (y <- y (3 - x y^2) / 2), which brings it to about one ulp; the radial
// kernels of every multipole order start from it.
template <> __device__ inline float rsqrt_<float>(float x) {
    const float y = rsqrtf(x);
    const float h = fmaf(-0.5f * x * y, y, 0.5f);   // (1 - x y^2) / 2
    return fmaf(y, h, y);
}
template <> __device__ inline double rsqrt_<double>(double x) { return rsqrt(x); }
// Reciprocal.  FP32: the hardware approximation refined by one Newton step
// (y <- y + y (1 - x y)), in place of the IEEE division sequence and its
// slow-path branch; FP64: the plain division.
template <typename R> __device__ inline R rcp_(R x);
template <> __device__ inline float rcp_<float>(float x) {
    const float y = __fdividef(1.0f, x);
    return fmaf(y, fmaf(-x, y, 1.0f), y);
}
template <> __device__ inline double rcp_<double>(double x) { return 1.0 / x; }
template <typename R> __device__ inline R exp_(R x);
template <> __device__ inline float exp_<float>(float x) { return expf(x); }
template <> __device__ inline double exp_<double>(double x) { return exp(x); }
template <typename R> __device__ inline R erfc_(R x);
template <> __device__ inline float erfc_<float>(float x) { return erfcf(x); }
template <> __device__ inline double erfc_<double>(double x) { return erfc(x); }
template <typename R> __device__ inline R sqrt_(R x);
template <> __device__ inline float sqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ inline double sqrt_<double>(double x) { return sqrt(x); }

// Symmetric 3x3 stored as xx yy zz xy xz yz
template <typename R>
struct Sym {
    R xx, yy, zz, xy, xz, yz;
};
template <typename R>
__device__ inline V3<R> symv(const Sym<R> &t, V3<R> v) {
    return {t.xx * v.x + t.xy * v.y + t.xz * v.z, t.xy * v.x + t.yy * v.y + t.yz * v.z,
            t.xz * v.x + t.yz * v.y + t.zz * v.z};
}
template <typename R>
__device__ inline R symdd(const Sym<R> &a, const Sym<R> &b) {
    return a.xx * b.xx + a.yy * b.yy + a.zz * b.zz + R(2) * (a.xy * b.xy + a.xz * b.xz + a.yz * b.yz);
}

// Virial accumulation: W[3a + b] += c g_a x_b (g a gradient, x a displacement)
template <typename R>
__device__ inline void vir_add(R (&W)[9], V3<R> g, V3<R> x, R c) {
    const R ga[3] = {c * g.x, c * g.y, c * g.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        W[3 * a] += ga[a] * x.x;
        W[3 * a + 1] += ga[a] * x.y;
        W[3 * a + 2] += ga[a] * x.z;
    }
}

// A point multipole: charge, dipole, traceless quadrupole (1/3 convention:
// phi = q g0 - mu.grad g0 + (1/3) Theta : grad grad g0).
template <typename R>
struct Mp {
    R q;
    V3<R> mu;
    Sym<R> th;
};

// ---------------------------------------------------------------------------
// Radial kernels: g[n+1](r) = (1/r) d g[n]/dr.
// ---------------------------------------------------------------------------
template <typename R, int N>
__device__ inline void g_bare(R rinv, R *g) {
    R r2i = rinv * rinv;
    g[0] = rinv;
#pragma unroll
    for (int n = 1; n <= N; ++n) g[n] = -R(2 * n - 1) * g[n - 1] * r2i;
}

// erfc(alpha r)/r, Smith's recursion B_n = [(2n-1)B_{n-1} + (2a^2)^n e^{-a^2 r^2}/(a sqrt(pi))]/r^2,
// g_n = (-1)^n B_n.
template <typename R, int N>
__device__ inline void g_erfc(R r, R rinv, R alpha, R *g) {
    const R r2i = rinv * rinv;
    const R ar = alpha * r;
    const R ex = exp_(-ar * ar) * (R(0.56418958354775628695) * rcp_(alpha));   // 1/(a sqrt(pi))
    R b = erfc_(ar) * rinv;
    g[0] = b;
    R tw = R(2) * alpha * alpha, p = tw;
#pragma unroll
    for (int n = 1; n <= N; ++n) {
        b = (R(2 * n - 1) * b + p * ex) * r2i;
        p *= tw;
        g[n] = (n & 1) ? -b : b;
    }
}

// exp(-b r)/r: g_n = (-1)^n e^{-b r} theta_n(b r)/r^(2n+1), theta = reverse Bessel polynomials.
template <typename R, int N>
__device__ inline void g_exp(R r, R rinv, R bb, R *g);

// same kernel with the exponent argument x = b r supplied by the caller
template <typename R, int N>
__device__ inline void g_exp_x(R x, R rinv, R *g) {
    const R e = exp_(-x) * rinv;
    R th0 = R(1), th1 = x + R(1);
    R r2i = rinv * rinv;
    R pw = e;
    g[0] = e;
    if (N >= 1) { pw *= r2i; g[1] = -th1 * pw; }
#pragma unroll
    for (int n = 2; n <= N; ++n) {
        R th2 = R(2 * n - 1) * th1 + x * x * th0;
        th0 = th1;
        th1 = th2;
        pw *= r2i;
        g[n] = (n & 1) ? -th2 * pw : th2 * pw;
    }
}

template <typename R, int N>
__device__ inline void g_exp(R r, R rinv, R bb, R *g) {
    const R x = bb * r;
    const R e = exp_(-x) * rinv;
    R th0 = R(1), th1 = x + R(1);
    R r2i = rinv * rinv;
    R pw = e;
    g[0] = e;
    if (N >= 1) { pw *= r2i; g[1] = -th1 * pw; }
#pragma unroll
    for (int n = 2; n <= N; ++n) {
        R th2 = R(2 * n - 1) * th1 + x * x * th0;
        th0 = th1;
        th1 = th2;
        pw *= r2i;
        g[n] = (n & 1) ? -th2 * pw : th2 * pw;
    }
}

// erf(alpha r)/r and its radial derivatives g_0..g_N (intramolecular Ewald
// exclusions), free of the cancellation in 1/r - erfc(alpha r)/r at small r.
// With y = (alpha r)^2 and B_n = (-1)^n g_n, term-wise differentiation of the
// Maclaurin series of erf gives
//   B_N = (2 alpha / sqrt(pi)) (2 alpha^2)^N sum_j (-y)^j / (j! (2j + 2N + 1)),
// and the erf form of the Ewald recursion runs downward without loss:
//   B_{n-1} = (r^2 B_n + (2 alpha^2)^n e^{-y} / (alpha sqrt(pi))) / (2n - 1).
// For y > 2 (no cancellation left) the difference of the two kernels is used.
template <typename R, int N>
__device__ inline void g_erf_s(R r2, R alpha, R *g) {
    const R a2 = alpha * alpha, y = a2 * r2;
    if (y > R(2)) {
        const R rinv = rsqrt_(r2);
        R gb[N + 1];
        g_bare<R, N>(rinv, gb);
        g_erfc<R, N>(r2 * rinv, rinv, alpha, g);
#pragma unroll
        for (int n = 0; n <= N; ++n) g[n] = gb[n] - g[n];
        return;
    }
    R term = R(1), s = R(1) / R(2 * N + 1);
#pragma unroll
    for (int j = 1; j <= 22; ++j) {
        term *= -y * R(1.0 / j);
        s += term * R(1.0 / (2 * j + 2 * N + 1));
        // FP64: stop once the terms (alternating, decreasing for j > y) fall
        // below the last bit; 22 terms reach it at y = 2, ~14 at the
        // intramolecular distances of a water with alpha = 0.4
        if constexpr (sizeof(R) == 8) {
            if (fabs(term) < 1e-17 * fabs(s)) break;
        }
    }
    const R tw = R(2) * a2, itw = R(1) / tw;
    R pw = R(1);
#pragma unroll
    for (int n = 0; n < N; ++n) pw *= tw;
    R B = R(1.12837916709551257390) * alpha * pw * s;                   // 2 alpha / sqrt(pi)
    const R ex = exp_(-y) * (R(0.56418958354775628695) / alpha);        // e^{-y} / (alpha sqrt(pi))
    g[N] = (N & 1) ? -B : B;
#pragma unroll
    for (int n = N; n >= 1; --n) {
        B = (r2 * B + pw * ex) * R(1.0 / (2 * n - 1));
        pw *= itw;
        g[n - 1] = ((n - 1) & 1) ? -B : B;
    }
}

// Exponential Thole factors on top of a bare or Ewald kernel for n = 1..N.
// gas:      g_n = lambda_{2n+1} g_n(1/r)
// periodic: g_n = g_n(erfc) + (lambda_{2n+1} - 1) g_n(1/r)
// gbase holds the base kernel already evaluated at r (erfc in periodic
// systems, bare in the gas phase).
template <typename R, int N>
__device__ inline void g_thole_on(R r, R rinv, R Ainv3, R a, bool periodic, const R *gbase, R *g) {
    const R t = a * r * r * r * Ainv3;
    const R e = exp_(-t);
    R lam[4];
    lam[0] = R(1) - e;
    lam[1] = R(1) - (R(1) + t) * e;
    lam[2] = R(1) - (R(1) + t + R(0.6) * t * t) * e;
    lam[3] = R(1) - (R(1) + t + R(18.0 / 35.0) * t * t + R(9.0 / 35.0) * t * t * t) * e;
    g[0] = R(0);
    if (periodic) {
        R gb[N + 1];
        g_bare<R, N>(rinv, gb);
#pragma unroll
        for (int n = 1; n <= N; ++n) g[n] = gbase[n] + (lam[n - 1] - R(1)) * gb[n];
    } else {
#pragma unroll
        for (int n = 1; n <= N; ++n) g[n] = lam[n - 1] * gbase[n];
    }
}

template <typename R, int N>
__device__ inline void g_thole(R r, R rinv, R Ainv3, R a, bool periodic, R alpha, R *g) {
    R gbase[N + 1];
    if (periodic) g_erfc<R, N>(r, rinv, alpha, gbase);
    else g_bare<R, N>(rinv, gbase);
    g_thole_on<R, N>(r, rinv, Ainv3, a, periodic, gbase, g);
}

// ---------------------------------------------------------------------------
// Potential derivatives at displacement x (target minus source) produced by a
// source multipole s through a radial kernel with weights g[0..5]:
//   phi, d1 = grad phi, d2 = grad grad phi (symmetric).
// d3 is never formed: its contraction with a target multipole is returned
// through the target-side helper below.
// ---------------------------------------------------------------------------
template <typename R>
struct FieldTerms {
    R phi;
    R phi_mp;   // the dipole and quadrupole part of phi (phi - q g0)
    V3<R> d1;
    Sym<R> d2;
    V3<R> d1_mp;   // the dipole and quadrupole parts of d1, d2 (without the charge)
    Sym<R> d2_mp;
    // intermediates for the third-derivative contraction
    R Rs, S;
    V3<R> U, W, v;
};

template <typename R, int NDER>
__device__ inline void source_field(const Mp<R> &s, V3<R> x, const R *g, FieldTerms<R> &f) {
    const R sx = dot(s.mu, x);
    const V3<R> v = symv(s.th, x);
    const R w = dot(x, v);
    const R third = R(1) / R(3), twoth = R(2) / R(3);
    f.phi_mp = third * w * g[2] - sx * g[1];
    f.phi = s.q * g[0] + f.phi_mp;
    if constexpr (NDER >= 1) {
        const R P = s.q * g[1] - sx * g[2] + third * w * g[3];
        const V3<R> Q = R(-g[1]) * s.mu + (twoth * g[2]) * v;
        f.d1 = P * x + Q;
        const R Pm = third * w * g[3] - sx * g[2];
        f.d1_mp = Pm * x + Q;
        if constexpr (NDER >= 2) {
            const R Rr = s.q * g[2] - sx * g[3] + third * w * g[4];
            const V3<R> U = R(-g[2]) * s.mu + (twoth * g[3]) * v;
            const R t2 = twoth * g[2];
            f.d2.xx = P + x.x * x.x * Rr + R(2) * x.x * U.x + t2 * s.th.xx;
            f.d2.yy = P + x.y * x.y * Rr + R(2) * x.y * U.y + t2 * s.th.yy;
            f.d2.zz = P + x.z * x.z * Rr + R(2) * x.z * U.z + t2 * s.th.zz;
            f.d2.xy = x.x * x.y * Rr + x.x * U.y + x.y * U.x + t2 * s.th.xy;
            f.d2.xz = x.x * x.z * Rr + x.x * U.z + x.z * U.x + t2 * s.th.xz;
            f.d2.yz = x.y * x.z * Rr + x.y * U.z + x.z * U.y + t2 * s.th.yz;
            const R Rm = third * w * g[4] - sx * g[3];
            f.d2_mp.xx = Pm + x.x * x.x * Rm + R(2) * x.x * U.x + t2 * s.th.xx;
            f.d2_mp.yy = Pm + x.y * x.y * Rm + R(2) * x.y * U.y + t2 * s.th.yy;
            f.d2_mp.zz = Pm + x.z * x.z * Rm + R(2) * x.z * U.z + t2 * s.th.zz;
            f.d2_mp.xy = x.x * x.y * Rm + x.x * U.y + x.y * U.x + t2 * s.th.xy;
            f.d2_mp.xz = x.x * x.z * Rm + x.x * U.z + x.z * U.x + t2 * s.th.xz;
            f.d2_mp.yz = x.y * x.z * Rm + x.y * U.z + x.z * U.y + t2 * s.th.yz;
            f.Rs = Rr;
            f.U = U;
            if constexpr (NDER >= 3) {
                f.S = s.q * g[3] - sx * g[4] + third * w * g[5];
                f.W = R(-g[3]) * s.mu + (twoth * g[4]) * v;
                f.v = v;
            }
        }
    }
}

// a^3 - b^3 and a^5 - b^5 for a = 1/|x|, b = 1/|y| from dd = |y|^2 - |x|^2
// and the lengths rx = |x|, ry = |y|, without the cancellation of the direct
// differences (a - b = dd a b / (rx + ry)).
template <typename R>
__device__ inline void ref_diff35(R dd, R a, R b, R rx, R ry, R &d3, R &d5) {
    const R d1 = dd * a * b / (rx + ry);
    const R a2 = a * a, b2 = b * b, ab = a * b;
    d3 = d1 * (a2 + ab + b2);
    d5 = d1 * (a2 * a2 + ab * (a2 + b2) + ab * ab + b2 * b2);
}

// Target contraction.  Energy U = q phi + mu.d1 + (1/3) Th:d2; gradient of U
// with respect to the target position (= -force) needs d3:
//   dU/dx = q d1 + d2.mu + (1/3) Th : d3.
// With Phi = target quadrupole (traceless), Theta = source quadrupole:
//   (Phi:d3)_a = 2 (Phi (x R + U))_a + x_a [ (x Phi x) S + 2 x.Phi.W ]
//               + (x Phi x) W_a + (2/3) g3 [ 2 (Theta Phi x)_a + x_a (Phi:Theta) ]
template <typename R>
__device__ inline V3<R> target_grad(const Mp<R> &t, const Mp<R> &s, V3<R> x, const R *g,
                                    const FieldTerms<R> &f) {
    V3<R> gr = t.q * f.d1 + symv(f.d2, t.mu);
    const V3<R> px = symv(t.th, x);
    const R xpx = dot(x, px);
    const V3<R> a1 = f.Rs * px + symv(t.th, f.U);       // Phi (x R + U)
    const R xpw = dot(px, f.W);
    const V3<R> thpx = symv(s.th, px);                   // Theta Phi x
    const R pdt = symdd(t.th, s.th);
    const R c3 = R(2.0 / 3.0) * g[3];
    V3<R> th3 = R(2) * a1 + (xpx * f.S + R(2) * xpw) * x + xpx * f.W + c3 * (R(2) * thpx + pdt * x);
    return gr + R(1.0 / 3.0) * th3;
}

// ---------------------------------------------------------------------------
// Cardinal B-spline weights of order 5 and derivatives (w.r.t. u) at
// arguments w + j, j = 0..4, w = frac(u); grid point of j is floor(u) - j.
// ---------------------------------------------------------------------------
template <typename R, int NDER>
__device__ inline void bspline5(R w, R *m0, R *m1, R *m2, R *m3) {
    R b2[2] = {w, R(1) - w};
    R b3[3], b4[4];
    // order 3
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        R v = w + R(j);
        R a = (j <= 1) ? b2[j] : R(0);
        R b = (j >= 1) ? b2[j - 1] : R(0);
        b3[j] = (v * a + (R(3) - v) * b) * R(0.5);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        R v = w + R(j);
        R a = (j <= 2) ? b3[j] : R(0);
        R b = (j >= 1) ? b3[j - 1] : R(0);
        b4[j] = (v * a + (R(4) - v) * b) * R(1.0 / 3.0);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        R v = w + R(j);
        R a = (j <= 3) ? b4[j] : R(0);
        R b = (j >= 1) ? b4[j - 1] : R(0);
        m0[j] = (v * a + (R(5) - v) * b) * R(0.25);
        if constexpr (NDER >= 1) m1[j] = a - b;
        if constexpr (NDER >= 2) {
            R c0 = (j <= 2) ? b3[j] : R(0);
            R c1 = (j >= 1 && j <= 3) ? b3[j - 1] : R(0);
            R c2 = (j >= 2) ? b3[j - 2] : R(0);
            m2[j] = c0 - R(2) * c1 + c2;
        }
        if constexpr (NDER >= 3) {
            R d0 = (j <= 1) ? b2[j] : R(0);
            R d1 = (j >= 1 && j <= 2) ? b2[j - 1] : R(0);
            R d2 = (j >= 2 && j <= 3) ? b2[j - 2] : R(0);
            R d3 = (j >= 3) ? b2[j - 3] : R(0);
            m3[j] = d0 - R(3) * d1 + R(3) * d2 - d3;
        }
    }
}

// ---------------------------------------------------------------------------
// Warp reduction in double
// ---------------------------------------------------------------------------
__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums NV per-lane values over the warp, transposed: on return lane k < NV
// holds the sum of value k over the 32 lanes (other lanes hold 0).  The
// values pass through buf (NV * 33 elements of this warp's shared memory,
// padded so that both the writes and the column sums are conflict-free);
// the caller then needs one FP64 operation per value instead of a shuffle
// tree per value.
template <typename R, int NV>
__device__ inline R warp_transpose_sum(const R (&v)[NV], R *buf, int lane) {
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k * 33 + lane] = v[k];
    __syncwarp();
    R s0 = R(0), s1 = R(0);
    if (lane < NV) {
#pragma unroll 8
        for (int j = 0; j < 32; j += 2) {
            s0 += buf[lane * 33 + j];
            s1 += buf[lane * 33 + j + 1];
        }
    }
    __syncwarp();
    return s0 + s1;
}

// Virial epilogue of the molecule-pair kernels (translation-invariance form):
// lanes 0-14 hold the warp-reduced gradients g of i's points O, H1, H2, LP1,
// LP2 (offsets P from O_i); adds sum_p G_p (x) off_p and the warp sum of the
// per-lane W to vir[i].
template <typename R>
__device__ inline void vir_points_out(const DevState<R> &d, int i, const V3<R> (&P)[5], R g, const R (&W)[9],
                                      R *buf, int lane) {
    __syncwarp();
    if (lane < 15) buf[lane] = g;
    __syncwarp();
    R wo = R(0);
    if (lane < 9) {
        const int a = lane / 3, b = lane % 3;
#pragma unroll
        for (int k = 0; k < 5; ++k) wo += buf[k * 3 + a] * (b == 0 ? P[k].x : (b == 1 ? P[k].y : P[k].z));
    }
    __syncwarp();
    const R wv = warp_transpose_sum<R, 9>(W, buf, lane);
    if (lane < 9) d.vir[i * 9 + lane] += double(wo) + double(wv);
}

// position of point k of molecule m relative to its O (points: 5 sites, 2 lone pairs)
template <typename R>
__device__ inline V3<R> my_pt(const DevState<R> &d, int i, int pt) {
    const R *o = d.off + (i * NP + pt) * 3;
    return mk(o[0], o[1], o[2]);
}

// cos(u, v) and its gradients with respect to u and v
template <typename R>
__device__ inline R cosv(V3<R> u, V3<R> v, V3<R> &du, V3<R> &dv) {
    const R uu = dot(u, u), vv = dot(v, v);
    const R iu = rsqrt_(uu), iv = rsqrt_(vv);
    const R c = dot(u, v) * iu * iv;
    du = (iu * iv) * v - (c * iu * iu) * u;
    dv = (iu * iv) * u - (c * iv * iv) * v;
    return c;
}

// exclusive prefix sum of c over the lanes of a warp; total = sum over all lanes
__device__ inline int warp_excl_scan(int c, int lane, int &total) {
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - c;
}

// Compensated (two-sum) accumulator used for per-lane energy partial sums.
template <typename R>
struct Acc {
    R hi = R(0), lo = R(0);
    __device__ inline void add(R v) {
        R s = hi + v;
        R bp = s - hi;
        R err = (hi - (s - bp)) + (v - bp);
        hi = s;
        lo += err;
    }
    __device__ inline double get() const { return double(hi) + double(lo); }
};

// Warp sum of compensated partials.  FP32: a two-sum butterfly on (hi, lo)
// pairs, so the only FP64 work is the final conversion; FP64: plain tree.
__device__ inline double warp_sum_acc(const Acc<float> &a) {
    float hi = a.hi, lo = a.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = hi + h2, bp = s - hi;
        const float err = (hi - (s - bp)) + (h2 - bp);
        hi = s;
        lo = lo + l2 + err;
    }
    return double(hi) + double(lo);
}
__device__ inline double warp_sum_acc(const Acc<double> &a) { return warp_sum(a.get()); }

// Minimum-image displacement of molecule j's O from molecule i's O (FP64).
__device__ inline void min_image(const KParams &p, const double *pos, int i, int j, double &dx, double &dy,
                                 double &dz) {
    dx = pos[j * 9 + 0] - pos[i * 9 + 0];
    dy = pos[j * 9 + 1] - pos[i * 9 + 1];
    dz = pos[j * 9 + 2] - pos[i * 9 + 2];
    if (p.periodic) {
        dx -= p.box[0] * rint(dx * p.ibox[0]);
        dy -= p.box[1] * rint(dy * p.ibox[1]);
        dz -= p.box[2] * rint(dz * p.ibox[2]);
    }
}

// source multipole row through the read-only path with vector loads (rows
// are GMP values long, so every row starts on a 16-byte boundary)
template <typename R>
__device__ inline Mp<R> load_mp_g(const R *g);
template <>
__device__ inline Mp<float> load_mp_g<float>(const float *g) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(g));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(g) + 1);
    const float2 c = __ldg(reinterpret_cast<const float2 *>(g) + 4);
    Mp<float> m;
    m.q = a.x;
    m.mu = mk(a.y, a.z, a.w);
    m.th = Sym<float>{b.x, b.y, b.z, b.w, c.x, c.y};
    return m;
}
template <>
__device__ inline Mp<double> load_mp_g<double>(const double *g) {
    const double2 *v = reinterpret_cast<const double2 *>(g);
    const double2 a = __ldg(v), b = __ldg(v + 1), c = __ldg(v + 2), e = __ldg(v + 3), f = __ldg(v + 4);
    Mp<double> m;
    m.q = a.x;
    m.mu = mk(a.y, b.x, b.y);
    m.th = Sym<double>{c.x, c.y, e.x, e.y, f.x, f.y};
    return m;
}

template <typename R>
__device__ inline Mp<R> load_mp(const R *g) {
    Mp<R> m;
    m.q = g[0];
    m.mu = mk(g[1], g[2], g[3]);
    m.th = Sym<R>{g[4], g[5], g[6], g[7], g[8], g[9]};
    return m;
}

// ---------------------------------------------------------------------------
// Local frames of a water (shared by the site kernel and the chain rule, so
// both see the same axes).  W is the arithmetic type: FP64 on the FP64 path,
// FP32 on the mixed path, where the rotated multipoles and point offsets are
// stored in FP32 anyway.
// ---------------------------------------------------------------------------
// Bond vectors r1 = H1 - O, r2 = H2 - O: FP64 differences, rounded once to W.
template <typename W>
__device__ inline void bond_vectors(const double *x, V3<W> &r1, V3<W> &r2) {
    r1 = mk(W(x[3] - x[0]), W(x[4] - x[1]), W(x[5] - x[2]));
    r2 = mk(W(x[6] - x[0]), W(x[7] - x[1]), W(x[8] - x[2]));
}

// Axis generators of frame f: frame 0 (O, lone pairs) has z along the
// bisector u1 + u2 (u = r / |r|) and x toward H1; frame 1 (H1, O-H1
// midpoint) has z along O - H1 and x toward H2; frame 2 (H2, O-H2 midpoint)
// has z along O - H2 and x toward H1.  s1 = 1/|r1|, s2 = 1/|r2|.
template <typename W>
__device__ inline void frame_generators(int f, V3<W> r1, V3<W> r2, W s1, W s2, V3<W> &zv, V3<W> &xv) {
    const V3<W> b = s1 * r1 + s2 * r2;
    zv = f == 0 ? b : (f == 1 ? -r1 : -r2);
    xv = f == 0 ? r1 : (f == 1 ? r2 - r1 : r1 - r2);
}

// Orthonormal frame with z along zv and x in the (z, xv) plane; y = z x x.
template <typename W>
__device__ inline void frame_axes(V3<W> zv, V3<W> xv, V3<W> &ex, V3<W> &ey, V3<W> &ez) {
    ez = rsqrt_<W>(dot(zv, zv)) * zv;
    const V3<W> xp = xv - dot(xv, ez) * ez;
    ex = rsqrt_<W>(dot(xp, xp)) * xp;
    ey = cross(ez, ex);
}

// frame carrying site s: O -> 0, H1 and the O-H1 midpoint -> 1, H2 and the O-H2 midpoint -> 2
__device__ inline int site_frame(int s) { return s == 0 ? 0 : (s == 1 || s == 3 ? 1 : 2); }

// ---------------------------------------------------------------------------
// Host-side launchers (explicitly instantiated for float and double)
// ---------------------------------------------------------------------------
struct Launch {
    cudaStream_t s;
    uint64_t *count;
};

template <typename R> void launch_sites(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_neighbors(const KParams &p, DevState<R> &d, int ncell[3], Launch L);
template <typename R> void launch_real_perm(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_lp_potential(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_short(const KParams &p, DevState<R> &d, Launch L, int max_blocks = 0,
                                         int max_per_sm = 0);
template <typename R> void launch_ct(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_intra_perm(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_real_tmu(const KParams &p, DevState<R> &d, double *out,
                                           Launch L);
template <typename R> void launch_real_polforce(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_intra_polforce(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_finalize(const KParams &p, DevState<R> &d, double *forces_out, Launch L);
template <typename R> void launch_merge_rec(const KParams &p, DevState<R> &d, Launch L);

// The view of a state whose accumulators are the reciprocal-chain set.
template <typename R>
inline DevState<R> rec_view(const DevState<R> &d) {
    DevState<R> r = d;
    r.gpt = d.gpt_r;
    r.gmu = d.gmu_r;
    r.gth = d.gth_r;
    r.efield = d.efield_r;
    r.vlp = d.vlp_r;
    r.dvlp = d.dvlp_r;
    r.va = d.va_r;
    r.dva = d.dva_r;
    r.epart = d.epart_r;
    r.vir = d.vir_r;
    return r;
}
// the short-range kernels' view: their own point-gradient array
template <typename R>
inline DevState<R> short_view(const DevState<R> &d) {
    DevState<R> r = d;
    r.gpt = d.gpt_s;
    return r;
}

// SPME
enum SpreadKind { SPREAD_PERM = 0, SPREAD_DIP = 1, SPREAD_LAMBDA = 2, SPREAD_DIP_PCG = 3 };
template <typename R> void launch_spread(const KParams &p, DevState<R> &d, int kind, const double *vec, R *grid,
                                         Launch L);
template <typename R> void launch_convolve(const KParams &p, DevState<R> &d, void *cgrid, int ngrid, int check,
                                           Launch L);
template <typename R> void launch_gather_perm(const KParams &p, DevState<R> &d, Launch L);
template <typename R> void launch_gather_field(const KParams &p, DevState<R> &d, double *out, Launch L);
template <typename R> void launch_gather_polforce(const KParams &p, DevState<R> &d, Launch L);
void launch_influence(const KParams &p, double *infl, Launch L);
template <typename R> void launch_influence_copy(const KParams &p, DevState<R> &d, Launch L);

// PCG
template <typename R> void launch_pcg_init(const KParams &p, DevState<R> &d, int warm, Launch L);
template <typename R> void launch_pcg_first(const KParams &p, DevState<R> &d, Launch L);
// maxit > 0: inside the solver graph, also set the loop condition through `loop`
template <typename R> void launch_pcg_step(const KParams &p, DevState<R> &d, Launch L,
                                           cudaGraphConditionalHandle loop = 0, int maxit = 0);
template <typename R> void launch_pol_energy(const KParams &p, DevState<R> &d, Launch L);
void launch_energy_reduce(int M, const double *epart, const double *epart_r, const double *eintra, double *partial,
                          double *out, Launch L);
// mixed periodic path: the intramolecular Ewald energy of every molecule in FP64 into eintra
template <typename R> void launch_intra_energy64(const KParams &p, DevState<R> &d, Launch L);
// k-space virial sums of one convolution pass (0: permanent, 1: force pass) fused with the convolution
template <typename R> void launch_convolve_vir(const KParams &p, DevState<R> &d, int pass, Launch L);
// out[9] = -dE/d eps summed over molecules, both chains and the k-space partials
template <typename R> void launch_virial_total(const KParams &p, DevState<R> &d, double *out, Launch L);
template <typename R> void launch_cluster_energy(const KParams &p, DevState<R> &d, double *out, Launch L);
void launch_begin(double *scal, int *flags, double tol_D, Launch L);
void launch_pcg_check(const double *scal, int *flags, Launch L);
void launch_water_intra(int M, const double *pos, double *F, double kb, double r0, double ka, double th0, int anh,
                        double kub, double rub, Launch L);
void launch_beeman(int M, double *pos, double *vel, const double *inv_mass, double *F, double *Fprev, double dt,
                   int half, Launch L);
void launch_sd_step(int M, double *pos, const double *F, double gamma, double cap, Launch L);
enum { SC_RZ = 0, SC_RES = 4, SC_IT = 6, SC_DONE = 7, SC_TOL = 8 };
void launch_md_kick(int M, double *pos, double *vel, const double *inv_mass, const double *forces, double dt,
                    int drift, Launch L);

inline void count(Launch &L, int n = 1) {
    if (L.count) *L.count += n;
}

}  // namespace sibfa
