// Exchange-repulsion (Technical Appendix: S^2/R and S^2/R^2 overlap terms
// over bond-bond, bond-lone pair and lone pair-lone pair pairs), dispersion
// (C6/C8/C10 with damping) and exchange-dispersion.
//
// One warp per molecule i walks its neighbour list 32 entries at a time.
// Every molecule pair (i, j) expands into 41 items:
//   BB  bond O-H_kb of i with bond O-H_kc of j          4
//   BL  bond of i with lone pair l of j                 4
//   LB  lone pair l of i with bond of j                 4
//   LL  lone pair of i with lone pair of j              4
//   D   point u of i with the points v of j            5    (u, v: O, H1, H2, LP1, LP2)
// Repulsion items inside the cutoff (per item, on the distance of its radial
// factor) are appended to one ring queue per class in shared memory and
// evaluated in full 32-lane rounds, so all lanes of a round do the same work.
// A dispersion item is a point u of i with every point v of j, queued when
// at least one of the five point pairs is inside the cutoff and carrying the
// mask of those that are; the lane runs the five v unrolled, so the
// partner's data and u's factors are read once per item.  Gradients go to i's
// points only (the full list visits each pair from both sides).
#include <cstddef>

#include "sibfa_internal.cuh"

namespace sibfa {

// Atom-pair overlap with each p orbital measured at its own atom:
// O = A + B cx + C cy + D cx cy, cx = cos(ux, y - x), cy = cos(uy, x - y),
// ux = xp - x (xp an i-side point), uy fixed (j side).
// Returns O; gx = dO/dx and gxp = dO/dxp.
template <typename R>
__device__ inline R overlap_i(V3<R> x, V3<R> xp, V3<R> y, V3<R> uy, R A, R B, R C, R D, V3<R> &gx, V3<R> &gxp) {
    V3<R> du, dv, du2, dv2;
    const R cx = cosv(xp - x, y - x, du, dv);
    const R cy = cosv(uy, x - y, du2, dv2);
    const R ox = B + D * cy, oy = C + D * cx;
    gxp = ox * du;
    gx = R(-1) * ox * (du + dv) + oy * dv2;
    return A + B * cx + C * cy + D * cx * cy;
}

template <typename R>
struct RepAtom {
    R cs, cp, g, cf;
    int kind;   // 0 = O, 1 = H, 2 = lone pair (selects the pair-type exponent coefficients)
    R sg;       // sqrt(g cf): the pair prefactor sqrt(g_a g_b cf_a cf_b) is sg_a sg_b
};

template <typename R>
__device__ inline RepAtom<R> rep_atom(R cs, R cp, R g, R cf, int kind) {
    return {cs, cp, g, cf, kind, sqrt_(g * cf)};
}

// Pair-type coefficient tables copied to shared memory: items of one round
// mix pair types, and divergent indices into the parameter bank serialise.
struct ShortTables {
    KParams::Coef rep_k1[3][3], rep_k2[3][3], disp_km[3][3], disp_gS[3][3][3], xd_k[3][3];
};

// Adds the overlap and exponential factor of one atom pair to O1/O2 and the
// i-side gradients dO1/dx, dO1/dxp, dO2/dx, dO2/dxp.
template <typename R>
__device__ inline void rep_pair_term(V3<R> x, V3<R> xp, const RepAtom<R> &ai, V3<R> y, V3<R> uy, const RepAtom<R> &aj,
                                     R pp, R f, const ShortTables &T, R &O1, R &O2, V3<R> &g1x, V3<R> &g1xp,
                                     V3<R> &g2x, V3<R> &g2xp) {
    V3<R> gx, gxp;
    const R O = overlap_i(x, xp, y, uy, ai.cs * aj.cs, aj.cs * ai.cp * f, ai.cs * aj.cp * f, pp * ai.cp * aj.cp, gx, gxp);
    const V3<R> v = x - y;
    const R vv = dot(v, v), irr = rsqrt_(vv), rr = vv * irr;
    const KParams::Coef &k1 = T.rep_k1[ai.kind][aj.kind], &k2 = T.rep_k2[ai.kind][aj.kind];
    const R M = ai.sg * aj.sg;
    const R S1 = M * exp_(-mulc(rr, k1)), S2 = M * exp_(-mulc(rr, k2));
    O1 += O * S1;
    O2 += O * S2;
    const V3<R> drdx = irr * v;
    g1x = S1 * gx + (O * S1 * (-cval<R>(k1))) * drdx;
    g2x = S2 * gx + (O * S2 * (-cval<R>(k2))) * drdx;
    g1xp = S1 * gxp;
    g2xp = S2 * gxp;
}

// E = pref (C1 O1^2 / r + C2 O2^2 / r^2) from ri = 1/r: returns E and dE/dO1,
// dE/dO2, dE/dr.
template <typename R>
__device__ inline R rep_energy(R pref, R C1, R C2, R O1, R O2, R ri, R &e1, R &e2, R &er) {
    e1 = pref * C1 * R(2) * O1 * ri;
    e2 = pref * C2 * R(2) * O2 * ri * ri;
    er = pref * (-C1 * O1 * O1 * ri * ri - R(2) * C2 * O2 * O2 * ri * ri * ri);
    return pref * (C1 * O1 * O1 * ri + C2 * O2 * O2 * ri * ri);
}

// Queue layout (words: slot * 32 + item code)
constexpr int SQ_BB = 0, SQ_BL = 160, SQ_LB = 320, SQ_LL = 480, SQ_D = 640;
constexpr int SQ_CAP = 160;    // >= 31 carried + 32 lanes x 4 items
constexpr int SQ_CAPD = 192;   // >= 31 carried + 32 lanes x 5 items (points u of i)
constexpr int SQ_WORDS = 1024; // also holds the FP64 reduction buffer (15 x 33 doubles)

// i-side state of one warp
template <typename R>
struct ShortI {
    V3<R> P[5];            // O, H1, H2, LP1, LP2 relative to O_i
    RepAtom<R> A[3];       // O, H1, H2 of i
    R cf[5];               // valence factors 1 - q/N of O, H1, H2 and (O's) for the lone pairs
};

template <typename R>
struct ShortAcc {
    V3<R> G[5];
    Acc<R> Erep, Ed, Ex;
    R W[9];   // virial: -1/2 sum over items of (gradient on i's points) (x) dO_ij (VIR kernels only)
};

template <typename R>
__device__ inline void addG(ShortAcc<R> &a, int k, V3<R> v) {
#pragma unroll
    for (int t = 0; t < 5; ++t)
        if (t == k) a.G[t] = a.G[t] + v;
}
template <typename R>
__device__ inline V3<R> selP(const ShortI<R> &I, int k) {
    V3<R> r = I.P[0];
#pragma unroll
    for (int t = 1; t < 5; ++t)
        if (t == k) r = I.P[t];
    return r;
}

// Per-molecule data of the short-range items, packed so that an item reads
// one aligned 4-vector per point of its neighbour: for the points O, H1, H2,
// LP1, LP2 the offset from O and the valence factor 1 - q/N_val of the
// point's atom (O's for the lone pairs).  Written each evaluation before the
// short-range launches, from the site offsets and the global charges.
constexpr int SPK = 5 * 4;
template <typename R>
__global__ void k_short_pack(KParams p, DevState<R> d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.M * 5) return;
    const Scal<R> &S = sc<R>(p);
    const int m = t / 5, k = t % 5;
    const int s = k < 3 ? k : k + 2, a = k < 3 ? k : 0;
    const R *o = d.off + (m * NP + s) * 3;
    const R q = d.gmp[(m * NS + a) * GMP];
    R *w = d.spk + (size_t)t * 4;
    w[0] = o[0];
    w[1] = o[1];
    w[2] = o[2];
    w[3] = R(1) - q * (a == 0 ? S.inv_nval_o : S.inv_nval_h);
}

template <typename R>
__device__ inline void ld4(const R *w, R &a, R &b, R &c, R &e);
template <>
__device__ inline void ld4<float>(const float *w, float &a, float &b, float &c, float &e) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(w));
    a = v.x, b = v.y, c = v.z, e = v.w;
}
template <>
__device__ inline void ld4<double>(const double *w, double &a, double &b, double &c, double &e) {
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(w)), v1 = __ldg(reinterpret_cast<const double2 *>(w) + 1);
    a = v0.x, b = v0.y, c = v1.x, e = v1.y;
}

// point k (0 O, 1 H1, 2 H2, 3 LP1, 4 LP2) of neighbour j relative to O_i,
// and the valence factor of its atom
template <typename R>
__device__ inline V3<R> qpt(const DevState<R> &d, int j, V3<R> dO, int k, R &cf) {
    R a, b, c;
    ld4(d.spk + ((size_t)j * 5 + k) * 4, a, b, c, cf);
    return dO + mk(a, b, c);
}
template <typename R>
__device__ inline V3<R> qpt(const DevState<R> &d, int j, V3<R> dO, int k) {
    R cf;
    return qpt(d, j, dO, k, cf);
}
// valence factor of atom k (0 O, 1 H1, 2 H2) of molecule j
template <typename R>
__device__ inline R qcf(const DevState<R> &d, int j, int k) { return d.spk[((size_t)j * 5 + k) * 4 + 3]; }

template <typename R>
__device__ inline RepAtom<R> atom_j(const Scal<R> &S, R cf, int k) {
    if (k == 0) return rep_atom(S.cs_o, S.cp_o, S.g_o, cf, 0);
    return rep_atom(S.cs_h, S.cp_h, S.g_h, cf, 1);
}

template <typename R>
__device__ inline void neighbour(const DevState<R> &d, int i, int slot, int &j, V3<R> &dO) {
    j = d.nbr[i * MAXN + slot];
    const R *dp = d.ndo + ((size_t)i * MAXN + slot) * 3;
    dO = mk(dp[0], dp[1], dp[2]);
}

// ---- item evaluation -------------------------------------------------------

template <typename R, bool VIR>
__device__ void item_bb(const Scal<R> &S, const ShortTables &T, const DevState<R> &d, const ShortI<R> &I, int i,
                        int word, ShortAcc<R> &a) {
    const int slot = word >> 5, c = word & 31;
    const int kb = 1 + (c >> 1), kc = 1 + (c & 1);
    int j;
    V3<R> dO;
    neighbour(d, i, slot, j, dO);
    const V3<R> P0 = I.P[0], Pb = kb == 1 ? I.P[1] : I.P[2];
    const RepAtom<R> Ab = kb == 1 ? I.A[1] : I.A[2];
    R cfc;
    const V3<R> Q0 = dO, Qc = qpt(d, j, dO, kc, cfc);
    const RepAtom<R> AjO = atom_j(S, qcf(d, j, 0), 0), Ajc = atom_j(S, cfc, kc);
    const V3<R> dm = R(0.5) * (P0 + Pb) - R(0.5) * (Q0 + Qc);
    const R irm = rsqrt_(dot(dm, dm));
    R O1 = 0, O2 = 0;
    const V3<R> z = mk(R(0), R(0), R(0));
    V3<R> g1a = z, g1b = z, g2a = z, g2b = z;   // gradients at O_i (a) and H_kb (b)
#pragma unroll 1
    for (int uv = 0; uv < 4; ++uv) {
        const bool u = uv >> 1, v = uv & 1;
        V3<R> t1x, t1xp, t2x, t2xp;
        rep_pair_term(u ? Pb : P0, u ? P0 : Pb, u ? Ab : I.A[0], v ? Qc : Q0, v ? Q0 - Qc : Qc - Q0, v ? Ajc : AjO,
                      R(2), S.rep_f, T, O1, O2, t1x, t1xp, t2x, t2xp);
        if (!u) { g1a = g1a + t1x; g2a = g2a + t2x; g1b = g1b + t1xp; g2b = g2b + t2xp; }
        else { g1b = g1b + t1x; g2b = g2b + t2x; g1a = g1a + t1xp; g2a = g2a + t2xp; }
    }
    R e1, e2, er;
    a.Erep.add(R(0.5) * rep_energy(S.occ * S.occ, S.rep_c1, S.rep_c2, O1, O2, irm, e1, e2, er));
    const V3<R> drm = (R(0.5) * irm) * dm;
    const V3<R> ga = e1 * g1a + e2 * g2a + er * drm, gb = e1 * g1b + e2 * g2b + er * drm;
    a.G[0] = a.G[0] + ga;
    addG(a, kb, gb);
    if (VIR) vir_add(a.W, ga + gb, dO, R(-0.5));
}

template <typename R, bool VIR>
__device__ void item_bl(const Scal<R> &S, const ShortTables &T, const DevState<R> &d, const ShortI<R> &I, int i,
                        int word, ShortAcc<R> &a) {
    const int slot = word >> 5, c = word & 31;
    const int kb = 1 + (c >> 1), l = c & 1;
    int j;
    V3<R> dO;
    neighbour(d, i, slot, j, dO);
    const V3<R> P0 = I.P[0], Pb = kb == 1 ? I.P[1] : I.P[2];
    const RepAtom<R> Ab = kb == 1 ? I.A[1] : I.A[2];
    const V3<R> Ql = qpt(d, j, dO, 3 + l);
    const RepAtom<R> Alp = rep_atom(S.cs_lp, S.cp_lp, S.g_o, R(1) - S.nlp * S.inv_nval_o, 2);
    const V3<R> dm = R(0.5) * (P0 + Pb) - Ql;
    const R irr = rsqrt_(dot(dm, dm));
    R O1 = 0, O2 = 0;
    const V3<R> z = mk(R(0), R(0), R(0));
    V3<R> g1a = z, g1b = z, g2a = z, g2b = z;
#pragma unroll 1
    for (int u = 0; u < 2; ++u) {
        V3<R> t1x, t1xp, t2x, t2xp;
        rep_pair_term(u ? Pb : P0, u ? P0 : Pb, u ? Ab : I.A[0], dO, Ql - dO, Alp, S.rep_f, S.rep_f, T, O1, O2, t1x,
                      t1xp, t2x, t2xp);
        if (!u) { g1a = g1a + t1x; g2a = g2a + t2x; g1b = g1b + t1xp; g2b = g2b + t2xp; }
        else { g1b = g1b + t1x; g2b = g2b + t2x; g1a = g1a + t1xp; g2a = g2a + t2xp; }
    }
    R e1, e2, er;
    a.Erep.add(R(0.5) * rep_energy(S.occ * S.nlp, S.rep_c1, S.rep_c2, O1, O2, irr, e1, e2, er));
    const V3<R> drm = (R(0.5) * irr) * dm;
    const V3<R> ga = e1 * g1a + e2 * g2a + er * drm, gb = e1 * g1b + e2 * g2b + er * drm;
    a.G[0] = a.G[0] + ga;
    addG(a, kb, gb);
    if (VIR) vir_add(a.W, ga + gb, dO, R(-0.5));
}

// lone pair of i (a pseudo-atom at its carrier O_i) with a bond of j
template <typename R, bool VIR>
__device__ void item_lb(const Scal<R> &S, const ShortTables &T, const DevState<R> &d, const ShortI<R> &I, int i,
                        int word, ShortAcc<R> &a) {
    const int slot = word >> 5, c = word & 31;
    const int l = c >> 1, kc = 1 + (c & 1);
    int j;
    V3<R> dO;
    neighbour(d, i, slot, j, dO);
    const V3<R> P0 = I.P[0], Pl = l ? I.P[4] : I.P[3];
    R cfc;
    const V3<R> Q0 = dO, Qc = qpt(d, j, dO, kc, cfc);
    const RepAtom<R> AjO = atom_j(S, qcf(d, j, 0), 0), Ajc = atom_j(S, cfc, kc);
    const RepAtom<R> Alp = rep_atom(S.cs_lp, S.cp_lp, S.g_o, R(1) - S.nlp * S.inv_nval_o, 2);
    const V3<R> dm = Pl - R(0.5) * (Q0 + Qc);
    const R irr = rsqrt_(dot(dm, dm));
    R O1 = 0, O2 = 0;
    const V3<R> z = mk(R(0), R(0), R(0));
    V3<R> g1c = z, g1l = z, g2c = z, g2l = z;
#pragma unroll 1
    for (int v = 0; v < 2; ++v) {
        V3<R> t1x, t1xp, t2x, t2xp;
        rep_pair_term(P0, Pl, Alp, v ? Qc : Q0, v ? Q0 - Qc : Qc - Q0, v ? Ajc : AjO, S.rep_f, S.rep_f, T, O1, O2,
                      t1x, t1xp, t2x, t2xp);
        g1c = g1c + t1x; g2c = g2c + t2x; g1l = g1l + t1xp; g2l = g2l + t2xp;
    }
    R e1, e2, er;
    a.Erep.add(R(0.5) * rep_energy(S.occ * S.nlp, S.rep_c1, S.rep_c2, O1, O2, irr, e1, e2, er));
    const V3<R> gc = e1 * g1c + e2 * g2c, gl = e1 * g1l + e2 * g2l + (er * irr) * dm;
    a.G[0] = a.G[0] + gc;
    addG(a, 3 + l, gl);
    if (VIR) vir_add(a.W, gc + gl, dO, R(-0.5));
}

// lone pair - lone pair, angles toward the other lone pair's position
template <typename R, bool VIR>
__device__ void item_ll(const Scal<R> &S, const ShortTables &T, const DevState<R> &d, const ShortI<R> &I, int i,
                        int word, ShortAcc<R> &a) {
    const int slot = word >> 5, c = word & 31;
    const int l1 = c >> 1, l2 = c & 1;
    int j;
    V3<R> dO;
    neighbour(d, i, slot, j, dO);
    const V3<R> P0 = I.P[0], Ip = l1 ? I.P[4] : I.P[3];
    const V3<R> Jp = qpt(d, j, dO, 3 + l2);
    const V3<R> dIJ = Ip - Jp;
    const R irr = rsqrt_(dot(dIJ, dIJ));
    V3<R> dui, dvi, duj, dvj;
    const R ci = cosv(Ip - P0, Jp - P0, dui, dvi);   // depends on I and A
    const R cj = cosv(Jp - dO, Ip - dO, duj, dvj);   // depends on I
    const R cs = S.cs_lp, cp = S.cp_lp, f = S.rep_f;
    const R O = cs * cs + cs * cp * f * cj + cs * cp * f * ci + R(2) * cp * cp * ci * cj;
    const R dci = cs * cp * f + R(2) * cp * cp * cj, dcj = cs * cp * f + R(2) * cp * cp * ci;
    const V3<R> dOdI = dci * dui + dcj * dvj;
    const V3<R> dOdA = R(-1) * dci * (dui + dvi);
    const V3<R> dAB = P0 - dO;
    const R ab2 = dot(dAB, dAB), irab = rsqrt_(ab2), rab = ab2 * irab;
    const R M = S.g_o * (R(1) - S.nlp * S.inv_nval_o);
    const R S1 = M * exp_(-mulc(rab, T.rep_k1[2][2])), S2 = M * exp_(-mulc(rab, T.rep_k2[2][2]));
    const R O1 = O * S1, O2 = O * S2;
    R e1, e2, er;
    a.Erep.add(R(0.5) * rep_energy(S.nlp * S.nlp, S.rep_c1, S.rep_c2, O1, O2, irr, e1, e2, er));
    const V3<R> drab = irab * dAB;
    const V3<R> go = (e1 * S1 + e2 * S2) * dOdA +
                     (e1 * O1 * (-cval<R>(T.rep_k1[2][2])) + e2 * O2 * (-cval<R>(T.rep_k2[2][2]))) * drab;
    const V3<R> gl = (e1 * S1 + e2 * S2) * dOdI + (er * irr) * dIJ;
    a.G[0] = a.G[0] + go;
    addG(a, 3 + l1, gl);
    if (VIR) vir_add(a.W, go + gl, dO, R(-0.5));
}

// dispersion and exchange-dispersion of point u of i with the points v of j
// whose bits are set in vmask (v = 0..4 unrolled: the partner's point, kind
// and prefactors are compile-time per v; the neighbour's data and u's are
// read once per item)
template <typename R, bool VIR>
__device__ void item_du(const KParams &p, const Scal<R> &S, const ShortTables &T, const DevState<R> &d,
                        const ShortI<R> &I, int i, int word, ShortAcc<R> &a) {
    const int slot = word >> 8, u = (word >> 5) & 7, vmask = word & 31;
    int j;
    V3<R> dO;
    neighbour(d, i, slot, j, dO);
    const V3<R> Pu = selP(I, u);
    const int ku = u == 0 ? 0 : (u < 3 ? 1 : 2);
    const bool lu = u >= 3;
    const R bu = betap<R>(p, u), nlp = S.nlp;
    R cfi = I.cf[0];
#pragma unroll
    for (int t = 1; t < 5; ++t)
        if (t == u) cfi = I.cf[t];
    V3<R> gu = mk(R(0), R(0), R(0));
    R ed = R(0), ex_sum = R(0);   // this item's few terms, then one compensated add each
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        if (!((vmask >> v) & 1)) continue;
        R cfj;
        const V3<R> dv = Pu - qpt(d, j, dO, v, cfj);
        const R r2 = dot(dv, dv);
        const R ri = rsqrt_(r2), r = r2 * ri;
        const int kv = v == 0 ? 0 : (v < 3 ? 1 : 2);
        const R m = mulc(r, T.disp_km[ku][kv]), mi = rcp_(m);
        const R a6 = mulc(ri, T.disp_gS[0][ku][kv]), a8 = mulc(ri, T.disp_gS[1][ku][kv]),
                a10 = mulc(ri, T.disp_gS[2][ku][kv]);
        const R m2i = mi * mi, m6i = m2i * m2i * m2i, m8i = m6i * m2i, m10i = m8i * m2i;
        const R e6 = S.c6 * exp_(S.g6 - a6) * m6i;
        const R e8 = S.c8 * exp_(S.g8 - a8) * m8i;
        const R e10 = S.c10 * exp_(S.g10 - a10) * m10i;
        const R fsum = e6 + e8 + e10;
        const R dfdr = e6 * ((a6 - R(6)) * ri) + e8 * ((a8 - R(8)) * ri) + e10 * ((a10 - R(10)) * ri);
        const bool lv = v >= 3;
        const R bv = betap<R>(p, v);
        R pref, xc;
        if (!lu && !lv) { pref = -bu * bv; xc = S.xd_c1; }
        else if (lu && lv) { pref = -nlp * nlp * R(0.25); xc = nlp * nlp * R(0.25) * S.xd_c2; }
        else { pref = -S.delta * R(0.5); xc = nlp * R(0.5) * S.xd_c3; }
        const R K = bu * bv * cfi * cfj;
        const R ex = xc * K * exp_(-mulc(r, T.xd_k[ku][kv]));
        ed += pref * fsum;
        ex_sum += ex;
        const R dEdr = pref * dfdr - cval<R>(T.xd_k[ku][kv]) * ex;
        gu = gu + (dEdr * ri) * dv;
    }
    a.Ed.add(R(0.5) * ed);
    a.Ex.add(R(0.5) * ex_sum);
    addG(a, u, gu);
    if (VIR) vir_add(a.W, gu, dO, R(-0.5));
}

// ---- kernel ------------------------------------------------------------------

// PART 0: exchange-repulsion items (BB, BL, LB, LL); PART 1: dispersion and
// exchange-dispersion items (D).  Two launches keep each kernel's code small.
// VIR: also the virial, in the translation-invariance form of the pair
// kernels (see vir_points_out): per item -1/2 (gradient on i's points) (x)
// dO_ij, plus sum_p G_p (x) off_p at the end.
// Resident blocks per SM: periodic 4 (repulsion) and 6 (dispersion), the
// registers those need; gas phase 5 (measured faster for cluster batches).
template <typename R, bool PER, int PART, bool VIR>
__global__ void __launch_bounds__(128, PER ? (PART == 0 ? 4 : 6) : 5) k_short(KParams p, DevState<R> d) {
    __shared__ ShortTables T;
    __shared__ int qbuf[4][SQ_WORDS];
    static_assert(SQ_D + SQ_CAPD <= SQ_WORDS && 15 * 33 * sizeof(R) <= SQ_WORDS * sizeof(int), "queue layout");
    static_assert(offsetof(KParams, xd_k) - offsetof(KParams, rep_k1) == offsetof(ShortTables, xd_k) &&
                      sizeof(ShortTables) == sizeof(KParams::Coef) * (9 * 4 + 27),
                  "coefficient tables are copied as one block");
    {
        const KParams::Coef *src = &p.rep_k1[0][0];
        KParams::Coef *dst = &T.rep_k1[0][0];
        for (int k = threadIdx.x; k < (int)(sizeof(ShortTables) / sizeof(KParams::Coef)); k += blockDim.x) {
            // rep_k1, rep_k2, disp_km, disp_gS, xd_k are consecutive in KParams and in ShortTables
            dst[k] = src[k];
        }
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *q = qbuf[w];
    const Scal<R> &S = sc<R>(p);
    // molecules i = 4 block + w, then strided by the grid (a persistent launch
    // with a capped grid leaves room for the kernels of the other streams)
    for (int i = blockIdx.x * 4 + w; i < p.M; i += gridDim.x * 4) {
        const R rc2 = S.rc2;
        ShortI<R> I;
        for (int k = 0; k < 3; ++k) I.P[k] = my_pt(d, i, k);
        I.P[3] = my_pt(d, i, 5);
        I.P[4] = my_pt(d, i, 6);
        {
            const R q0 = d.gmp[(i * NS) * GMP], q1 = d.gmp[(i * NS + 1) * GMP], q2 = d.gmp[(i * NS + 2) * GMP];
            I.A[0] = rep_atom(S.cs_o, S.cp_o, S.g_o, R(1) - q0 * S.inv_nval_o, 0);
            I.A[1] = rep_atom(S.cs_h, S.cp_h, S.g_h, R(1) - q1 * S.inv_nval_h, 1);
            I.A[2] = rep_atom(S.cs_h, S.cp_h, S.g_h, R(1) - q2 * S.inv_nval_h, 1);
            I.cf[0] = I.A[0].cf;
            I.cf[1] = I.A[1].cf;
            I.cf[2] = I.A[2].cf;
            I.cf[3] = I.A[0].cf;
            I.cf[4] = I.A[0].cf;
        }
        ShortAcc<R> acc;
        for (int k = 0; k < 5; ++k) acc.G[k] = mk(R(0), R(0), R(0));
    #pragma unroll
        for (int k = 0; k < 9; ++k) acc.W[k] = R(0);
        int h[5] = {0, 0, 0, 0, 0}, t[5] = {0, 0, 0, 0, 0};   // heads and tails: BB, BL, LB, LL, D
        const int nn = d.nnbr[i];
        for (int base = 0;; base += 32) {
            const bool flush = base >= nn;
            const int slot = base + lane;
            const bool live = slot < nn;
            int j = 0;
            V3<R> dO = mk(R(0), R(0), R(0));
            if (live) neighbour(d, i, slot, j, dO);
            // PART 0, stage 0: repulsion items; PART 1, stage 1: dispersion items
            const int s0 = PART == 0 ? 0 : 1, s1 = PART == 0 ? 1 : 2;
            for (int stage = s0; stage < s1; ++stage) {
                if (PART == 0) {
                    unsigned bb = 0, bl = 0, lb = 0, ll = 0;
                    if (live) {
                        const V3<R> Q1 = qpt(d, j, dO, 1), Q2 = qpt(d, j, dO, 2);
                        const V3<R> L1 = qpt(d, j, dO, 3), L2 = qpt(d, j, dO, 4);
                        const V3<R> mi1 = R(0.5) * (I.P[0] + I.P[1]), mi2 = R(0.5) * (I.P[0] + I.P[2]);
                        const V3<R> mj1 = R(0.5) * (dO + Q1), mj2 = R(0.5) * (dO + Q2);
                        auto in = [&](V3<R> x) { return !PER || dot(x, x) < rc2; };
                        bb = in(mi1 - mj1) | in(mi1 - mj2) << 1 | in(mi2 - mj1) << 2 | in(mi2 - mj2) << 3;
                        bl = in(mi1 - L1) | in(mi1 - L2) << 1 | in(mi2 - L1) << 2 | in(mi2 - L2) << 3;
                        lb = in(I.P[3] - mj1) | in(I.P[3] - mj2) << 1 | in(I.P[4] - mj1) << 2 | in(I.P[4] - mj2) << 3;
                        ll = in(I.P[3] - L1) | in(I.P[3] - L2) << 1 | in(I.P[4] - L1) << 2 | in(I.P[4] - L2) << 3;
                    }
                    const unsigned bits[4] = {bb, bl, lb, ll};
                    const int off[4] = {SQ_BB, SQ_BL, SQ_LB, SQ_LL};
    #pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        int n;
                        int pos = warp_excl_scan(__popc(bits[c]), lane, n);
    #pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if ((bits[c] >> k) & 1u) q[off[c] + (t[c] + pos++) % SQ_CAP] = slot * 32 + k;
                        t[c] += n;
                    }
                } else {
                    // one item per point u of i with at least one point v of j inside the cutoff
                    unsigned vm[5] = {0, 0, 0, 0, 0};
                    if (live) {
                        V3<R> Q[5];
    #pragma unroll
                        for (int v = 0; v < 5; ++v) Q[v] = qpt(d, j, dO, v);
    #pragma unroll
                        for (int u = 0; u < 5; ++u)
    #pragma unroll
                            for (int v = 0; v < 5; ++v) {
                                const V3<R> x = I.P[u] - Q[v];
                                if (!PER || dot(x, x) < rc2) vm[u] |= 1u << v;
                            }
                    }
                    int cnt = 0;
    #pragma unroll
                    for (int u = 0; u < 5; ++u) cnt += vm[u] != 0;
                    int n;
                    int pos = warp_excl_scan(cnt, lane, n);
    #pragma unroll
                    for (int u = 0; u < 5; ++u)
                        if (vm[u]) q[SQ_D + (t[4] + pos++) % SQ_CAPD] = (slot << 8) | (u << 5) | (int)vm[u];
                    t[4] += n;
                }
                __syncwarp();
                const bool last = flush && stage == s1 - 1;
                if (PART == 1) {
                    while (t[4] - h[4] >= 32 || (last && t[4] > h[4])) {
                        if (lane < t[4] - h[4]) item_du<R, VIR>(p, S, T, d, I, i, q[SQ_D + (h[4] + lane) % SQ_CAPD], acc);
                        h[4] += min(32, t[4] - h[4]);
                    }
                    __syncwarp();
                    continue;
                }
                while (t[0] - h[0] >= 32 || (last && t[0] > h[0])) {
                    if (lane < t[0] - h[0]) item_bb<R, VIR>(S, T, d, I, i, q[SQ_BB + (h[0] + lane) % SQ_CAP], acc);
                    h[0] += min(32, t[0] - h[0]);
                }
                while (t[1] - h[1] >= 32 || (last && t[1] > h[1])) {
                    if (lane < t[1] - h[1]) item_bl<R, VIR>(S, T, d, I, i, q[SQ_BL + (h[1] + lane) % SQ_CAP], acc);
                    h[1] += min(32, t[1] - h[1]);
                }
                while (t[2] - h[2] >= 32 || (last && t[2] > h[2])) {
                    if (lane < t[2] - h[2]) item_lb<R, VIR>(S, T, d, I, i, q[SQ_LB + (h[2] + lane) % SQ_CAP], acc);
                    h[2] += min(32, t[2] - h[2]);
                }
                while (t[3] - h[3] >= 32 || (last && t[3] > h[3])) {
                    if (lane < t[3] - h[3]) item_ll<R, VIR>(S, T, d, I, i, q[SQ_LL + (h[3] + lane) % SQ_CAP], acc);
                    h[3] += min(32, t[3] - h[3]);
                }
                __syncwarp();
            }
            if (flush) break;
        }
        // lane reduction; points 3, 4 are the lone pairs (point slots 5, 6)
        const R vals[15] = {acc.G[0].x, acc.G[0].y, acc.G[0].z, acc.G[1].x, acc.G[1].y, acc.G[1].z,
                            acc.G[2].x, acc.G[2].y, acc.G[2].z, acc.G[3].x, acc.G[3].y, acc.G[3].z,
                            acc.G[4].x, acc.G[4].y, acc.G[4].z};
        const R s = warp_transpose_sum<R, 15>(vals, reinterpret_cast<R *>(q), lane);
        const int pt = lane / 3;
        if (lane < 15) d.gpt[(i * NP + (pt < 3 ? pt : pt + 2)) * 3 + lane % 3] += double(s);
        if (VIR) vir_points_out(d, i, I.P, s, acc.W, reinterpret_cast<R *>(q), lane);
        if (PART == 0) {
            const double er_ = warp_sum_acc(acc.Erep);
            if (lane == 0) d.epart[i * NTERM + T_REP] += er_;
        } else {
            const double ed_ = warp_sum_acc(acc.Ed), ex_ = warp_sum_acc(acc.Ex);
            if (lane == 0) {
                d.epart[i * NTERM + T_DISP] += ed_;
                d.epart[i * NTERM + T_XDISP] += ex_;
            }
        }
    }
}

// max_blocks > 0 caps the grid (each block then walks several molecules per
// warp); max_per_sm > 0 caps the blocks resident per SM by reserving unused
// dynamic shared memory, which leaves registers on every SM for the kernels
// of the other streams.
template <typename R>
void launch_short(const KParams &p, DevState<R> &d, Launch L, int max_blocks, int max_per_sm) {
    unsigned nb = (p.M + 3) / 4;
    if (max_blocks > 0 && nb > (unsigned)max_blocks) nb = (unsigned)max_blocks;
    size_t sm = 0;
    if (max_per_sm > 0 && !p.vir) {
        auto k0 = p.periodic ? k_short<R, true, 0, false> : k_short<R, false, 0, false>;
        auto k1 = p.periodic ? k_short<R, true, 1, false> : k_short<R, false, 1, false>;
        int dev = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k0);
        // one byte more per block than a (max_per_sm + 1)-th block would leave room for
        const long long need = per_sm / (max_per_sm + 1) + 1 - (long long)fa.sharedSizeBytes;
        if (need > 0) {
            sm = (size_t)need;
            cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        }
    }
    k_short_pack<R><<<(p.M * 5 + 255) / 256, 256, 0, L.s>>>(p, d);
    count(L);
    if (p.vir) {
        if (p.periodic) {
            k_short<R, true, 0, true><<<nb, 128, sm, L.s>>>(p, d);
            k_short<R, true, 1, true><<<nb, 128, sm, L.s>>>(p, d);
        } else {
            k_short<R, false, 0, true><<<nb, 128, sm, L.s>>>(p, d);
            k_short<R, false, 1, true><<<nb, 128, sm, L.s>>>(p, d);
        }
    } else if (p.periodic) {
        k_short<R, true, 0, false><<<nb, 128, sm, L.s>>>(p, d);
        k_short<R, true, 1, false><<<nb, 128, sm, L.s>>>(p, d);
    } else {
        k_short<R, false, 0, false><<<nb, 128, sm, L.s>>>(p, d);
        k_short<R, false, 1, false><<<nb, 128, sm, L.s>>>(p, d);
    }
    count(L, 2);
}

template void launch_short<float>(const KParams &, DevState<float> &, Launch, int, int);
template void launch_short<double>(const KParams &, DevState<double> &, Launch, int, int);

}  // namespace sibfa
