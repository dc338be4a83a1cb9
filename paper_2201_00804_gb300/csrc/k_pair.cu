// Real-space pair kernels over the full molecular neighbour list.
//
// Every kernel walks the neighbours of one molecule i and accumulates only
// i's quantities (energy halves, gradients of i's points, multipole
// sensitivities of i's sites), so no two threads write the same output and
// no atomics are needed; the neighbour list is full, each molecule pair is
// visited from both sides.  Pair arithmetic runs in R (float in the mixed
// path, double in the FP64 path); per-lane partial sums are reduced across
// the warp in double.
#include "sibfa_internal.cuh"

namespace sibfa {

template <typename R>
__device__ inline void symadd(Sym<R> &a, const Sym<R> &b, R s) {
    a.xx += s * b.xx; a.yy += s * b.yy; a.zz += s * b.zz;
    a.xy += s * b.xy; a.xz += s * b.xz; a.yz += s * b.yz;
}

// ---------------------------------------------------------------------------
// Work queues.  A warp walks its molecule's neighbour list 32 entries at a
// time, tests each (neighbour, source site) pair against the cutoff and
// appends the pairs inside it to a per-warp ring queue in shared memory
// (source position relative to O_i, neighbour index and site).  Pairs are
// evaluated in rounds of 32 only while the queue holds a full round, so
// lanes stay busy whatever the cutoff rejects; the tail is flushed at the
// end.  Atom and midpoint sources go to separate queues because only atom
// sources carry a valence (penetration), which keeps every round uniform.
// ---------------------------------------------------------------------------
constexpr int QCAP_A = 128;   // >= 31 carried + 3 atom sites x 32 new entries
constexpr int QCAP_M = 96;    // >= 31 carried + 2 midpoints x 32 new entries

template <typename R, int CAP = QCAP_A + QCAP_M>
struct PairQueue {
    int js[CAP];   // j * 8 + s
    R rx[CAP], ry[CAP], rz[CAP];
    __device__ inline void put(int e, int j, int s, V3<R> r) {
        js[e] = j * 8 + s;
        rx[e] = r.x;
        ry[e] = r.y;
        rz[e] = r.z;
    }
    __device__ inline V3<R> at(int e) const { return mk(rx[e], ry[e], rz[e]); }
};

// ---------------------------------------------------------------------------
// Permanent electrostatics + penetration (Eq. 2), Thole-damped permanent
// field on the polarizable atoms, potential on the lone pairs.
// Warps 0..4: target site w of molecule i.  Warps 5, 6: target lone pair.
// ---------------------------------------------------------------------------
template <typename R>
struct PermAcc {
    Acc<R> Ue, Up, Vl;
    V3<R> gr, gm, ef;
    Sym<R> gt;
    R W[9];   // virial (VIR kernels only)
};

// VIR: also accumulate the pair virial 1/2 g (x) x of the target's gradient g
// (both molecules of a pair see it, so each adds half); the lone-pair
// potential's share is taken with the lambda charges in the force pass.
//
// Periodic systems: rv is the source position relative to O_i (O-O
// displacement plus the source's offset).  Gas phase: rv is the O-O
// displacement D = O_j - O_i itself and the pair displacement is formed as
// x = (target offset - source offset) - D.  The energy terms that involve a
// charge are taken as differences from reference points, because over a
// neutral molecule they cancel to the molecular interaction (site-pair
// terms of ~10 kcal/mol for a total of a few) and FP32 would keep only their
// rounding: with a = 1/|x|, b = 1/|y| for a reference vector y and
// d = |y|^2 - |x|^2 computed from the offsets without cancellation,
//   a - b = d a b / (|x| + |y|),  a^3 - b^3 = (a - b)(a^2 + ab + b^2),
//   a^5 - b^5 = (a - b)(a^4 + a^3 b + a^2 b^2 + a b^3 + b^4).
//   charge-charge:        y0 = -D (O_i - O_j):  q_t q_s (a - b0);
//   target charge in the source dipole/quadrupole potential, y1 = O_i - x_s:
//     q_t [mu_s.o_t a^3 + mu_s.y1 (a^3 - b1^3) + (o_t Th_s o_t + 2 y1 Th_s o_t) a^5
//          + y1 Th_s y1 (a^5 - b1^5)]   (x = y1 + o_t);
//   source charge in the target dipole/quadrupole, y2 = x_t - O_j:
//     q_s [mu_t.o_s a^3 - mu_t.y2 (a^3 - b2^3) + (o_s Th_t o_s - 2 y2 Th_t o_s) a^5
//          + y2 Th_t y2 (a^5 - b2^5)]   (x = y2 - o_s).
// The remainders (the reference values times the molecule's total charge,
// zero for neutral molecules) are added once per molecule pair (Q_i Q_j / R),
// per target site and neighbour, and per source site on the O target's warp.
// For gas-phase clusters this brings the FP32 multipole energy some 30x
// closer to FP64 than summing the site-pair energies directly.
template <typename R, bool PER, bool ATOM_SRC, bool VIR>
__device__ __forceinline__ void perm_pair(const KParams &p, const DevState<R> &d, int w, bool is_lp, V3<R> ot,
                                          const Mp<R> &mt, R Nt_, R Qi, int js, V3<R> rv, size_t te,
                                          PermAcc<R> &A) {
    const Scal<R> &S = sc<R>(p);
    const R third = R(1) / R(3);
    const int j = js >> 3, s = js & 7;
    V3<R> x, sv, osrc;
    if (PER) {
        x = ot - rv;
    } else {
        const R *os = d.off + (j * NP + s) * 3;
        osrc = mk(__ldg(os), __ldg(os + 1), __ldg(os + 2));
        sv = ot - osrc;
        x = sv - rv;
    }
    const R r2 = dot(x, x);
    const R rinv = rsqrt_(r2);
    const R r = r2 * rinv;
    const Mp<R> ms = load_mp_g(d.gmp + (j * NS + s) * GMP);
    R g[6];
    if (PER) g_erfc<R, 5>(r, rinv, S.alpha, g);
    else g_bare<R, 5>(rinv, g);
    if (is_lp) {
        FieldTerms<R> f;
        source_field<R, 1>(ms, x, g, f);
        A.Vl.add(f.phi);
        A.gr = A.gr + f.d1;
        return;
    }
    FieldTerms<R> f;
    source_field<R, 3>(ms, x, g, f);
    R U;
    if (PER) {
        U = mt.q * f.phi + dot(mt.mu, f.d1) + third * symdd(mt.th, f.d2);
    } else {
        const R a = rinv, a3 = a * a * a, a5 = a3 * a * a;
        // charge-charge, reference -D
        const R RR = dot(rv, rv), b0 = rsqrt_(RR);
        U = mt.q * ms.q * ((R(2) * dot(sv, rv) - dot(sv, sv)) * a * b0 / (r + RR * b0));
        // target charge, reference O_i - x_s
        const V3<R> y1 = R(-1) * (rv + osrc);
        const R y1y1 = dot(y1, y1), b1 = rsqrt_(y1y1);
        R B3, B5;
        ref_diff35(-(R(2) * dot(y1, ot) + dot(ot, ot)), a, b1, r, y1y1 * b1, B3, B5);
        const V3<R> Tso = symv(ms.th, ot), Tsy = symv(ms.th, y1);
        const R mu_y1 = dot(ms.mu, y1), y1Ty1 = dot(y1, Tsy);
        U += mt.q * (dot(ms.mu, ot) * a3 + mu_y1 * B3 + (dot(ot, Tso) + R(2) * dot(y1, Tso)) * a5 + y1Ty1 * B5);
        if (w == 0) {   // sum over the target sites of q_t times the reference value: Q_i phi_s(y1)
            const R b13 = b1 * b1 * b1;
            U += Qi * (mu_y1 * b13 + y1Ty1 * b13 * b1 * b1);
        }
        // source charge, reference x_t - O_j
        const V3<R> y2 = ot - rv;
        const R y2y2 = dot(y2, y2), b2 = rsqrt_(y2y2);
        R C3, C5;
        ref_diff35(R(2) * dot(y2, osrc) - dot(osrc, osrc), a, b2, r, y2y2 * b2, C3, C5);
        const V3<R> Tto = symv(mt.th, osrc), Tty = symv(mt.th, y2);
        U += ms.q * (dot(mt.mu, osrc) * a3 - dot(mt.mu, y2) * C3 + (dot(osrc, Tto) - R(2) * dot(y2, Tto)) * a5 +
                     dot(y2, Tty) * C5);
        // target dipole and quadrupole in the source dipole and quadrupole field
        U += dot(mt.mu, f.d1_mp) + third * symdd(mt.th, f.d2_mp);
    }
    A.Ue.add(R(0.5) * U);
    const V3<R> gel = target_grad(mt, ms, x, g, f);
    A.gr = A.gr + gel;
    V3<R> gv = gel;   // this pair's gradient (virial)
    A.gm = A.gm + f.d1;
    symadd(A.gt, f.d2, third);
    // ---- penetration: charge-charge*, charge-dipole*, charge-quadrupole*
    // Kernels exp(-b r)/r of the source (es) and target (et) valence; the
    // product kernel exp(-(b_s + b_t) r)/r of the N_t N_s term is es0 et0 r.
    if (ATOM_SRC || Nt_ != R(0)) {
        R pen = R(0), gq = R(0);
        R et[4];
        const R xt_b = mulc(r, p.pen_b[w]);   // b_t r
        if (Nt_ != R(0)) {
            g_exp_x<R, 3>(xt_b, rinv, et);
            const R c2 = ms.q * Nt_;            // q_s N_t exp(-b_t r)/r
            pen += c2 * et[0];
            gq += c2 * et[1];
        }
        if (ATOM_SRC) {
            const R Ns = zsite<R>(p, s) - ms.q;
            const R xs_b = mulc(r, p.pen_b[s]);   // b_s r
            R es[4];
            g_exp_x<R, 3>(xs_b, rinv, es);
            const R c1 = mt.q * Ns;                // q_t N_s exp(-b_s r)/r
            pen += c1 * es[0];
            gq += c1 * es[1];
            if (Nt_ != R(0)) {                     // N_t N_s exp(-(b_t + b_s) r)/r
                const R c3 = Nt_ * Ns;
                const R ec = es[0] * et[0] * r;
                pen += c3 * ec;
                gq -= c3 * (xt_b + xs_b + R(1)) * ec * (rinv * rinv);
            }
            // valence of s in the dipole/quadrupole potential of t
            Mp<R> m0 = mt;
            m0.q = R(0);
            const V3<R> xs = -x;
            FieldTerms<R> f3;
            source_field<R, 1>(m0, xs, es, f3);
            pen += Ns * f3.phi;
            A.gr = A.gr - Ns * f3.d1;
            if (VIR) gv = gv - Ns * f3.d1;
            A.gm = A.gm + (-Ns * es[1]) * xs;
            const R c = Ns * third * es[2];
            A.gt.xx += c * xs.x * xs.x; A.gt.yy += c * xs.y * xs.y; A.gt.zz += c * xs.z * xs.z;
            A.gt.xy += c * xs.x * xs.y; A.gt.xz += c * xs.x * xs.z; A.gt.yz += c * xs.y * xs.z;
        }
        A.gr = A.gr + gq * x;
        if (VIR) gv = gv + gq * x;
        if (Nt_ != R(0)) {   // valence of t in the dipole/quadrupole potential of s
            Mp<R> m0 = ms;
            m0.q = R(0);
            FieldTerms<R> f2;
            source_field<R, 1>(m0, x, et, f2);
            pen += Nt_ * f2.phi;
            A.gr = A.gr + Nt_ * f2.d1;
            if (VIR) gv = gv + Nt_ * f2.d1;
        }
        A.Up.add(R(0.5) * pen);
    }
    if (VIR) vir_add(A.W, gv, x, R(0.5));
    // ---- Thole-damped permanent field on the polarizable atom (same base kernel g)
    if (w < 3) {
        R gtol[4];
        g_thole_on<R, 3>(r, rinv, ainv3<R>(p, w, s), S.thole, PER, g, gtol);
        FieldTerms<R> f4;
        source_field<R, 1>(ms, x, gtol, f4);
        A.ef = A.ef - f4.d1;
        if (ATOM_SRC) {   // the same atom pair in the polarization matrix T
            // the field of a dipole mu at x is g2 (mu.x) x + g1 mu = sgn(g2) (mu.y) y + g1 mu
            // with y = sqrt|g2| x: four values and the sign of g2 in the index's top bit
            const R sq = sqrt_(fabs(gtol[2]));
            d.tl_j[te] = (j * 3 + s) | (gtol[2] < R(0) ? int(0x80000000u) : 0);
            d.tl_x[te] = sq * x.x;
            d.tl_y[te] = sq * x.y;
            d.tl_z[te] = sq * x.z;
            d.tl_g1[te] = gtol[1];
        }
    }
}

// One block per molecule whose NW warps take the target points W0 ..
// W0 + NW - 1: the five sites (W0 = 0) and, in a second launch on another
// stream, the lone pairs (W0 = 5: potential and gradient).  POT: the atoms
// O, H1, H2 as potential-only targets (potential and gradient, the acceptor
// potentials of the original charge transfer).  Each warp stores
// its energies, so the blocks need no barrier; the virial variant sums the
// site warps' virials in a fixed order.
// Site blocks: 3 resident per SM in periodic systems, 4 in the gas phase
// (96 registers; measured faster there, slower with the Ewald kernels).
template <typename R, bool PER, bool VIR, int W0, int NW, bool POT = false>
__global__ void __launch_bounds__(32 * NW, NW == 5 ? (PER ? 3 : 4) : (NW == 3 ? 5 : 8))
    k_real_perm(KParams p, DevState<R> d) {
    __shared__ double s_w[VIR ? NW : 1][9];
    __shared__ PairQueue<R> qs[NW];
    static_assert(sizeof(PairQueue<R>) >= 15 * 33 * sizeof(R), "reduction buffer aliases the queue");
    const int i = blockIdx.x;
    const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = W0 + wq;   // target point
    constexpr bool is_lp = W0 >= NS || POT;   // potential-only targets
    PairQueue<R> &q = qs[wq];
    const V3<R> ot = my_pt(d, i, w);
    Mp<R> mt{};
    if (!is_lp) mt = load_mp(d.gmp + (i * NS + w) * GMP);
    const R Nt = (!is_lp) ? zsite<R>(p, w) - mt.q * R(w < 3) : R(0);
    const R Nt_ = (w < 3) ? Nt : R(0);
    const R rc2 = sc<R>(p).rc2;
    const size_t tbase = (size_t)(i * 3 + (w < 3 ? w : 0)) * p.tls;   // T-pair list of target atom w

    PermAcc<R> A;
    A.gr = mk(R(0), R(0), R(0));
    A.gm = A.gr;
    A.ef = A.gr;
    A.gt = Sym<R>{};
#pragma unroll
    for (int k = 0; k < 9; ++k) A.W[k] = R(0);
    int ha = 0, ta = 0, hm = 0, tm = 0;   // queue heads and tails (warp-uniform, monotone)
    // gas phase: charge of molecule i (remainders of the reference-difference
    // energy terms, see perm_pair)
    R Qi = R(0);
    if (!PER && !is_lp)
        for (int s = 0; s < NS; ++s) Qi += d.gmp[(i * NS + s) * GMP];
    const int nn = d.nnbr[i];
    for (int base = 0;; base += 32) {
        const bool flush = base >= nn;   // list exhausted: evaluate what is left in the queues
        const int slot = base + lane;
        unsigned bits = 0;
        int j = 0;
        V3<R> rs[NS];
        if (slot < nn) {
            j = d.nbr[i * MAXN + slot];
            const R *dp = d.ndo + ((size_t)i * MAXN + slot) * 3;
            const V3<R> dO = mk(dp[0], dp[1], dp[2]);
            const R *offj = d.off + j * NP * 3;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                rs[s] = dO + mk(__ldg(offj + s * 3), __ldg(offj + s * 3 + 1), __ldg(offj + s * 3 + 2));
                const V3<R> x = ot - rs[s];
                if (!PER || dot(x, x) < rc2) bits |= 1u << s;
                if (!PER) rs[s] = dO;   // queued: the O-O displacement (see perm_pair)
            }
            if (!PER && !is_lp) {
                R Qj = R(0);
                for (int s = 0; s < NS; ++s) Qj += d.gmp[(j * NS + s) * GMP];
                // Q_j times the reference value of the target's terms: the
                // charge-charge one (O target only) and the dipole/quadrupole ones
                const V3<R> y2 = ot - dO;
                const R b2 = rsqrt_(dot(y2, y2)), b23 = b2 * b2 * b2;
                R rem = -dot(mt.mu, y2) * b23 + dot(y2, symv(mt.th, y2)) * b23 * b2 * b2;
                if (w == 0) rem += Qi * rsqrt_(dot(dO, dO));
                A.Ue.add(R(0.5) * Qj * rem);
            }
        }
        int na, nm;
        int pa = warp_excl_scan(__popc(bits & 7u), lane, na);
        int pm = warp_excl_scan(__popc(bits >> 3), lane, nm);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (!((bits >> s) & 1u)) continue;
            int e;
            if (s < 3) e = (ta + pa++) % QCAP_A;
            else e = QCAP_A + (tm + pm++) % QCAP_M;
            q.js[e] = j * 8 + s;
            q.rx[e] = rs[s].x;
            q.ry[e] = rs[s].y;
            q.rz[e] = rs[s].z;
        }
        ta += na;
        tm += nm;
        __syncwarp();
        while (ta - ha >= 32 || (flush && ta > ha)) {
            if (lane < ta - ha) {
                const int e = (ha + lane) % QCAP_A;
                perm_pair<R, PER, true, VIR>(p, d, w, is_lp, ot, mt, Nt_, Qi, q.js[e], q.at(e), tbase + ha + lane,
                                             A);
            }
            ha += min(32, ta - ha);
        }
        while (tm - hm >= 32 || (flush && tm > hm)) {
            if (lane < tm - hm) {
                const int e = QCAP_A + (hm + lane) % QCAP_M;
                perm_pair<R, PER, false, VIR>(p, d, w, is_lp, ot, mt, Nt_, Qi, q.js[e], q.at(e), 0, A);
            }
            hm += min(32, tm - hm);
        }
        __syncwarp();
        if (flush) break;
    }

    if (!POT && w < 3 && lane == 0) d.tl_n[i * 3 + w] = ta;
    const double ke = p.ke;
    R *buf = reinterpret_cast<R *>(&q);
    if (POT) {
        const double v = warp_sum_acc(A.Vl);
        const R vals[3] = {A.gr.x, A.gr.y, A.gr.z};
        const R t = warp_transpose_sum<R, 3>(vals, buf, lane);
        if (lane < 3) d.dva[(i * 3 + w) * 3 + lane] += ke * double(t);
        if (lane == 0) d.va[i * 3 + w] += ke * v;
    } else if (is_lp) {
        const int l = w - NS;
        const double v = warp_sum_acc(A.Vl);
        const R vals[3] = {A.gr.x, A.gr.y, A.gr.z};
        const R t = warp_transpose_sum<R, 3>(vals, buf, lane);
        if (lane < 3) d.dvlp[(i * 2 + l) * 3 + lane] += ke * double(t);
        if (lane == 0) d.vlp[i * 2 + l] += ke * v;
    } else {
        const R vals[15] = {A.gr.x, A.gr.y, A.gr.z, A.gm.x, A.gm.y, A.gm.z, A.gt.xx, A.gt.yy, A.gt.zz,
                            A.gt.xy, A.gt.xz, A.gt.yz, A.ef.x, A.ef.y, A.ef.z};
        const R t = warp_transpose_sum<R, 15>(vals, buf, lane);
        // one destination per lane, so the FP64 update is a single warp instruction
        double *dst = nullptr;
        if (lane < 3) dst = d.gpt + (i * NP + w) * 3 + lane;
        else if (lane < 6) dst = d.gmu + (i * NS + w) * 3 + lane - 3;
        else if (lane < 12) dst = d.gth + (i * NS + w) * 6 + lane - 6;
        else if (lane < 15 && w < 3) dst = d.efield + i * 9 + w * 3 + lane - 12;
        if (dst) *dst += (lane < 12 ? ke : 1.0) * double(t);
        if (VIR) {
            const R wv = warp_transpose_sum<R, 9>(A.W, buf, lane);
            if (lane < 9) s_w[wq][lane] = double(wv);
        }
        // per-warp energies (summed over the five sites in a fixed order by k_pol_energy)
        const double e0 = warp_sum_acc(A.Ue), e1 = warp_sum_acc(A.Up);
        if (lane == 0) {
            d.epw[(i * NS + w) * 2] = ke * e0;
            d.epw[(i * NS + w) * 2 + 1] = ke * e1;
        }
    }
    if (VIR) {   // the site warps' virials in a fixed order
        __syncthreads();
        if (threadIdx.x < 9) {
            double v = 0;
            for (int k = 0; k < NW; ++k) v += s_w[k][threadIdx.x];
            d.vir[i * 9 + threadIdx.x] += ke * v;
        }
    }
}

template <typename R>
void launch_real_perm(const KParams &p, DevState<R> &d, Launch L) {
    if (p.vir) {
        if (p.periodic) k_real_perm<R, true, true, 0, NS><<<p.M, 32 * NS, 0, L.s>>>(p, d);
        else k_real_perm<R, false, true, 0, NS><<<p.M, 32 * NS, 0, L.s>>>(p, d);
        count(L);
        return;
    }
    // the five sites in one block: as two launches (atoms, midpoints) the
    // second launch's tail cost more than the uneven warps of one block
    if (p.periodic) k_real_perm<R, true, false, 0, NS><<<p.M, 32 * NS, 0, L.s>>>(p, d);
    else k_real_perm<R, false, false, 0, NS><<<p.M, 32 * NS, 0, L.s>>>(p, d);
    count(L);
}

// potential and field of the permanent multipoles at the lone pairs (real
// space); with the original charge transfer also at the atoms O, H1, H2
template <typename R>
void launch_lp_potential(const KParams &p, DevState<R> &d, Launch L) {
    if (p.periodic) k_real_perm<R, true, false, NS, 2><<<p.M, 64, 0, L.s>>>(p, d);
    else k_real_perm<R, false, false, NS, 2><<<p.M, 64, 0, L.s>>>(p, d);
    count(L);
    if (p.ct_orig) {
        if (p.periodic) k_real_perm<R, true, false, 0, 3, true><<<p.M, 96, 0, L.s>>>(p, d);
        else k_real_perm<R, false, false, 0, 3, true><<<p.M, 96, 0, L.s>>>(p, d);
        count(L);
    }
}

// ---------------------------------------------------------------------------
// Reduced charge transfer (Eqs. 13-16).  Donors: lone pairs; acceptors: O-H
// bonds of other molecules with carrier-O distance below rc.
// ---------------------------------------------------------------------------
template <typename R>
struct CtOut {
    R E, dV, dVi1, dVi2, dsh;
    V3<R> gc, glp, ga1, ga2;
};

// Vi1, Vi2: the acceptor atoms' potentials in e1, e2 (V_int; the original
// form adds V*); shift: subtracted from the denominator (the original form's
// V(a1)); dsh = dE/dshift.
template <typename R>
__device__ inline CtOut<R> ct_pair(const KParams &p, V3<R> c, V3<R> lp, V3<R> a1, V3<R> a2, R V, R Vi1, R Vi2,
                                   int *flags, R shift = R(0)) {
    CtOut<R> o;
    const Scal<R> &S = sc<R>(p);
    const R cs = S.cs_lp, cp = S.cp_lp, t = S.ct_t, mm = S.ct_m, n = S.nlp;
    const V3<R> v1 = a1 - c, v2 = a2 - c, u = lp - c;
    const R q1 = dot(v1, v1), q2 = dot(v2, v2);
    const R ir1 = rsqrt_(q1), ir2 = rsqrt_(q2), r1 = q1 * ir1, r2 = q2 * ir2;
    V3<R> du1, dv1, du2, dv2;
    const R ca = cosv(u, v1, du1, dv1);
    const R cb = cosv(u, v2, du2, dv2);
    const R E1 = exp_(-mulc(r1, p.ct_k1)), E2 = exp_(-mulc(r2, p.ct_k2));
    const R ek1 = cval<R>(p.ct_k1), ek2 = cval<R>(p.ct_k2);   // eta / (2 sqrt(rv rv))
    const R K1 = cs * t + cp * mm * ca, K2 = cs * t + cp * mm * cb;
    const R e1 = E1 * (Vi1 - V) * K1, e2 = E2 * (Vi2 - V) * K2;
    const R D = e1 - e2;
    const R dE = S.ct_ae + V - S.ct_ah - shift;
    if (!(dE > R(0))) atomicOr(flags, F_CTDEN);
    const R idE = rcp_(dE);
    o.E = -n * D * D * idE;
    const R gD = R(-2) * n * D * idE;
    o.dV = gD * (-E1 * K1 + E2 * K2) + n * D * D * idE * idE;
    o.dVi1 = gD * E1 * K1;
    o.dVi2 = -gD * E2 * K2;
    o.dsh = -n * D * D * idE * idE;
    const R dr1 = gD * (-ek1 * e1), dr2 = gD * (ek2 * e2);
    const R dca = gD * E1 * (Vi1 - V) * cp * mm, dcb = -gD * E2 * (Vi2 - V) * cp * mm;
    const V3<R> n1 = ir1 * v1, n2 = ir2 * v2;
    o.glp = dca * du1 + dcb * du2;
    o.ga1 = dr1 * n1 + dca * dv1;
    o.ga2 = dr2 * n2 + dcb * dv2;
    o.gc = R(-1) * (o.glp + o.ga1 + o.ga2);
    return o;
}

// Bare potential (times ke) of the five multipole sites of molecule m at a
// point y given relative to m's O: the donor's part of an acceptor atom's
// potential in the original charge transfer.
template <typename R>
__device__ inline R mol_phi(const KParams &p, const DevState<R> &d, int m, V3<R> y) {
    R phi = R(0);
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
        const Mp<R> M = load_mp_g(d.gmp + (m * NS + s) * GMP);
        const V3<R> x = y - my_pt(d, m, s);
        R g[3];
        g_bare<R, 2>(rsqrt_(dot(x, x)), g);
        FieldTerms<R> f;
        source_field<R, 0>(M, x, g, f);
        phi += f.phi;
    }
    return R(p.ke) * phi;
}

// Working-precision per-molecule inputs of the charge transfer, so the pair
// loop reads no FP64: the lone-pair potentials (real space + reciprocal
// chain), V_int of O, H1, H2 and, for the original form, V(a) of O, H1, H2.
constexpr int CT_IN = 8;
template <typename R>
__global__ void k_ct_prep(int M, int orig, DevState<R> d) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    R *o = d.ctin + m * CT_IN;
    o[0] = R(d.vlp[m * 2] + d.vlp_r[m * 2]);
    o[1] = R(d.vlp[m * 2 + 1] + d.vlp_r[m * 2 + 1]);
    for (int a = 0; a < 3; ++a) {
        o[2 + a] = R(d.vint[m * 3 + a]);
        o[5 + a] = orig ? R(d.va[m * 3 + a] + d.va_r[m * 3 + a]) : R(0);
    }
}

// VIR: the virial of the pair terms by translation invariance: with X_p =
// O_i + off_p, sum over a molecule pair of g_p (x) X_p = sum_{p of i} g_p (x)
// off_p + sum_{p of j} g_p (x) off_p - G_{i<-j} (x) dO_ij, where G_{i<-j} is
// the total gradient on i's points and dO_ij = O_j - O_i; each side adds
// its own offsets term and half of the last one.
// One warp per molecule i.  The neighbour list is read 32 slots at a time;
// the slots inside the cutoff (carrier-carrier distance) are queued in
// shared memory and taken in full 32-lane rounds, each lane one molecule
// pair with its 8 donor-acceptor items (i donating to j and j to i).
template <typename R, bool PER, bool VIR>
__global__ void __launch_bounds__(128) k_ct(KParams p, DevState<R> d) {
    __shared__ R red[4][23 * 33];
    __shared__ int sq[4][64];
    const int wq = threadIdx.x >> 5;
    const int i = blockIdx.x * 4 + wq;
    const int lane = threadIdx.x & 31;
    if (i >= p.M) return;
    const R rc2 = sc<R>(p).rc2;
    V3<R> P[5];
    for (int k = 0; k < 3; ++k) P[k] = my_pt(d, i, k);
    P[3] = my_pt(d, i, 5);
    P[4] = my_pt(d, i, 6);
    const R *in_i = d.ctin + i * CT_IN;
    const R Vi[2] = {in_i[0], in_i[1]};
    const R Vint_i[3] = {in_i[2], in_i[3], in_i[4]};
    V3<R> G[5];
    for (int k = 0; k < 5; ++k) G[k] = mk(R(0), R(0), R(0));
    R lam[2] = {R(0), R(0)}, kap[3] = {R(0), R(0), R(0)};
    // original form: the acceptor potentials V(a) of i's atoms and dE/dV(a)
    const bool orig = p.ct_orig != 0;
    const R Va_i[3] = {in_i[5], in_i[6], in_i[7]};
    R lama[3] = {R(0), R(0), R(0)};
    R W[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = R(0);
    Acc<R> Ect;
    auto pair = [&](int slot) {
        const int j = d.nbr[i * MAXN + slot];
        const R *dp_ = d.ndo + ((size_t)i * MAXN + slot) * 3;
        const V3<R> dO = mk(dp_[0], dp_[1], dp_[2]);
        V3<R> Q[5];
        Q[0] = dO;
        Q[1] = dO + my_pt(d, j, 1);
        Q[2] = dO + my_pt(d, j, 2);
        Q[3] = dO + my_pt(d, j, 5);
        Q[4] = dO + my_pt(d, j, 6);
        const R *in_j = d.ctin + j * CT_IN;
        const R Vj[2] = {in_j[0], in_j[1]};
        // original form: W = V_int + V* in e1, e2 and V(a1) in the denominator,
        // V*(a) = V(a) minus the donor molecule's bare potential at a
        R Wj[3] = {in_j[2], in_j[3], in_j[4]}, Wi[3] = {Vint_i[0], Vint_i[1], Vint_i[2]};
        R sh_j = R(0), sh_i = R(0);
        R cd[3] = {R(0), R(0), R(0)}, ca[3] = {R(0), R(0), R(0)};
        if (orig) {
            for (int a = 0; a < 3; ++a) {
                Wj[a] += in_j[5 + a] - mol_phi(p, d, i, Q[a]);      // i's sites at j's atom a
                Wi[a] += Va_i[a] - mol_phi(p, d, j, P[a] - dO);      // j's sites at i's atom a
            }
            sh_j = in_j[5];
            sh_i = Va_i[0];
        }
        V3<R> Gj = mk(R(0), R(0), R(0));   // gradient on i's points from j (virial)
        for (int l = 0; l < 2; ++l)
            for (int k = 1; k <= 2; ++k) {
                // i donor (lone pair l of i), j acceptor (bond O-H_k of j)
                CtOut<R> o = ct_pair(p, P[0], P[3 + l], Q[0], Q[k], Vi[l], Wj[0], Wj[k], d.flags, sh_j);
                Ect.add(R(0.5) * o.E);
                G[0] = G[0] + o.gc;
                G[3 + l] = G[3 + l] + o.glp;
                lam[l] += o.dV;
                cd[0] += o.dVi1;
                cd[k] += o.dVi2;
                // j donor (lone pair l of j), i acceptor (bond O-H_k of i)
                CtOut<R> q = ct_pair(p, Q[0], Q[3 + l], P[0], P[k], Vj[l], Wi[0], Wi[k], d.flags, sh_i);
                Ect.add(R(0.5) * q.E);
                G[0] = G[0] + q.ga1;
                G[k] = G[k] + q.ga2;
                kap[0] += q.dVi1;
                kap[k] += q.dVi2;
                ca[0] += q.dVi1;
                ca[k] += q.dVi2;
                lama[0] += q.dVi1 + q.dsh;
                lama[k] += q.dVi2;
                if (VIR) Gj = Gj + o.gc + o.glp + q.ga1 + q.ga2;
            }
        if (orig) {
            R *cv = d.cvs + ((size_t)i * MAXN + slot) * 6;
            for (int a = 0; a < 3; ++a) cv[a] = cd[a], cv[3 + a] = ca[a];
        }
        if (VIR) vir_add(W, Gj, dO, R(-0.5));
    };
    int *q = sq[wq];
    int cnt = 0, base = 0;   // queued slots and next list slot (warp-uniform)
    const int nn = d.nnbr[i];
    for (;;) {
        while (cnt < 32 && base < nn) {
            const int slot = base + lane;
            bool in = false;
            if (slot < nn) {
                in = true;
                if (PER) {
                    const R *dp_ = d.ndo + ((size_t)i * MAXN + slot) * 3;
                    const R x = dp_[0], y = dp_[1], z = dp_[2];
                    in = x * x + y * y + z * z < rc2;
                }
                if (!in && orig) {   // no transfer: zero sensitivities for k_ct_vstar
                    R *cv = d.cvs + ((size_t)i * MAXN + slot) * 6;
                    for (int k = 0; k < 6; ++k) cv[k] = R(0);
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, in);
            if (in) q[cnt + __popc(b & ((1u << lane) - 1u))] = slot;
            cnt += __popc(b);
            base += 32;
            __syncwarp();
        }
        if (cnt == 0) break;
        const int take = cnt < 32 ? cnt : 32;
        if (lane < take) pair(q[lane]);
        __syncwarp();
        if (lane < cnt - take) q[lane] = q[take + lane];
        cnt -= take;
        __syncwarp();
    }
    const R vals[23] = {G[0].x, G[0].y, G[0].z, G[1].x, G[1].y, G[1].z, G[2].x, G[2].y, G[2].z,
                        G[3].x, G[3].y, G[3].z, G[4].x, G[4].y, G[4].z, lam[0], lam[1], kap[0], kap[1], kap[2],
                        lama[0], lama[1], lama[2]};
    const R t = warp_transpose_sum<R, 23>(vals, red[wq], lane);
    const int pt = lane / 3;
    double *dst = nullptr;
    if (lane < 15) dst = d.gpt + (i * NP + (pt < 3 ? pt : pt + 2)) * 3 + lane % 3;
    else if (lane < 17) dst = d.lam + i * 2 + lane - 15;
    else if (lane < 20) dst = d.kap + i * 3 + lane - 17;
    else if (lane < 23 && orig) dst = d.lama + i * 3 + lane - 20;
    if (dst) *dst += double(t);
    if (VIR) vir_points_out(d, i, P, t, W, red[wq], lane);
    const double e = warp_sum_acc(Ect);
    if (lane == 0) d.epart[i * NTERM + T_CT] += e;
}

// Original charge transfer, the dependence through V*(a) = V(a) - phi_D(a)
// (phi_D: the donor molecule's bare potential at the acceptor atom a) and
// through V(a).  With c = dE/dV*(a) per neighbour slot (k_ct: 0-2 at the
// partner's atoms for i donating, 3-5 at i's atoms for the partner
// donating) the energy varies as -sum c phi_D(a).  Warps 0-4: site s of i as
// the donor's source, point charges -c at the partners' atoms acting on its
// multipole (gradient at the site and multipole sensitivities); warps 5-7:
// atom a of i as the acceptor, the gradient of -c phi_j at the atom, plus
// the atom's own share of dE/dV(a) times the gradient of V(a) (the partners'
// share, charges dE/dV(a) on the atoms in the potential of every site, is
// taken in the force pass).
template <typename R>
__global__ void __launch_bounds__(256) k_ct_vstar(KParams p, DevState<R> d) {
    __shared__ R red[8][12 * 33];
    const int i = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nn = d.nnbr[i];
    const R third = R(1) / R(3);
    V3<R> gr = mk(R(0), R(0), R(0)), gm = gr;
    Sym<R> gt{};
    if (w < NS) {
        const Mp<R> mt = load_mp(d.gmp + (i * NS + w) * GMP);
        const V3<R> ot = my_pt(d, i, w);
        for (int slot = lane; slot < nn; slot += 32) {
            const R *c = d.cvs + ((size_t)i * MAXN + slot) * 6;
            if (c[0] == R(0) && c[1] == R(0) && c[2] == R(0)) continue;
            const int j = d.nbr[i * MAXN + slot];
            const R *dp = d.ndo + ((size_t)i * MAXN + slot) * 3;
            const V3<R> dO = mk(dp[0], dp[1], dp[2]);
            for (int a = 0; a < 3; ++a) {
                Mp<R> ms{};
                ms.q = -c[a];
                const V3<R> x = ot - (dO + my_pt(d, j, a));
                R g[6];   // source_field to third derivatives reads g_0..g_5
                g_bare<R, 5>(rsqrt_(dot(x, x)), g);
                FieldTerms<R> f;
                source_field<R, 3>(ms, x, g, f);
                gr = gr + target_grad(mt, ms, x, g, f);
                gm = gm + f.d1;
                symadd(gt, f.d2, third);
            }
        }
    } else {
        const int a = w - NS;
        const V3<R> ot = my_pt(d, i, a);
        for (int slot = lane; slot < nn; slot += 32) {
            const R c = d.cvs[((size_t)i * MAXN + slot) * 6 + 3 + a];
            if (c == R(0)) continue;
            const int j = d.nbr[i * MAXN + slot];
            const R *dp = d.ndo + ((size_t)i * MAXN + slot) * 3;
            const V3<R> dO = mk(dp[0], dp[1], dp[2]);
            for (int s = 0; s < NS; ++s) {
                const Mp<R> ms = load_mp_g(d.gmp + (j * NS + s) * GMP);
                const V3<R> x = ot - (dO + my_pt(d, j, s));
                R g[4];
                g_bare<R, 3>(rsqrt_(dot(x, x)), g);
                FieldTerms<R> f;
                source_field<R, 1>(ms, x, g, f);
                gr = gr - c * f.d1;
            }
        }
    }
    const R vals[12] = {gr.x, gr.y, gr.z, gm.x, gm.y, gm.z, gt.xx, gt.yy, gt.zz, gt.xy, gt.xz, gt.yz};
    const R t = warp_transpose_sum<R, 12>(vals, red[w], lane);
    const double ke = p.ke;
    // warps w < 3 (sites O, H1, H2) and 5 + w (the same atoms) both add to
    // the atom's point gradient: atomically
    if (w < NS) {
        if (lane < 3) atomicAdd(d.gpt + (i * NP + w) * 3 + lane, ke * double(t));
        else if (lane < 6) d.gmu[(i * NS + w) * 3 + lane - 3] += ke * double(t);
        else if (lane < 12) d.gth[(i * NS + w) * 6 + lane - 6] += ke * double(t);
    } else if (lane < 3) {
        const int a = w - NS;
        const double gv = d.dva[(i * 3 + a) * 3 + lane] + d.dva_r[(i * 3 + a) * 3 + lane];
        atomicAdd(d.gpt + (i * NP + a) * 3 + lane, ke * double(t) + d.lama[i * 3 + a] * gv);
    }
}

template <typename R>
void launch_ct(const KParams &p, DevState<R> &d, Launch L) {
    k_ct_prep<R><<<(p.M + 127) / 128, 128, 0, L.s>>>(p.M, p.ct_orig, d);
    count(L);
    const unsigned nb = (p.M + 3) / 4;
    if (p.vir) {
        if (p.periodic) k_ct<R, true, true><<<nb, 128, 0, L.s>>>(p, d);
        else k_ct<R, false, true><<<nb, 128, 0, L.s>>>(p, d);
    } else {
        if (p.periodic) k_ct<R, true, false><<<nb, 128, 0, L.s>>>(p, d);
        else k_ct<R, false, false><<<nb, 128, 0, L.s>>>(p, d);
    }
    count(L);
    if (p.ct_orig) {
        k_ct_vstar<R><<<p.M, 256, 0, L.s>>>(p, d);
        count(L);
    }
}

// ---------------------------------------------------------------------------
// Polarization matrix-vector product, real-space part: field at each
// polarizable atom from the dipoles vecR of the atoms of other molecules
// within rc (Thole-damped, Ewald-screened in periodic systems), streamed from
// the pair list that the permanent pass recorded.  out += field.  One warp
// per polarizable atom; each lane keeps four entries in flight.
// ---------------------------------------------------------------------------
constexpr int TW = 8;   // warps per block

// entry: partner atom index (the sign of g2 in its top bit), y = sqrt|g2| x, g1
template <typename R>
__device__ inline void tmu_entry(const DevState<R> &d, size_t k, int jraw, V3<R> &ef) {
    const R *mv = d.vecR + (jraw & 0x7fffffff) * 3;
    const V3<R> mu = mk(mv[0], mv[1], mv[2]);
    const V3<R> y = mk(d.tl_x[k], d.tl_y[k], d.tl_z[k]);
    const R my = dot(mu, y);
    ef = ef + (jraw < 0 ? -my : my) * y + d.tl_g1[k] * mu;
}

template <typename R>
__global__ void __launch_bounds__(32 * TW) k_real_tmu(int M, int tls, DevState<R> d, double *out) {
    __shared__ R red[TW][3 * 33];
    if (d.flags[1]) return;   // solver already converged
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * TW + w;
    if (t >= M * 3) return;
    const int n = d.tl_n[t];
    const size_t base = (size_t)t * tls;
    V3<R> ef = mk(R(0), R(0), R(0));
    int e = lane;
    for (; e + 96 < n; e += 128) {
        int jb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jb[u] = d.tl_j[base + e + 32 * u];
#pragma unroll
        for (int u = 0; u < 4; ++u) tmu_entry(d, base + e + 32 * u, jb[u], ef);
    }
    for (; e < n; e += 32) tmu_entry(d, base + e, d.tl_j[base + e], ef);
    const R vals[3] = {ef.x, ef.y, ef.z};
    const R s = warp_transpose_sum<R, 3>(vals, red[w], lane);
    if (lane < 3) out[t * 3 + lane] += double(s);
}

template <typename R>
void launch_real_tmu(const KParams &p, DevState<R> &d, double *out, Launch L) {
    k_real_tmu<R><<<(p.M * 3 + TW - 1) / TW, 32 * TW, 0, L.s>>>(p.M, p.tls, d, out);
    count(L);
}

// ---------------------------------------------------------------------------
// Polarization forces, real-space part, at fixed induced dipoles mu and
// charge-transfer sensitivities lambda (point charges on the lone pairs):
//   target site t of i:  d/dr_t and multipole sensitivities of
//       sum_b U(M_t, mu_b)   (Thole-damped)     + sum_l U(M_t, lambda_l) (undamped)
//   target pol atom a of i (a = t < 3): d/dr_a of
//       sum_s U(mu_a, M_s) + sum_b U(mu_a, mu_b)  (Thole-damped)
// One warp per target site; work queues as in the permanent kernel with
// three classes: atom sources (induced dipole and, for a polarizable target,
// permanent multipole, sharing one Thole kernel), midpoint sources
// (permanent multipole, polarizable targets only) and lambda charges.
// ---------------------------------------------------------------------------
constexpr int PQ_A = 128, PQ_M = 96, PQ_L = 96;

template <typename R>
struct PfAcc {
    V3<R> gr, gm;
    Sym<R> gt;
    R W[9];   // virial (VIR kernels only)
};

// VIR: also accumulate the pair virial g (x) x of the target's gradient g:
// half of it for dipole and multipole sources (the partner adds the other
// half), all of it for lambda charges (whose lone-pair side adds none).
template <typename R, bool PER, int KIND, bool VIR>   // KIND 0: atom source, 1: midpoint source, 2: lambda charge
__device__ __forceinline__ void polf_pair(const KParams &p, const DevState<R> &d, int w, V3<R> ot, const Mp<R> &mt,
                                          V3<R> mui, int js, V3<R> rs, PfAcc<R> &A) {
    const Scal<R> &S = sc<R>(p);
    const R third = R(1) / R(3);
    const int j = js >> 3, s = js & 7;
    const V3<R> x = ot - rs;
    const R r2 = dot(x, x);
    const R rinv = rsqrt_(r2), r = r2 * rinv;
    if (KIND == 2) {
        R g[6];
        if (PER) g_erfc<R, 5>(r, rinv, S.alpha, g);
        else g_bare<R, 5>(rinv, g);
        Mp<R> ms{};
        ms.q = d.lamR[j * 2 + s];
        FieldTerms<R> f;
        source_field<R, 3>(ms, x, g, f);
        const V3<R> gl = target_grad(mt, ms, x, g, f);
        A.gr = A.gr + gl;
        A.gm = A.gm + f.d1;
        symadd(A.gt, f.d2, third);
        if (VIR) vir_add(A.W, gl, x, R(1));
        return;
    }
    V3<R> gv = mk(R(0), R(0), R(0));   // this pair's gradient (virial)
    R gb[5], g[6];
    if (PER) g_erfc<R, 4>(r, rinv, S.alpha, gb);
    else g_bare<R, 4>(rinv, gb);
    g_thole_on<R, 4>(r, rinv, ainv3<R>(p, w, s), S.thole, PER, gb, g);
    g[5] = R(0);
    if (KIND == 0) {   // induced dipole of atom s of j at target site w
        Mp<R> ms{};
        const R *mj = d.muR + j * 9 + s * 3;
        ms.mu = mk(mj[0], mj[1], mj[2]);
        FieldTerms<R> f;
        source_field<R, 3>(ms, x, g, f);
        const V3<R> gm = target_grad(mt, ms, x, g, f);
        A.gr = A.gr + gm;
        A.gm = A.gm + f.d1;
        symadd(A.gt, f.d2, third);
        if (p.ct_orig) {   // original charge transfer: dE/dV(a) as a charge on atom s of j, undamped
            Mp<R> ml{};
            ml.q = d.lamaR[j * 3 + s];
            const R gl[6] = {gb[0], gb[1], gb[2], gb[3], gb[4], R(0)};
            FieldTerms<R> fl;
            source_field<R, 3>(ml, x, gl, fl);
            A.gr = A.gr + target_grad(mt, ml, x, gl, fl);
            A.gm = A.gm + fl.d1;
            symadd(A.gt, fl.d2, third);
        }
        if (VIR) gv = gm;
        // induced-induced, d/dr_a of mu_a . grad phi_b: for w < 3 the site
        // damping polarizability is the atom's, so f is the atom-atom field
        if (w < 3) {
            const V3<R> gi = symv(f.d2, mui);
            A.gr = A.gr + gi;
            if (VIR) gv = gv + gi;
        }
    }
    if (w < 3) {       // permanent multipoles of site s of j at polarizable atom w
        const Mp<R> ms = load_mp_g(d.gmp + (j * NS + s) * GMP);
        FieldTerms<R> f;
        source_field<R, 2>(ms, x, g, f);
        const V3<R> gp = symv(f.d2, mui);
        A.gr = A.gr + gp;
        if (VIR) gv = gv + gp;
    }
    if (VIR) vir_add(A.W, gv, x, R(0.5));
}

// Target sites W0 .. W0 + NW - 1 of one molecule per block: the atoms and
// the midpoints in two launches (the virial variant: all five in one block).
// The gas-phase launches keep more blocks resident (fewer registers), which
// measured faster there.
template <typename R, bool PER, bool VIR, int W0, int NW>
__global__ void __launch_bounds__(32 * NW, NW == 5 ? 3 : (NW == 3 ? (PER ? 5 : 6) : (PER ? 8 : 10))) k_real_polforce(KParams p,
                                                                                          DevState<R> d) {
    __shared__ PairQueue<R, PQ_A + PQ_M + PQ_L> qs[NW];
    static_assert(sizeof(PairQueue<R, PQ_A + PQ_M + PQ_L>) >= 12 * 33 * sizeof(R), "reduction buffer");
    const int i = blockIdx.x;
    const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = W0 + wq;   // target site
    PairQueue<R, PQ_A + PQ_M + PQ_L> &q = qs[wq];
    const V3<R> ot = my_pt(d, i, w);
    const Mp<R> mt = load_mp(d.gmp + (i * NS + w) * GMP);
    V3<R> mui = mk(R(0), R(0), R(0));
    if (w < 3) mui = mk(d.muR[i * 9 + w * 3], d.muR[i * 9 + w * 3 + 1], d.muR[i * 9 + w * 3 + 2]);
    const R rc2 = sc<R>(p).rc2;
    PfAcc<R> A;
    A.gr = mk(R(0), R(0), R(0));
    A.gm = A.gr;
    A.gt = Sym<R>{};
#pragma unroll
    for (int k = 0; k < 9; ++k) A.W[k] = R(0);
    int ha = 0, ta = 0, hm = 0, tm = 0, hl = 0, tl = 0;
    const int nn = d.nnbr[i];
    for (int base = 0;; base += 32) {
        const bool flush = base >= nn;
        const int slot = base + lane;
        unsigned bits = 0;   // bits 0-4 sites, 5-6 lone pairs
        int j = 0;
        V3<R> rs[NP];
        if (slot < nn) {
            j = d.nbr[i * MAXN + slot];
            const R *dp = d.ndo + ((size_t)i * MAXN + slot) * 3;
            const V3<R> dO = mk(dp[0], dp[1], dp[2]);
            const R *offj = d.off + j * NP * 3;
#pragma unroll
            for (int s = 0; s < NP; ++s) {
                rs[s] = dO + mk(__ldg(offj + s * 3), __ldg(offj + s * 3 + 1), __ldg(offj + s * 3 + 2));
                const V3<R> x = ot - rs[s];
                const bool in = !PER || dot(x, x) < rc2;
                const bool want = s < 3 || (s < NS ? w < 3 : d.lamR[j * 2 + s - NS] != R(0));
                if (in && want) bits |= 1u << s;
            }
        }
        int na, nm, nl;
        int pa = warp_excl_scan(__popc(bits & 7u), lane, na);
        int pm = warp_excl_scan(__popc((bits >> 3) & 3u), lane, nm);
        int pl = warp_excl_scan(__popc(bits >> 5), lane, nl);
#pragma unroll
        for (int s = 0; s < NP; ++s) {
            if (!((bits >> s) & 1u)) continue;
            if (s < 3) q.put((ta + pa++) % PQ_A, j, s, rs[s]);
            else if (s < NS) q.put(PQ_A + (tm + pm++) % PQ_M, j, s, rs[s]);
            else q.put(PQ_A + PQ_M + (tl + pl++) % PQ_L, j, s - NS, rs[s]);
        }
        ta += na;
        tm += nm;
        tl += nl;
        __syncwarp();
        while (ta - ha >= 32 || (flush && ta > ha)) {
            if (lane < ta - ha) {
                const int e = (ha + lane) % PQ_A;
                polf_pair<R, PER, 0, VIR>(p, d, w, ot, mt, mui, q.js[e], q.at(e), A);
            }
            ha += min(32, ta - ha);
        }
        while (tm - hm >= 32 || (flush && tm > hm)) {
            if (lane < tm - hm) {
                const int e = PQ_A + (hm + lane) % PQ_M;
                polf_pair<R, PER, 1, VIR>(p, d, w, ot, mt, mui, q.js[e], q.at(e), A);
            }
            hm += min(32, tm - hm);
        }
        while (tl - hl >= 32 || (flush && tl > hl)) {
            if (lane < tl - hl) {
                const int e = PQ_A + PQ_M + (hl + lane) % PQ_L;
                polf_pair<R, PER, 2, VIR>(p, d, w, ot, mt, mui, q.js[e], q.at(e), A);
            }
            hl += min(32, tl - hl);
        }
        __syncwarp();
        if (flush) break;
    }
    const double ke = p.ke;
    const R vals[12] = {A.gr.x, A.gr.y, A.gr.z, A.gm.x, A.gm.y, A.gm.z,
                        A.gt.xx, A.gt.yy, A.gt.zz, A.gt.xy, A.gt.xz, A.gt.yz};
    const R s = warp_transpose_sum<R, 12>(vals, reinterpret_cast<R *>(&q), lane);
    double *dst = nullptr;
    if (lane < 3) dst = d.gpt + (i * NP + w) * 3 + lane;
    else if (lane < 6) dst = d.gmu + (i * NS + w) * 3 + lane - 3;
    else if (lane < 12) dst = d.gth + (i * NS + w) * 6 + lane - 6;
    if (dst) *dst += ke * double(s);
    if (VIR) {   // the warps' virials summed in a fixed order
        __shared__ double s_w[NW][9];
        const R wv = warp_transpose_sum<R, 9>(A.W, reinterpret_cast<R *>(&q), lane);
        if (lane < 9) s_w[wq][lane] = double(wv);
        __syncthreads();
        if (threadIdx.x < 9) {
            double v = 0;
            for (int k = 0; k < NW; ++k) v += s_w[k][threadIdx.x];
            d.vir[i * 9 + threadIdx.x] += ke * v;
        }
    }
}

template <typename R>
void launch_real_polforce(const KParams &p, DevState<R> &d, Launch L) {
    if (p.vir) {
        if (p.periodic) k_real_polforce<R, true, true, 0, NS><<<p.M, 32 * NS, 0, L.s>>>(p, d);
        else k_real_polforce<R, false, true, 0, NS><<<p.M, 32 * NS, 0, L.s>>>(p, d);
        count(L);
        return;
    }
    if (p.periodic) {
        k_real_polforce<R, true, false, 0, 3><<<p.M, 96, 0, L.s>>>(p, d);
        k_real_polforce<R, true, false, 3, 2><<<p.M, 64, 0, L.s>>>(p, d);
    } else {
        k_real_polforce<R, false, false, 0, 3><<<p.M, 96, 0, L.s>>>(p, d);
        k_real_polforce<R, false, false, 3, 2><<<p.M, 64, 0, L.s>>>(p, d);
    }
    count(L, 2);
}

#define INST(R)                                                                                    \
    template void launch_real_perm<R>(const KParams &, DevState<R> &, Launch);                     \
    template void launch_lp_potential<R>(const KParams &, DevState<R> &, Launch);                  \
    template void launch_ct<R>(const KParams &, DevState<R> &, Launch);                            \
    template void launch_real_tmu<R>(const KParams &, DevState<R> &, double *, Launch);             \
    template void launch_real_polforce<R>(const KParams &, DevState<R> &, Launch);
INST(float)
INST(double)

}  // namespace sibfa
