// C ABI of the SIBFA library: context creation, one energy + force
// evaluation (the order of the method: sites -> neighbour list -> real-space
// pair terms -> SPME -> charge transfer -> polarization solve -> forces),
// the dipole-only solve and device-side velocity-Verlet steps.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <algorithm>
#include <cstdlib>

#include "sibfa_internal.cuh"
#include "pcg_guess.cuh"
#include "server_internal.h"

using namespace sibfa;

static thread_local std::string g_create_error = "no error";

struct sibfa_ctx {
    int M = 0;
    int capacity = 0;             // molecules the device arrays hold (M <= capacity)
    sibfa_run_opts opts{};
    KParams kp{};
    cudaStream_t s = nullptr;    // the library's own work stream (non-blocking)
    cudaStream_t s2 = nullptr;   // reciprocal-space chain, forked from s and joined back
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // short-range kernels (lowest priority), forked after the neighbour list
    // and joined before the chain rule: they fill the SMs that the permanent
    // pass's tail and the latency-bound polarization solve leave idle
    cudaStream_t s3 = nullptr;
    cudaEvent_t ev_fork3 = nullptr, ev_join3 = nullptr;
    bool short_pending = false;
    // Autotuner of the short-range schedule: resident blocks per SM (0 =
    // uncapped) and whether the short-range stream is joined before the
    // polarization solve (the solve then has the SMs to itself) or only
    // before the chain rule.  The first evaluations outside sibfa_minimize
    // after two warm-up ones
    // each run one candidate and are timed whole on the main stream (two per
    // candidate, the faster kept); then the fastest candidate is fixed.  The
    // choice changes only the scheduling, never the arithmetic.
    struct ShortTuner {
        bool on = true;
        int seen = 0;            // evaluations with forces seen
        int cand = 0;            // candidate being timed
        int reps = 0;
        int choice = -1;         // fixed candidate, -1 while tuning
        float tmin[5] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
        bool pending = false;    // events of the last timed evaluation not read yet
        cudaEvent_t e0 = nullptr, e1 = nullptr;
    } tune;
    // lone-pair potentials and charge transfer, forked after the neighbour
    // list and joined before the polarization energy: they run beside the
    // permanent pass and the polarization solve
    cudaStream_t s4 = nullptr;
    cudaEvent_t ev_fork4 = nullptr, ev_join4 = nullptr;
    bool ct_pending = false;
    cudaStream_t us = nullptr;   // the caller's stream (ordering only)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // polarization iterations as one CUDA graph with a device-side while loop
    cudaGraphExec_t pcg_exec = nullptr;
    int pcg_graph_state = 0;     // 0 untried, 1 in use, -1 unavailable (host loop)
    uint64_t pcg_iter_launches = 0;
    uint64_t pcg_graph_solves = 0;   // graph solves whose iteration count is not yet folded into launches
    bool capturing = false;
    int prec = SIBFA_PREC_MIXED;
    DevState<float> df{};
    DevState<double> dd{};
    cufftHandle r2c1 = 0, c2r1 = 0, r2c2 = 0, c2r2 = 0;
    bool have_fft = false;
    int ncell[3] = {0, 0, 0};
    int ncell_cap = 0;            // cells the cell-list arrays hold (set at create)
    double *d_forces = nullptr;   // M*9
    double *d_energy = nullptr;   // NTERM+1 energies; [16, 25) the virial
    double *d_vel = nullptr, *d_invm = nullptr;
    double *h_pin = nullptr;      // pinned staging, M*9*2 + 64 doubles
    double *h_scal = nullptr;     // pinned copy of the solver scalars of the last solve
    std::vector<void *> allocs;
    std::string err = "no error";
    uint64_t launches = 0;
    size_t dev_bytes = 0;         // device memory allocated by the context
    int last_iters = 0;
    double last_resid = 0;
    double e_tail = 0;            // dispersion beyond rc (homogeneous fluid), added to disp and the virial
    double *d_fprev = nullptr;    // Beeman: forces of the previous step (library-owned)
    bool have_mu = false;
    // converged dipoles of the last full evaluations (warm_start >= 2):
    // warm_start slots of capacity * 9 doubles, the newest at hist_head - 1
    double *mu_hist = nullptr;
    int hist_n = 0, hist_head = 0;
    bool md_forces_valid = false;
    bool minimizing = false;   // inside sibfa_minimize: its evaluations do not feed the tuner
    // optional per-phase timing with CUDA events on the context stream
    bool profiling = false;
    bool serial = false;   // profiling with every phase alone on the GPU (no stream overlap)
    struct Span {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> event_pool;
};

namespace {
struct Phase {
    sibfa_ctx *ctx;
    size_t idx = (size_t)-1;
    cudaStream_t st;
    Phase(sibfa_ctx *c, const char *name, cudaStream_t stream = nullptr) : ctx(c), st(stream ? stream : c->s) {
        if (!ctx->profiling || ctx->capturing) return;
        cudaEvent_t a, b;
        if (ctx->event_pool.size() >= 2) {
            a = ctx->event_pool.back();
            ctx->event_pool.pop_back();
            b = ctx->event_pool.back();
            ctx->event_pool.pop_back();
        } else {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
        }
        cudaEventRecord(a, st);
        ctx->spans.push_back({name, a, b});
        idx = ctx->spans.size() - 1;
    }
    ~Phase() {
        if (idx != (size_t)-1) cudaEventRecord(ctx->spans[idx].b, st);
    }
};
}  // namespace

namespace {

#define CK(call)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return SIBFA_E_CUDA;                                                    \
        }                                                                           \
    } while (0)

#define CKF(call)                                                                   \
    do {                                                                            \
        cufftResult r_ = (call);                                                    \
        if (r_ != CUFFT_SUCCESS) {                                                  \
            ctx->err = std::string(#call) + ": cufft error " + std::to_string(r_); \
            return SIBFA_E_CUDA;                                                    \
        }                                                                           \
    } while (0)

template <typename T>
sibfa_status dalloc(sibfa_ctx *ctx, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 16);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return SIBFA_E_OOM;
    }
    cudaMemsetAsync(q, 0, n * sizeof(T) + 16, ctx->s);   // ordered before any later work on the stream
    ctx->allocs.push_back(q);
    ctx->dev_bytes += n * sizeof(T) + 16;
    *p = (T *)q;
    return SIBFA_OK;
}

#define AL(ptr, n)                                          \
    do {                                                    \
        sibfa_status st_ = dalloc(ctx, &(ptr), (size_t)(n)); \
        if (st_ != SIBFA_OK) return st_;                    \
    } while (0)

template <typename R>
sibfa_status alloc_state(sibfa_ctx *ctx, DevState<R> &d) {
    const int M = ctx->M;
    d.M = M;
    AL(d.pos, M * 9);
    AL(d.mp_local, M * NS * NMP);
    AL(d.off, M * NP * 3);
    AL(d.gmp, M * NS * GMP);
    AL(d.vint, M * 3);
    AL(d.nbr, (size_t)M * MAXN);
    AL(d.ndo, (size_t)M * MAXN * 3);
    AL(d.ofw, (size_t)M * 3);
    AL(d.ufx, (size_t)M * 3);
    AL(d.sbase, (size_t)M * NP * 3);
    AL(d.sfrac, (size_t)M * NP * 3);
    AL(d.nnbr, M);
    // cluster arrays sized for up to one cluster per molecule, so that a
    // batch context can be regrouped in place (ctx_set_batch)
    AL(d.cl_of, M);
    AL(d.cl_start, M + 1);
    AL(d.cl_rr, M);
    AL(d.cl_energy, (size_t)M * (NTERM + 1));
    int ncell = std::max(1, ctx->ncell[0] * ctx->ncell[1] * ctx->ncell[2]);
    ctx->ncell_cap = ncell;
    AL(d.cell_of, M);
    AL(d.cell_start, ncell + 1);
    AL(d.cell_cursor, ncell);
    AL(d.cell_mol, M);
    AL(d.gpt, M * NP * 3);
    AL(d.gmu, M * NS * 3);
    AL(d.gth, M * NS * 6);
    AL(d.efield, M * 9);
    AL(d.d2rec, M * 18);
    AL(d.vlp, M * 2);
    AL(d.dvlp, M * 6);
    AL(d.lam, M * 2);
    AL(d.kap, M * 3);
    {
        // original charge transfer (allocated small when off)
        const bool cto = ctx->opts.ct_original != 0;
        AL(d.va, cto ? M * 3 : 1);
        AL(d.va_r, cto ? M * 3 : 1);
        AL(d.dva, cto ? M * 9 : 1);
        AL(d.dva_r, cto ? M * 9 : 1);
        AL(d.lama, cto ? M * 3 : 1);
        AL(d.lamaR, cto ? M * 3 : 1);
        AL(d.cvs, cto ? (size_t)M * MAXN * 6 : 1);
    }
    AL(d.ctin, M * 8);
    AL(d.spk, M * 20);
    AL(d.epart, M * NTERM);
    AL(d.epw, M * NS * 2);
    AL(d.vir, M * 9);
    AL(d.vir_r, M * 9);
    AL(d.vphi, M * 9);
    AL(d.gpt_r, M * NP * 3);
    AL(d.gpt_s, M * NP * 3);
    AL(d.gmu_r, M * NS * 3);
    AL(d.gth_r, M * NS * 6);
    AL(d.efield_r, M * 9);
    AL(d.vlp_r, M * 2);
    AL(d.dvlp_r, M * 6);
    AL(d.epart_r, M * NTERM);
    AL(d.eintra, M);
    AL(d.epartial, 128 * NTERM);
    AL(d.efp_r, M * 9);
    AL(d.mu, M * 9);
    AL(d.res, M * 9);
    AL(d.zv, M * 9);
    AL(d.pv, M * 9);
    AL(d.ap, M * 9);
    AL(d.efp, M * 9);
    AL(d.vecR, M * 9);
    AL(d.muR, M * 9);
    AL(d.lamR, M * 2);
    AL(d.tl_n, M * 3);
    const size_t nt = (size_t)M * 3 * ctx->kp.tls;
    AL(d.tl_j, nt);
    AL(d.tl_x, nt);
    AL(d.tl_y, nt);
    AL(d.tl_z, nt);
    AL(d.tl_g1, nt);
    AL(d.partial, 4 * ((M * 9 + 255) / 256) + 64);
    AL(d.scal, 32);
    AL(d.counter, 4);
    AL(d.flags, 4);
    AL(d.ext, 4);
    AL(d.oref, M * 3);
    AL(d.lst, 4);
    AL(d.lflag, 2);
    if (ctx->opts.periodic) {
        const size_t ng = (size_t)ctx->kp.K[0] * ctx->kp.K[1] * ctx->kp.K[2];
        const size_t nh = (size_t)ctx->kp.K[0] * ctx->kp.K[1] * (ctx->kp.K[2] / 2 + 1);
        AL(d.grid, 2 * ng);
        if (sizeof(R) == 4) {
            cufftComplex *c;
            AL(c, 2 * nh);
            d.cgrid = c;
        } else {
            cufftDoubleComplex *c;
            AL(c, 2 * nh);
            d.cgrid = c;
        }
        AL(d.infl, nh);
        AL(d.inflR, nh);
        AL(d.virk, (size_t)2 * VK_BLOCKS * 8);
        if (sizeof(R) == 4) {
            cufftComplex *c;
            AL(c, nh);
            d.qhat_p = c;
        } else {
            cufftDoubleComplex *c;
            AL(c, nh);
            d.qhat_p = c;
        }
    }
    return SIBFA_OK;
}

template <typename R>
void fill_scal(Scal<R> &s, const KParams &k) {
    s.rc2 = R(k.rc2); s.alpha = R(k.alpha); s.thole = R(k.thole);
    s.cs_o = R(k.cs_o); s.cp_o = R(k.cp_o); s.cs_h = R(k.cs_h); s.cp_h = R(k.cp_h);
    s.cs_lp = R(k.cs_lp); s.cp_lp = R(k.cp_lp); s.g_o = R(k.g_o); s.g_h = R(k.g_h);
    s.inv_nval_o = R(1.0 / k.nval_o); s.inv_nval_h = R(1.0 / k.nval_h);
    s.rep_f = R(k.rep_f); s.rep_c1 = R(k.rep_c1); s.rep_c2 = R(k.rep_c2); s.occ = R(k.occ); s.nlp = R(k.nlp);
    s.c6 = R(k.c6); s.c8 = R(k.c8); s.c10 = R(k.c10); s.g6 = R(k.g6); s.g8 = R(k.g8); s.g10 = R(k.g10);
    s.delta = R(k.delta); s.xd_c1 = R(k.xd_c1); s.xd_c2 = R(k.xd_c2); s.xd_c3 = R(k.xd_c3);
    s.ct_t = R(k.ct_t); s.ct_m = R(k.ct_m); s.ct_ae = R(k.ct_ae); s.ct_ah = R(k.ct_ah);
    for (int c = 0; c < 3; ++c) s.kl[c] = k.box[c] > 0 ? R((double)k.K[c] / k.box[c]) : R(0);
    s.ike = R(1.0 / k.ke);
}

// Dispersion beyond the cutoff for a homogeneous fluid (pair distribution 1
// past rc): 2 pi M (M-1) / V times, over the point types u, v of a water (O,
// H1, H2 and the two lone pairs), the integral from rc to infinity of r^2
// times the damped C6/C8/C10 pair function.  With t = 1/r each C_n term
// becomes pref C_n e^{g} k^n int_0^{1/rc} t^(n-4) e^{-g c t} dt
// (c = (rv_u + rv_v) alpha_disp, k = 2 sqrt(rv_u rv_v)), a smooth integrand
// taken by composite Simpson quadrature on 4096 intervals.  The
// exchange-dispersion, exponential in r, is negligible past the cutoff.
double disp_tail_energy(const sibfa_params &P, int M, double volume, double rc) {
    const double rv[5] = {P.rvdw_disp_o, P.rvdw_disp_h, P.rvdw_disp_h, P.rvdw_disp_lp, P.rvdw_disp_lp};
    const double beta[3] = {P.beta_o, P.beta_h, P.beta_h};
    const double Cn[3] = {P.c6, P.c8, P.c10}, gn[3] = {P.gamma6, P.gamma8, P.gamma10};
    const int order[3] = {6, 8, 10};
    const int NI = 4096;
    double total = 0;
    for (int u = 0; u < 5; ++u)
        for (int v = 0; v < 5; ++v) {
            const double pref = (u < 3 && v < 3) ? -beta[u] * beta[v]
                                                 : ((u >= 3 && v >= 3) ? -0.25 * P.n_lp * P.n_lp : -0.5 * P.disp_delta);
            const double c = (rv[u] + rv[v]) * P.disp_alpha, k = 2.0 * std::sqrt(rv[u] * rv[v]);
            for (int o = 0; o < 3; ++o) {
                const double h = (1.0 / rc) / NI, b = gn[o] * c;
                double sum = 0;
                for (int q = 0; q <= NI; ++q) {
                    const double t = q * h, w = (q == 0 || q == NI) ? 1.0 : (q % 2 ? 4.0 : 2.0);
                    sum += w * std::pow(t, order[o] - 4) * std::exp(-b * t);
                }
                total += pref * Cn[o] * std::exp(gn[o]) * std::pow(k, order[o]) * sum * h / 3.0;
            }
        }
    return 2.0 * M_PI * (double)M * (double)(M - 1) / volume * total;
}

void fill_params(KParams &k, const sibfa_params &P, const sibfa_run_opts &o, int M) {
    k.M = M;
    k.periodic = o.periodic;
    for (int i = 0; i < 3; ++i) {
        k.box[i] = o.box[i];
        k.ibox[i] = o.box[i] > 0 ? 1.0 / o.box[i] : 0.0;
    }
    k.rc = o.rc;
    k.rc2 = o.rc * o.rc;
    k.skin = o.periodic ? LIST_SKIN : 0.0;
    k.ct_orig = o.ct_original ? 1 : 0;
    k.alpha = o.ewald_alpha;
    for (int i = 0; i < 3; ++i) k.K[i] = o.grid[i];
    k.ke = P.ke;
    k.d_lp = P.d_lp;
    const double th = P.lp_half_deg * M_PI / 180.0;
    k.lp_cos = cos(th);
    k.lp_sin = sin(th);
    k.a_pol[0] = P.alpha_o;
    k.a_pol[1] = k.a_pol[2] = P.alpha_h;
    for (int a = 0; a < 3; ++a) k.a_pol_inv[a] = 1.0 / k.a_pol[a];
    k.a_damp[0] = P.alpha_o;
    k.a_damp[1] = k.a_damp[2] = P.alpha_h;
    k.a_damp[3] = k.a_damp[4] = P.alpha_m_damp;
    k.thole = P.thole;
    k.z[0] = P.z_o;
    k.z[1] = k.z[2] = P.z_h;
    k.z[3] = k.z[4] = 0.0;
    k.b[0] = P.b_o;
    k.b[1] = k.b[2] = P.b_h;
    k.b[3] = k.b[4] = 0.0;
    k.cs_o = P.cs_o; k.cp_o = P.cp_o; k.cs_h = P.cs_h; k.cp_h = P.cp_h; k.cs_lp = P.cs_lp; k.cp_lp = P.cp_lp;
    k.g_o = P.g_o; k.g_h = P.g_h; k.nval_o = P.nval_o; k.nval_h = P.nval_h;
    k.rv_rep_o = P.rvdw_rep_o; k.rv_rep_h = P.rvdw_rep_h; k.rv_rep_lp = P.rvdw_rep_lp;
    k.rep_a1 = P.rep_alpha; k.rep_a2 = P.rep_alpha2; k.rep_c1 = P.rep_c1; k.rep_c2 = P.rep_c2; k.rep_f = P.rep_f;
    k.occ = P.occ_bond; k.nlp = P.n_lp;
    k.rv_d[0] = P.rvdw_disp_o; k.rv_d[1] = k.rv_d[2] = P.rvdw_disp_h; k.rv_d[3] = k.rv_d[4] = P.rvdw_disp_lp;
    k.beta[0] = P.beta_o; k.beta[1] = k.beta[2] = P.beta_h; k.beta[3] = k.beta[4] = P.beta_o;
    k.disp_alpha = P.disp_alpha; k.c6 = P.c6; k.c8 = P.c8; k.c10 = P.c10;
    k.g6 = P.gamma6; k.g8 = P.gamma8; k.g10 = P.gamma10; k.delta = P.disp_delta;
    k.xd_c1 = P.xd_c1; k.xd_a1 = P.xd_a1; k.xd_c2 = P.xd_c2; k.xd_a2 = P.xd_a2; k.xd_c3 = P.xd_c3; k.xd_a3 = P.xd_a3;
    k.ct_eta = P.ct_eta; k.ct_t = P.ct_t; k.ct_m = P.ct_m; k.ct_ae = P.ct_ae; k.ct_ah = P.ct_ah;
    k.rv_ct_o = P.rvdw_ct_o; k.rv_ct_h = P.rvdw_ct_h;
    // pair-type coefficients in FP64 (kinds O, H, lone pair)
    auto coef = [](double v) {
        KParams::Coef c;
        c.d = v;
        c.hi = (float)v;
        c.lo = (float)(v - (double)c.hi);
        return c;
    };
    const double rvr[3] = {P.rvdw_rep_o, P.rvdw_rep_h, P.rvdw_rep_lp};
    const double rvd[3] = {P.rvdw_disp_o, P.rvdw_disp_h, P.rvdw_disp_lp};
    const double gam[3] = {P.gamma6, P.gamma8, P.gamma10};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double kr = 1.0 / (4.0 * sqrt(rvr[a] * rvr[b]));
            k.rep_k1[a][b] = coef(P.rep_alpha * kr);
            k.rep_k2[a][b] = coef(P.rep_alpha2 * kr);
            const double km = 1.0 / (2.0 * sqrt(rvd[a] * rvd[b]));
            k.disp_km[a][b] = coef(km);
            for (int n = 0; n < 3; ++n) k.disp_gS[n][a][b] = coef(gam[n] * (rvd[a] + rvd[b]) * P.disp_alpha);
            const bool la = a == 2, lb = b == 2;
            const double A = (!la && !lb) ? P.xd_a1 : ((la && lb) ? P.xd_a2 : P.xd_a3);
            k.xd_k[a][b] = coef(A * km);
        }
    k.ct_k1 = coef(P.ct_eta / (2.0 * sqrt(P.rvdw_ct_o * P.rvdw_ct_o)));
    k.ct_k2 = coef(P.ct_eta / (2.0 * sqrt(P.rvdw_ct_o * P.rvdw_ct_h)));
    for (int s = 0; s < 5; ++s) k.pen_b[s] = coef(k.b[s]);
    for (int i = 0; i < 3; ++i) k.fxs[i] = (float)(o.box[i] / 4294967296.0);
    fill_scal(k.sd, k);
    fill_scal(k.sf, k);
    for (int s = 0; s < 5; ++s) {
        k.zf[s] = (float)k.z[s];
        k.betaf[s] = (float)k.beta[s];
        for (int t = 0; t < 5; ++t) {
            k.ainv3[s][t] = 1.0 / sqrt(k.a_damp[s] * k.a_damp[t]);
            k.ainv3f[s][t] = (float)k.ainv3[s][t];
        }
    }
}

// Order the work stream after the caller's stream at entry, and the caller's
// stream after the work stream at exit.
sibfa_status enter(sibfa_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_in, ctx->us));
    CK(cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0));
    return SIBFA_OK;
}
sibfa_status leave(sibfa_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_out, ctx->s));
    CK(cudaStreamWaitEvent(ctx->us, ctx->ev_out, 0));
    return SIBFA_OK;
}

// Fork the reciprocal-space chain onto s2 after the work queued on s so
// far, and join it back into s.
sibfa_status fork_rec(sibfa_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_fork, ctx->s));
    CK(cudaStreamWaitEvent(ctx->s2, ctx->ev_fork, 0));
    return SIBFA_OK;
}
sibfa_status fork_short(sibfa_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_fork3, ctx->s));
    CK(cudaStreamWaitEvent(ctx->s3, ctx->ev_fork3, 0));
    return SIBFA_OK;
}
sibfa_status join_short(sibfa_ctx *ctx) {
    if (!ctx->short_pending) return SIBFA_OK;
    ctx->short_pending = false;
    CK(cudaEventRecord(ctx->ev_join3, ctx->s3));
    CK(cudaStreamWaitEvent(ctx->s, ctx->ev_join3, 0));
    return SIBFA_OK;
}
sibfa_status fork_ct(sibfa_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_fork4, ctx->s));
    CK(cudaStreamWaitEvent(ctx->s4, ctx->ev_fork4, 0));
    return SIBFA_OK;
}
sibfa_status join_ct(sibfa_ctx *ctx) {
    if (!ctx->ct_pending) return SIBFA_OK;
    ctx->ct_pending = false;
    CK(cudaEventRecord(ctx->ev_join4, ctx->s4));
    CK(cudaStreamWaitEvent(ctx->s, ctx->ev_join4, 0));
    return SIBFA_OK;
}

// Short-range schedule candidates: resident blocks per SM (0 = uncapped) and
// the join of the short-range stream before the solve.
struct ShortSched {
    int cap;
    bool join_before_solve;
};
constexpr int kNSched = 5;
constexpr ShortSched kSched[kNSched] = {{3, false}, {0, false}, {2, false}, {0, true}, {3, true}};
constexpr int kTuneWarm = 2, kTuneReps = 2;

ShortSched short_sched(const sibfa_ctx *ctx) {
    const auto &T = ctx->tune;
    if (!T.on) return {ctx->kp.periodic ? 3 : 0, false};
    return kSched[T.choice >= 0 ? T.choice : T.cand];
}
int short_cap(const sibfa_ctx *ctx) { return short_sched(ctx).cap; }

// Reads the last timed evaluation (waiting for it, only while tuning) and
// advances the candidate; after the last candidate, fixes the fastest.
void tune_account(sibfa_ctx *ctx) {
    auto &T = ctx->tune;
    if (!T.pending) return;
    T.pending = false;
    float ms = 0;
    if (cudaEventSynchronize(T.e1) != cudaSuccess || cudaEventElapsedTime(&ms, T.e0, T.e1) != cudaSuccess) {
        cudaGetLastError();
        T.on = false;   // no timing: keep the fixed default shape
        return;
    }
    if (T.seen++ < kTuneWarm) return;
    T.tmin[T.cand] = std::min(T.tmin[T.cand], ms);
    if (++T.reps < kTuneReps) return;
    T.reps = 0;
    if (++T.cand < kNSched) return;
    int best = 0;
    for (int c = 1; c < kNSched; ++c)
        if (T.tmin[c] < T.tmin[best]) best = c;
    T.choice = best;
}

sibfa_status join_rec(sibfa_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_join, ctx->s2));
    CK(cudaStreamWaitEvent(ctx->s, ctx->ev_join, 0));
    return SIBFA_OK;
}

// Statistics of the last solve (valid after the call's final synchronisation).
void solve_stats(sibfa_ctx *ctx) {
    ctx->last_iters = (int)ctx->h_scal[SC_IT];
    ctx->last_resid = ctx->h_scal[SC_RES];
    if (ctx->pcg_graph_solves) {
        // kernel launches inside the device loop, counted per executed iteration
        ctx->launches += (uint64_t)ctx->last_iters * ctx->pcg_iter_launches * ctx->pcg_graph_solves;
        ctx->pcg_graph_solves = 0;
    }
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory (cudaMallocHost, cudaHostRegister): the copy
// engines read and write it directly, so it needs no staging copy.
bool is_pinned_host_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

template <typename R>
DevState<R> &state(sibfa_ctx *ctx);
template <>
DevState<float> &state<float>(sibfa_ctx *ctx) { return ctx->df; }
template <>
DevState<double> &state<double>(sibfa_ctx *ctx) { return ctx->dd; }

template <typename R>
sibfa_status fft(sibfa_ctx *ctx, DevState<R> &d, bool forward, int ngrid) {
    if (sizeof(R) == 4) {
        if (forward) CKF(cufftExecR2C(ngrid == 1 ? ctx->r2c1 : ctx->r2c2, (cufftReal *)d.grid, (cufftComplex *)d.cgrid));
        else CKF(cufftExecC2R(ngrid == 1 ? ctx->c2r1 : ctx->c2r2, (cufftComplex *)d.cgrid, (cufftReal *)d.grid));
    } else {
        if (forward)
            CKF(cufftExecD2Z(ngrid == 1 ? ctx->r2c1 : ctx->r2c2, (cufftDoubleReal *)d.grid, (cufftDoubleComplex *)d.cgrid));
        else
            CKF(cufftExecZ2D(ngrid == 1 ? ctx->c2r1 : ctx->c2r2, (cufftDoubleComplex *)d.cgrid, (cufftDoubleReal *)d.grid));
    }
    return SIBFA_OK;
}

// T vec (field part): real space into d.efp on s, reciprocal and
// intramolecular into d.efp_r on s2, concurrently; vec is the PCG vector
// already copied to d.vecR.
template <typename R>
sibfa_status matvec(sibfa_ctx *ctx, DevState<R> &d, const double *vec, Launch L) {
    const KParams &p = ctx->kp;
    if (p.periodic) {
        sibfa_status st = fork_rec(ctx);
        if (st) return st;
        Launch L2{ctx->s2, L.count};
        // the grid was cleared by the PCG vector kernel that preceded this product
        launch_spread(p, d, SPREAD_DIP_PCG, vec, d.grid, L2);
        st = fft(ctx, d, true, 1);
        if (st) return st;
        launch_convolve(p, d, d.cgrid, 1, 1, L2);
        st = fft(ctx, d, false, 1);
        if (st) return st;
        launch_gather_field(p, d, d.efp_r, L2);   // includes the intramolecular part
        // serial profiling, outside the captured loop: the real-space product alone
        if (ctx->serial && !ctx->capturing && (st = join_rec(ctx))) return st;
    }
    { Phase ph(ctx, "real_tmu");  launch_real_tmu(p, d, d.efp, L); }
    if (p.periodic) return join_rec(ctx);
    return SIBFA_OK;
}

// One PCG iteration (T p product, step, residual, direction update) captured
// as the body of a graph while-node; the loop runs on the device and the host
// waits once per solve.
template <typename R>
sibfa_status build_pcg_graph(sibfa_ctx *ctx, DevState<R> &d, int maxit) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return SIBFA_E_CUDA;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    cudaGraph_t out = nullptr;
    uint64_t before = ctx->launches;
    sibfa_status st = SIBFA_E_CUDA;
    do {
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(ctx->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess)
            break;
        ctx->capturing = true;
        Launch L{ctx->s, &ctx->launches};
        sibfa_status sm = matvec(ctx, d, d.pv, L);
        launch_pcg_step(ctx->kp, d, L, h, maxit);   // also sets the loop condition
        ctx->capturing = false;
        const cudaError_t ec = cudaStreamEndCapture(ctx->s, &out);
        if (sm != SIBFA_OK || ec != cudaSuccess) break;
        if (cudaGraphInstantiate(&ctx->pcg_exec, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) break;
        st = SIBFA_OK;
    } while (0);
    ctx->capturing = false;
    ctx->pcg_iter_launches = ctx->launches - before;
    ctx->launches = before;     // counted per executed iteration instead
    cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
}

// Initial guess from the stored solutions of full evaluations: the
// polynomial through the last n of them (times -1..-n) taken at time 0,
// coefficients (-1)^(j+1) C(n, j) for the j-th newest.
MuGuess mu_guess(const sibfa_ctx *ctx, bool full) {
    MuGuess g{};
    const int want = ctx->opts.warm_start;
    if (!full || want < 2 || ctx->hist_n < 1) return g;
    static const double C[MU_HIST + 1][MU_HIST] = {{0, 0, 0, 0, 0, 0},      {1, 0, 0, 0, 0, 0},
                                                  {2, -1, 0, 0, 0, 0},     {3, -3, 1, 0, 0, 0},
                                                  {4, -6, 4, -1, 0, 0},    {5, -10, 10, -5, 1, 0},
                                                  {6, -15, 20, -15, 6, -1}};
    g.n = std::min(want, ctx->hist_n);
    const size_t stride = (size_t)ctx->capacity * 9;
    for (int j = 0; j < g.n; ++j) {
        g.h[j] = ctx->mu_hist + (size_t)((ctx->hist_head - 1 - j + 2 * want) % want) * stride;
        g.c[j] = C[g.n][j];
    }
    return g;
}

// Store the converged dipoles of a full evaluation (stream-ordered after the solve).
sibfa_status push_mu(sibfa_ctx *ctx, const double *mu, bool full) {
    if (!full || ctx->opts.warm_start < 2) return SIBFA_OK;
    const size_t stride = (size_t)ctx->capacity * 9;
    CK(cudaMemcpyAsync(ctx->mu_hist + (size_t)ctx->hist_head * stride, mu, (size_t)ctx->M * 9 * sizeof(double),
                       cudaMemcpyDeviceToDevice, ctx->s));
    ctx->hist_head = (ctx->hist_head + 1) % ctx->opts.warm_start;
    ctx->hist_n = std::min(ctx->hist_n + 1, ctx->opts.warm_start);
    return SIBFA_OK;
}

template <typename R>
sibfa_status solve(sibfa_ctx *ctx, DevState<R> &d, double tol, Launch L, bool full) {
    const KParams &p = ctx->kp;
    const int warm = (ctx->opts.warm_start && ctx->have_mu) ? 1 : 0;
    const MuGuess g = mu_guess(ctx, full);
    if (g.n > 0) launch_pcg_init_guess(p, d, g, L);
    else launch_pcg_init(p, d, warm, L);
    sibfa_status st = matvec(ctx, d, d.mu, L);
    if (st) return st;
    launch_pcg_first(p, d, L);
    double *h = ctx->h_pin;
    int it = 0;
    const int maxit = ctx->opts.pcg_max_iter > 0 ? ctx->opts.pcg_max_iter : 200;
    if (ctx->pcg_graph_state == 0) ctx->pcg_graph_state = build_pcg_graph(ctx, d, maxit) == SIBFA_OK ? 1 : -1;
    if (ctx->pcg_graph_state == 1) {
        // device-side loop; no host synchronisation: the convergence check is a
        // flag and the statistics are read at the end of the call
        CK(cudaGraphLaunch(ctx->pcg_exec, ctx->s));
        launch_pcg_check(d.scal, d.flags, L);
        CK(cudaMemcpyAsync(ctx->h_scal, d.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
        ctx->pcg_graph_solves += 1;
        ctx->have_mu = true;
        return push_mu(ctx, d.mu, full);
    }
    for (;;) {
        CK(cudaMemcpyAsync(h, d.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        if (h[SC_DONE] != 0.0 || it >= maxit) break;
        st = matvec(ctx, d, d.pv, L);
        if (st) return st;
        launch_pcg_step(p, d, L);
        ++it;
    }
    std::memcpy(ctx->h_scal, h, 16 * sizeof(double));
    ctx->have_mu = true;
    launch_pcg_check(d.scal, d.flags, L);
    return push_mu(ctx, d.mu, full);
}

// One evaluation on the positions already in d.pos.
template <typename R>
sibfa_status evaluate_impl(sibfa_ctx *ctx, bool want_forces, bool dipoles_only, double tol);

// One evaluation; the short-range stream is joined back on every path.
// Full evaluations (not the dipole-only solve nor the virial variant) feed
// the short-range autotuner.
template <typename R>
sibfa_status evaluate(sibfa_ctx *ctx, bool want_forces, bool dipoles_only, double tol) {
    auto &T = ctx->tune;
    // relaxation steps start each solve far from its answer (many more PCG
    // iterations than along a trajectory), so they are not timed
    const bool timed = T.on && T.choice < 0 && !dipoles_only && !ctx->kp.vir && !ctx->capturing && !ctx->minimizing;
    if (timed) {
        tune_account(ctx);
        if (T.choice < 0) CK(cudaEventRecord(T.e0, ctx->s));
    }
    const sibfa_status st = evaluate_impl<R>(ctx, want_forces, dipoles_only, tol);
    const sibfa_status sj = join_short(ctx);
    const sibfa_status sc = join_ct(ctx);
    if (timed && T.choice < 0) {
        CK(cudaEventRecord(T.e1, ctx->s));
        T.pending = true;
    }
    return st ? st : (sj ? sj : sc);
}

template <typename R>
sibfa_status evaluate_impl(sibfa_ctx *ctx, bool want_forces, bool dipoles_only, double tol) {
    DevState<R> &d = state<R>(ctx);
    DevState<R> dr = rec_view(d);   // accumulators of the reciprocal chain
    const KParams &p = ctx->kp;
    Launch L{ctx->s, &ctx->launches};
    Launch L2{ctx->s2, &ctx->launches};
    launch_begin(d.scal, d.flags, tol, L);
    { Phase ph(ctx, "sites");  launch_sites(p, d, L); }
    const size_t ng = (size_t)p.K[0] * p.K[1] * p.K[2];
    sibfa_status st;
    if (p.periodic) {
        // permanent multipoles in reciprocal space, concurrent with the
        // neighbour list and the real-space pair kernels
        if ((st = fork_rec(ctx))) return st;
        Phase ph(ctx, "spme_perm", ctx->s2);
        CK(cudaMemsetAsync(d.grid, 0, ng * sizeof(R), ctx->s2));
        launch_spread(p, d, SPREAD_PERM, nullptr, d.grid, L2);
        if ((st = fft(ctx, d, true, 1))) return st;
        if (p.vir) launch_convolve_vir(p, d, 0, L2);
        else launch_convolve(p, d, d.cgrid, 1, 0, L2);
        if ((st = fft(ctx, d, false, 1))) return st;
        launch_gather_perm(p, dr, L2);
        launch_intra_perm(p, dr, L2);
        if (ctx->serial && (st = join_rec(ctx))) return st;
    }
    { Phase ph(ctx, "neighbors");  launch_neighbors(p, d, ctx->ncell, L); }
    // Short-range terms on the third, lowest-priority stream beside the
    // permanent pass and the solve (which is latency-bound and leaves SMs
    // idle): their short blocks fill in behind the other streams' work.  They
    // write their own gradient array and are joined before the chain rule.
    // The virial variant runs in order on the main stream.
    const bool bg_short = !dipoles_only && !p.vir && !ctx->serial;
    if (bg_short) {
        if ((st = fork_short(ctx))) return st;
        ctx->short_pending = true;
        Phase ph(ctx, "short", ctx->s3);
        DevState<R> ds = short_view(d);
        // resident blocks per SM (0: uncapped), chosen by the autotuner: a cap
        // leaves every SM registers for the solve's small kernels
        launch_short(p, ds, Launch{ctx->s3, &ctx->launches}, 0, short_cap(ctx));
    }
    // mixed periodic path: the FP64 intramolecular Ewald energy, beside everything else
    if (sizeof(R) == 4 && p.periodic && !dipoles_only)
        launch_intra_energy64(p, d, bg_short ? Launch{ctx->s3, &ctx->launches} : L);
    // Lone-pair potentials and then the charge transfer on the fourth stream
    // (the transfer after the reciprocal chain); joined before the
    // polarization energy, which copies the lambdas.
    const bool bg_ct = !dipoles_only && !p.vir && !ctx->serial;
    if (bg_ct) {
        if ((st = fork_ct(ctx))) return st;
        ctx->ct_pending = true;
        launch_lp_potential(p, d, Launch{ctx->s4, &ctx->launches});
    }
    { Phase ph(ctx, "real_perm");  launch_real_perm(p, d, L); }
    if (!dipoles_only && !bg_short) { Phase ph(ctx, "short");  launch_short(p, d, L); }
    if (p.periodic) {
        if ((st = join_rec(ctx))) return st;
        launch_merge_rec(p, d, L);
    }
    if (!dipoles_only) {
        if (!bg_ct) {
            launch_lp_potential(p, d, L);
            Phase ph(ctx, "ct");
            launch_ct(p, d, L);
        } else {   // beside the solve, which does not read its results
            // after the permanent pass on this stream (both add into the
            // point gradients) and the reciprocal chain (lone-pair potentials)
            if ((st = fork_ct(ctx))) return st;
            Phase ph(ctx, "ct", ctx->s4);
            launch_ct(p, d, Launch{ctx->s4, &ctx->launches});
        }
    }
    // schedule choice: the short-range kernels finish before the solve
    if (bg_short && short_sched(ctx).join_before_solve && (st = join_short(ctx))) return st;
    {
        Phase ph(ctx, "pcg");
        st = solve(ctx, d, tol, L, !dipoles_only);
    }
    if (st == SIBFA_E_CUDA) return st;
    sibfa_status st_solve = st;
    if (dipoles_only) return st_solve;
    // the lambdas of the charge transfer feed k_pol_energy's working-precision copy
    if ((st = join_ct(ctx))) return st;
    launch_pol_energy(p, d, L);
    if (want_forces) {
        if (p.periodic) {
            // induced dipoles and charge-transfer lambdas in reciprocal space,
            // concurrent with the real-space force kernel
            sibfa_status sf = fork_rec(ctx);
            if (sf) return sf;
            Phase ph(ctx, "spme_polforce", ctx->s2);
            CK(cudaMemsetAsync(d.grid, 0, 2 * ng * sizeof(R), ctx->s2));
            launch_spread(p, d, SPREAD_DIP, nullptr, d.grid, L2);
            launch_spread(p, d, SPREAD_LAMBDA, nullptr, d.grid + ng, L2);
            if ((sf = fft(ctx, d, true, 2))) return sf;
            if (p.vir) launch_convolve_vir(p, d, 1, L2);
            else launch_convolve(p, d, d.cgrid, 2, 0, L2);
            if ((sf = fft(ctx, d, false, 2))) return sf;
            launch_gather_polforce(p, dr, L2);
            launch_intra_polforce(p, dr, L2);
            if (ctx->serial && (sf = join_rec(ctx))) return sf;
        }
        { Phase ph(ctx, "real_polforce");  launch_real_polforce(p, d, L); }
        if (p.periodic) {
            sibfa_status sj = join_rec(ctx);
            if (sj) return sj;
        }
        if ((st = join_short(ctx))) return st;
        { Phase ph(ctx, "finalize");  launch_finalize(p, d, ctx->d_forces, L); }
    }
    if ((st = join_short(ctx))) return st;
    if (p.n_cl > 1) launch_cluster_energy(p, d, ctx->d_energy, L);
    else launch_energy_reduce(p.M, d.epart, d.epart_r, (sizeof(R) == 4 && p.periodic) ? d.eintra : nullptr,
                              d.epartial, ctx->d_energy, L);
    return st_solve;
}

sibfa_status check_flags(sibfa_ctx *ctx, int flags) {
    if (flags & F_CUTOFF) {
        ctx->err = "cutoff plus twice the site extent exceeds half the box (or a site is > 1.3 A from its O)";
        return SIBFA_E_CUTOFF;
    }
    if (flags & F_NEIGHBOR) {
        ctx->err = "neighbour list overflow";
        return SIBFA_E_NEIGHBOR;
    }
    if (flags & F_CTDEN) {
        ctx->err = "charge-transfer denominator ae + V - ah <= 0";
        return SIBFA_E_CT_DENOM;
    }
    if (flags & F_NOCONV) {
        ctx->err = "PCG did not reach the tolerance within pcg_max_iter";
        return SIBFA_E_NOT_CONVERGED;
    }
    return SIBFA_OK;
}

// A new orthorhombic box for a periodic context (constant-pressure MD):
// the box-dependent parameters (box, inverse box, fixed-point scale, SPME
// grid points per length), the influence function, the cell grid (within
// the cells allocated at create), the dispersion tail (proportional to
// 1/V), a neighbour-list rebuild at the next evaluation, and the captured
// solve loop (its kernels hold the parameters by value) rebuilt on first
// use.  Called on the work stream after enter().
template <typename R>
sibfa_status set_box(sibfa_ctx *ctx, DevState<R> &d, const double *box) {
    for (int k = 0; k < 3; ++k)
        if (!(box[k] > 0)) {
            ctx->err = "box lengths must be > 0";
            return SIBFA_E_INVALID;
        }
    const double half = 0.5 * std::min(box[0], std::min(box[1], box[2]));
    if (ctx->opts.rc + 2.0 * 0.9572 > half) {
        ctx->err = "rc + 2 * O-H distance exceeds half the new box";
        return SIBFA_E_CUTOFF;
    }
    const double cell = ctx->opts.rc + 2.6 + LIST_SKIN;
    int nc[3];
    for (int k = 0; k < 3; ++k) nc[k] = (int)floor(box[k] / cell);
    if (nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3 && nc[0] * nc[1] * nc[2] > ctx->ncell_cap) {
        ctx->err = "the new box needs more cells than the context allocated at create";
        return SIBFA_E_INVALID;
    }
    const double v_old = ctx->kp.box[0] * ctx->kp.box[1] * ctx->kp.box[2];
    KParams &k = ctx->kp;
    for (int i = 0; i < 3; ++i) {
        ctx->opts.box[i] = box[i];
        k.box[i] = box[i];
        k.ibox[i] = 1.0 / box[i];
        k.fxs[i] = (float)(box[i] / 4294967296.0);
        ctx->ncell[i] = nc[i];
    }
    fill_scal(k.sd, k);
    fill_scal(k.sf, k);
    ctx->e_tail *= v_old / (box[0] * box[1] * box[2]);
    Launch L{ctx->s, &ctx->launches};
    launch_influence(k, d.infl, L);
    launch_influence_copy(k, d, L);
    CK(cudaMemsetAsync(d.lflag + 1, 0, sizeof(int), ctx->s));   // no list yet: rebuild
    if (ctx->pcg_graph_state == 1) {
        cudaGraphExecDestroy(ctx->pcg_exec);
        ctx->pcg_exec = nullptr;
        ctx->pcg_graph_state = 0;
    }
    return SIBFA_OK;
}

template <typename R>
sibfa_status run(sibfa_ctx *ctx, const double *pos, const double *box, sibfa_energy_terms *e, double *forces,
                 bool dipoles_only, double tol, double *mu_out, int *iters, double *resid, double *virial = nullptr) {
    DevState<R> &d = state<R>(ctx);
    const int M = ctx->M;
    const size_t nb = (size_t)M * 9 * sizeof(double);
    if (virial && ctx->kp.ct_orig) {
        ctx->err = "the virial is not available with the original charge transfer";
        return SIBFA_E_INVALID;
    }
    bool new_box = false;
    if (box) {
        for (int k = 0; k < 3; ++k) new_box = new_box || box[k] != ctx->kp.box[k];
        if (new_box && !ctx->opts.periodic) {
            ctx->err = "a gas-phase context has no box";
            return SIBFA_E_INVALID;
        }
    }
    sibfa_status st0 = enter(ctx);
    if (st0) return st0;
    if (new_box && (st0 = set_box<R>(ctx, d, box))) return leave(ctx) ? SIBFA_E_CUDA : st0;
    CK(cudaMemsetAsync(d.flags, 0, sizeof(int), ctx->s));
    if (pos) {
        if (is_device_ptr(pos)) {
            CK(cudaMemcpyAsync(d.pos, pos, nb, cudaMemcpyDeviceToDevice, ctx->s));
        } else if (is_pinned_host_ptr(pos)) {
            CK(cudaMemcpyAsync(d.pos, pos, nb, cudaMemcpyHostToDevice, ctx->s));
        } else {
            CK(cudaStreamSynchronize(ctx->s));
            std::memcpy(ctx->h_pin, pos, nb);
            CK(cudaMemcpyAsync(d.pos, ctx->h_pin, nb, cudaMemcpyHostToDevice, ctx->s));
        }
    }
    ctx->md_forces_valid = false;
    // the virial needs the force pass; kernels read the switch from their parameters
    ctx->kp.vir = virial != nullptr;
    sibfa_status st = evaluate<R>(ctx, forces != nullptr || virial != nullptr, dipoles_only, tol);
    ctx->kp.vir = 0;
    if (st == SIBFA_E_CUDA) return st;
    double *h = ctx->h_pin;
    if (virial) {
        KParams pv = ctx->kp;
        pv.vir = 1;
        launch_virial_total(pv, d, ctx->d_energy + 16, Launch{ctx->s, &ctx->launches});
        CK(cudaMemcpyAsync(h + 20, ctx->d_energy + 16, 9 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    }
    // results: energies + flags (+ dipoles) to pinned memory
    CK(cudaMemcpyAsync(h, ctx->d_energy, (NTERM + 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync((int *)(h + 16), d.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    // outputs: device memory device to device, page-locked host memory
    // directly, pageable host memory through the pinned staging buffer
    const bool f_dev = is_device_ptr(forces), f_pin = !f_dev && is_pinned_host_ptr(forces);
    const bool m_dev = is_device_ptr(mu_out), m_pin = !m_dev && is_pinned_host_ptr(mu_out);
    if (forces) {
        if (f_dev) CK(cudaMemcpyAsync(forces, ctx->d_forces, nb, cudaMemcpyDeviceToDevice, ctx->s));
        else CK(cudaMemcpyAsync(f_pin ? forces : h + 32, ctx->d_forces, nb, cudaMemcpyDeviceToHost, ctx->s));
    }
    if (mu_out) {
        if (m_dev) CK(cudaMemcpyAsync(mu_out, d.mu, nb, cudaMemcpyDeviceToDevice, ctx->s));
        else CK(cudaMemcpyAsync(m_pin ? mu_out : h + 32, d.mu, nb, cudaMemcpyDeviceToHost, ctx->s));
    }
    st0 = leave(ctx);
    if (st0) return st0;
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaGetLastError());
    if (forces && !f_dev && !f_pin) std::memcpy(forces, h + 32, nb);
    if (virial) {
        std::memcpy(virial, h + 20, 9 * sizeof(double));
        // the tail scales as 1/V at fixed cutoff: W = -dE/d eps = E_tail on the diagonal
        virial[0] += ctx->e_tail;
        virial[4] += ctx->e_tail;
        virial[8] += ctx->e_tail;
    }
    if (mu_out && !m_dev && !m_pin) std::memcpy(mu_out, h + 32, nb);
    solve_stats(ctx);
    sibfa_status fl = check_flags(ctx, *(int *)(h + 16));
    if (fl && fl != SIBFA_E_NOT_CONVERGED) return fl;
    if (fl) st = fl;
    if (e) {
        e->elec = h[T_ELEC];
        e->pen = h[T_PEN];
        e->rep = h[T_REP];
        e->disp = h[T_DISP] + ctx->e_tail;
        e->xdisp = h[T_XDISP];
        e->pol = h[T_POL];
        e->ct = h[T_CT];
        e->total = h[NTERM] + ctx->e_tail;
    }
    if (iters) *iters = ctx->last_iters;
    if (resid) *resid = ctx->last_resid;
    return st;
}

template <typename R>
sibfa_status create_impl(sibfa_ctx *ctx, const sibfa_topology *topo) {
    const int M = ctx->M;
    sibfa_status st = alloc_state<R>(ctx, state<R>(ctx));
    if (st) return st;
    DevState<R> &d = state<R>(ctx);
    CK(cudaMemcpyAsync(d.mp_local, topo->mp_local, (size_t)M * NS * NMP * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->s));
    {
        const int nc = ctx->kp.n_cl;
        std::vector<int> start(nc + 1), of(M);
        if (nc > 1) std::memcpy(start.data(), topo->cluster_start, (nc + 1) * sizeof(int));
        else start[0] = 0, start[1] = M;
        for (int c = 0; c < nc; ++c)
            for (int m = start[c]; m < start[c + 1]; ++m) of[m] = c;
        CK(cudaMemcpyAsync(d.cl_start, start.data(), (nc + 1) * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
        CK(cudaMemcpyAsync(d.cl_of, of.data(), M * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
    }
    CK(cudaStreamSynchronize(ctx->s));
    if (ctx->opts.periodic) {
        Launch L{ctx->s, &ctx->launches};
        launch_influence(ctx->kp, d.infl, L);
        launch_influence_copy(ctx->kp, d, L);
        int n[3] = {ctx->kp.K[0], ctx->kp.K[1], ctx->kp.K[2]};
        const bool f32 = sizeof(R) == 4;
        const int ng = n[0] * n[1] * n[2], nh = n[0] * n[1] * (n[2] / 2 + 1);
        CKF(cufftPlan3d(&ctx->r2c1, n[0], n[1], n[2], f32 ? CUFFT_R2C : CUFFT_D2Z));
        CKF(cufftPlan3d(&ctx->c2r1, n[0], n[1], n[2], f32 ? CUFFT_C2R : CUFFT_Z2D));
        CKF(cufftPlanMany(&ctx->r2c2, 3, n, nullptr, 1, ng, nullptr, 1, nh, f32 ? CUFFT_R2C : CUFFT_D2Z, 2));
        CKF(cufftPlanMany(&ctx->c2r2, 3, n, nullptr, 1, nh, nullptr, 1, ng, f32 ? CUFFT_C2R : CUFFT_Z2D, 2));
        CKF(cufftSetStream(ctx->r2c1, ctx->s2));
        CKF(cufftSetStream(ctx->c2r1, ctx->s2));
        CKF(cufftSetStream(ctx->r2c2, ctx->s2));
        CKF(cufftSetStream(ctx->c2r2, ctx->s2));
        ctx->have_fft = true;
    }
    CK(cudaStreamSynchronize(ctx->s));
    return SIBFA_OK;
}

}  // namespace

__global__ void k_inverse(int n, const double *a, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = 1.0 / a[k];
}

template <typename R>
static sibfa_status md_impl(sibfa_ctx *ctx, double *pos, double *vel, const double *masses, double dt, int n,
                            sibfa_energy_terms *e) {
    DevState<R> &d = state<R>(ctx);
    const int M = ctx->M;
    const size_t nb = (size_t)M * 9 * sizeof(double);
    if (!is_device_ptr(pos) || !is_device_ptr(vel) || !is_device_ptr(masses)) {
        ctx->err = "sibfa_md_steps needs device pointers for pos, vel and masses";
        return SIBFA_E_INVALID;
    }
    if (!ctx->d_invm) {
        // sized for the capacity: a batch context grows after its first MD call
        sibfa_status st = dalloc(ctx, &ctx->d_invm, (size_t)ctx->capacity * 3);
        if (st) return st;
    }
    const double tol = ctx->opts.pcg_tol_D > 0 ? ctx->opts.pcg_tol_D : 1e-6;
    Launch L{ctx->s, &ctx->launches};
    sibfa_status st_e = enter(ctx);
    if (st_e) return st_e;
    k_inverse<<<(M * 3 + 255) / 256, 256, 0, ctx->s>>>(M * 3, masses, ctx->d_invm);
    ctx->launches += 1;
    CK(cudaMemsetAsync(d.flags, 0, sizeof(int), ctx->s));
    CK(cudaMemcpyAsync(d.pos, pos, nb, cudaMemcpyDeviceToDevice, ctx->s));
    const sibfa_run_opts &o = ctx->opts;
    const double th0 = o.md_theta0_deg * M_PI / 180.0;
    sibfa_status st = SIBFA_OK;
    const bool beeman = o.md_integrator == 1;
    if (beeman && !ctx->d_fprev) {
        sibfa_status sa = dalloc(ctx, &ctx->d_fprev, (size_t)ctx->capacity * 9);
        if (sa) {
            leave(ctx);
            return sa;
        }
    }
    if (!ctx->md_forces_valid) {
        st = evaluate<R>(ctx, true, false, tol);
        if (st) {
            leave(ctx);   // keep the caller's stream ordered after what was queued
            return st;
        }
        launch_water_intra(M, d.pos, ctx->d_forces, o.md_k_bond, o.md_r0, o.md_k_angle, th0, o.md_anharmonic,
                           o.md_k_ub, o.md_r_ub, L);
        // Beeman's first step takes a(t - dt) = a(t)
        if (beeman) CK(cudaMemcpyAsync(ctx->d_fprev, ctx->d_forces, nb, cudaMemcpyDeviceToDevice, ctx->s));
    }
    for (int k = 0; k < n; ++k) {
        if (beeman) launch_beeman(M, d.pos, vel, ctx->d_invm, ctx->d_forces, ctx->d_fprev, dt, 1, L);
        else launch_md_kick(M, d.pos, vel, ctx->d_invm, ctx->d_forces, dt, 1, L);
        st = evaluate<R>(ctx, true, false, tol);
        if (st) {
            ctx->md_forces_valid = false;
            leave(ctx);
            return st;
        }
        launch_water_intra(M, d.pos, ctx->d_forces, o.md_k_bond, o.md_r0, o.md_k_angle, th0, o.md_anharmonic,
                           o.md_k_ub, o.md_r_ub, L);
        if (beeman) launch_beeman(M, d.pos, vel, ctx->d_invm, ctx->d_forces, ctx->d_fprev, dt, 2, L);
        else launch_md_kick(M, d.pos, vel, ctx->d_invm, ctx->d_forces, dt, 0, L);
    }
    CK(cudaMemcpyAsync(pos, d.pos, nb, cudaMemcpyDeviceToDevice, ctx->s));
    double *h = ctx->h_pin;
    CK(cudaMemcpyAsync(h, ctx->d_energy, (NTERM + 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync((int *)(h + 16), d.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    st_e = leave(ctx);
    if (st_e) return st_e;
    CK(cudaStreamSynchronize(ctx->s));
    ctx->md_forces_valid = true;
    solve_stats(ctx);
    sibfa_status fl = check_flags(ctx, *(int *)(h + 16));
    if (fl) return fl;
    if (e) {
        e->elec = h[T_ELEC]; e->pen = h[T_PEN]; e->rep = h[T_REP]; e->disp = h[T_DISP] + ctx->e_tail;
        e->xdisp = h[T_XDISP]; e->pol = h[T_POL]; e->ct = h[T_CT]; e->total = h[NTERM] + ctx->e_tail;
    }
    return SIBFA_OK;
}

extern "C" {

sibfa_status sibfa_create(const sibfa_params *params, const sibfa_topology *topo, const sibfa_run_opts *opts,
                          sibfa_ctx **out) {
    if (out) *out = nullptr;
    if (!params || !topo || !opts || !out || topo->n_mol <= 0 || !topo->mp_local) {
        g_create_error = "sibfa_create: null argument or n_mol <= 0";
        return SIBFA_E_INVALID;
    }
    if (topo->n_clusters > 1) {
        bool ok = !opts->periodic && topo->cluster_start && topo->cluster_start[0] == 0 &&
                  topo->cluster_start[topo->n_clusters] == topo->n_mol;
        for (int c = 0; ok && c < topo->n_clusters; ++c) {
            const int n = topo->cluster_start[c + 1] - topo->cluster_start[c];
            ok = n >= 1 && n <= MAXN + 1;
        }
        if (!ok) {
            g_create_error = "sibfa_create: cluster batches need periodic = 0 and increasing cluster_start from 0 to "
                             "n_mol with 1..385 molecules per cluster";
            return SIBFA_E_INVALID;
        }
    }
    if (opts->precision != SIBFA_PREC_FP64 && opts->precision != SIBFA_PREC_MIXED) {
        g_create_error = "sibfa_create: unknown precision";
        return SIBFA_E_INVALID;
    }
    if (opts->ct_original < 0 || opts->ct_original > 1) {
        g_create_error = "sibfa_create: ct_original must be 0 (reduced) or 1 (original)";
        return SIBFA_E_INVALID;
    }
    if (opts->md_integrator < 0 || opts->md_integrator > 1) {
        g_create_error = "sibfa_create: md_integrator must be 0 (velocity Verlet) or 1 (Beeman)";
        return SIBFA_E_INVALID;
    }
    if (opts->warm_start < 0 || opts->warm_start > MU_HIST) {
        g_create_error = "sibfa_create: warm_start must be 0..6";
        return SIBFA_E_INVALID;
    }
    if (opts->periodic) {
        if (opts->order != 5 && opts->order != 0) {
            g_create_error = "sibfa_create: only B-spline order 5 is implemented";
            return SIBFA_E_INVALID;
        }
        for (int k = 0; k < 3; ++k)
            if (!(opts->box[k] > 0) || opts->grid[k] < 8) {
                g_create_error = "sibfa_create: box lengths must be > 0 and grid sizes >= 8";
                return SIBFA_E_INVALID;
            }
        if (!(opts->rc > 0) || !(opts->ewald_alpha > 0)) {
            g_create_error = "sibfa_create: rc and ewald_alpha must be > 0";
            return SIBFA_E_INVALID;
        }
        const double half = 0.5 * std::min(opts->box[0], std::min(opts->box[1], opts->box[2]));
        if (opts->rc + 2.0 * 0.9572 > half) {
            g_create_error = "sibfa_create: rc + 2 * O-H distance exceeds half the box";
            return SIBFA_E_CUTOFF;
        }
    }
    sibfa_ctx *ctx = new sibfa_ctx();
    ctx->M = topo->n_mol;
    ctx->capacity = topo->n_mol;
    ctx->opts = *opts;
    ctx->prec = opts->precision;
    ctx->us = (cudaStream_t)opts->stream;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    // the reciprocal chain is a sequence of small latency-bound kernels: it
    // gets the highest priority so that its blocks start ahead of the large
    // real-space grids that run beside it; the short-range kernels the
    // lowest, so that they only take what the other two streams leave
    const int prio_mid = prio_hi < prio_lo ? prio_hi + 1 : prio_hi;
    if (cudaStreamCreateWithPriority(&ctx->s, cudaStreamNonBlocking, prio_mid) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ctx->s2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ctx->s3, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ctx->s4, cudaStreamNonBlocking, prio_mid) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork4, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&ctx->tune.e0) != cudaSuccess || cudaEventCreate(&ctx->tune.e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join4, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork3, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join3, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        g_create_error = "sibfa_create: could not create the work stream";
        delete ctx;
        return SIBFA_E_CUDA;
    }
    fill_params(ctx->kp, *params, *opts, ctx->M);
    if (opts->periodic && opts->disp_tail)
        ctx->e_tail = disp_tail_energy(*params, ctx->M, opts->box[0] * opts->box[1] * opts->box[2], opts->rc);
    ctx->kp.n_cl = topo->n_clusters > 1 ? topo->n_clusters : 1;
    {
        // the most neighbours a molecule can have: the list capacity in a box,
        // the largest cluster minus one in the gas phase
        int nmax = MAXN;
        if (!opts->periodic) {
            int big = topo->n_mol;
            if (topo->n_clusters > 1) {
                big = 0;
                for (int c = 0; c < topo->n_clusters; ++c)
                    big = std::max(big, topo->cluster_start[c + 1] - topo->cluster_start[c]);
            }
            nmax = std::min(MAXN, std::max(1, big - 1));
        }
        ctx->kp.tls = 3 * nmax;
    }
    {
        const char *e = getenv("SIBFA_PCG_HOST_LOOP");
        if (e && e[0] == '1') ctx->pcg_graph_state = -1;
        const char *t = getenv("SIBFA_TUNE");
        if (t && t[0] == '0') ctx->tune.on = false;
    }
    if (opts->periodic) {
        const double cell = opts->rc + 2.6 + LIST_SKIN;   // rc + 2 * maximum site extent (1.3 A) + skin
        for (int k = 0; k < 3; ++k) ctx->ncell[k] = (int)floor(opts->box[k] / cell);
    }
    sibfa_status st = SIBFA_OK;
    do {
        st = dalloc(ctx, &ctx->d_forces, (size_t)ctx->M * 9);
        if (st) break;
        st = dalloc(ctx, &ctx->d_energy, 32);
        if (st) break;
        if (opts->warm_start >= 2) {
            st = dalloc(ctx, &ctx->mu_hist, (size_t)opts->warm_start * ctx->capacity * 9);
            if (st) break;
        }
        if (cudaMallocHost((void **)&ctx->h_pin, ((size_t)ctx->M * 9 * 2 + 64) * sizeof(double)) != cudaSuccess ||
            cudaMallocHost((void **)&ctx->h_scal, 16 * sizeof(double)) != cudaSuccess) {
            ctx->err = "cudaMallocHost failed";
            st = SIBFA_E_OOM;
            break;
        }
        st = ctx->prec == SIBFA_PREC_MIXED ? create_impl<float>(ctx, topo) : create_impl<double>(ctx, topo);
    } while (0);
    if (st != SIBFA_OK) {
        g_create_error = ctx->err;
        sibfa_destroy(ctx);
        return st;
    }
    *out = ctx;
    return SIBFA_OK;
}

sibfa_status sibfa_energy_forces(sibfa_ctx *ctx, const double *pos, const double *box, sibfa_energy_terms *e,
                                 double *forces, double *virial) {
    if (!ctx || !pos) return SIBFA_E_INVALID;
    const double tol = ctx->opts.pcg_tol_D > 0 ? ctx->opts.pcg_tol_D : 1e-6;
    return ctx->prec == SIBFA_PREC_MIXED
               ? run<float>(ctx, pos, box, e, forces, false, tol, nullptr, nullptr, nullptr, virial)
               : run<double>(ctx, pos, box, e, forces, false, tol, nullptr, nullptr, nullptr, virial);
}

sibfa_status sibfa_solve_dipoles(sibfa_ctx *ctx, const double *pos, const double *box, double tol_D, double *mu,
                                 int *iters, double *resid_D) {
    if (!ctx || !pos) return SIBFA_E_INVALID;
    const double tol = tol_D > 0 ? tol_D : (ctx->opts.pcg_tol_D > 0 ? ctx->opts.pcg_tol_D : 1e-6);
    return ctx->prec == SIBFA_PREC_MIXED ? run<float>(ctx, pos, box, nullptr, nullptr, true, tol, mu, iters, resid_D)
                                         : run<double>(ctx, pos, box, nullptr, nullptr, true, tol, mu, iters, resid_D);
}

}  // extern "C"

template <typename R>
static sibfa_status minimize_impl(sibfa_ctx *ctx, double *pos, int n, double cap, sibfa_energy_terms *e) {
    DevState<R> &d = state<R>(ctx);
    const int M = ctx->M;
    const size_t nb = (size_t)M * 9 * sizeof(double);
    if (!is_device_ptr(pos)) {
        ctx->err = "sibfa_minimize needs a device pointer for pos";
        return SIBFA_E_INVALID;
    }
    const double tol = ctx->opts.pcg_tol_D > 0 ? ctx->opts.pcg_tol_D : 1e-6;
    Launch L{ctx->s, &ctx->launches};
    const sibfa_run_opts &o = ctx->opts;
    const double th0 = o.md_theta0_deg * M_PI / 180.0;
    sibfa_status st_e = enter(ctx);
    if (st_e) return st_e;
    // Relaxation steps are not a trajectory to extrapolate along: the stored
    // dipole history is cleared on every exit from here on, error or not.
    struct ClearHistory {
        sibfa_ctx *c;
        ~ClearHistory() {
            c->hist_n = 0;
            c->md_forces_valid = false;
            c->minimizing = false;
        }
    } clear_history{ctx};
    ctx->minimizing = true;
    CK(cudaMemsetAsync(d.flags, 0, sizeof(int), ctx->s));
    CK(cudaMemcpyAsync(d.pos, pos, nb, cudaMemcpyDeviceToDevice, ctx->s));
    for (int k = 0; k < n; ++k) {
        sibfa_status st = evaluate<R>(ctx, true, false, tol);
        if (st) {
            leave(ctx);   // keep the caller's stream ordered after what was queued
            return st;
        }
        launch_water_intra(M, d.pos, ctx->d_forces, o.md_k_bond, o.md_r0, o.md_k_angle, th0, o.md_anharmonic,
                           o.md_k_ub, o.md_r_ub, L);
        launch_sd_step(M, d.pos, ctx->d_forces, 1e-4, cap, L);
    }
    CK(cudaMemcpyAsync(pos, d.pos, nb, cudaMemcpyDeviceToDevice, ctx->s));
    double *h = ctx->h_pin;
    CK(cudaMemcpyAsync(h, ctx->d_energy, (NTERM + 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync((int *)(h + 16), d.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    st_e = leave(ctx);
    if (st_e) return st_e;
    CK(cudaStreamSynchronize(ctx->s));
    solve_stats(ctx);
    {
        sibfa_status fl = check_flags(ctx, *(int *)(h + 16));
        if (fl) return fl;
    }
    if (e) {
        e->elec = h[T_ELEC]; e->pen = h[T_PEN]; e->rep = h[T_REP]; e->disp = h[T_DISP] + ctx->e_tail;
        e->xdisp = h[T_XDISP]; e->pol = h[T_POL]; e->ct = h[T_CT]; e->total = h[NTERM] + ctx->e_tail;
    }
    return SIBFA_OK;
}

extern "C" {

sibfa_status sibfa_minimize(sibfa_ctx *ctx, double *pos, int n_steps, double max_disp_A, sibfa_energy_terms *e) {
    if (!ctx || !pos || n_steps < 0 || !(max_disp_A > 0)) return SIBFA_E_INVALID;
    return ctx->prec == SIBFA_PREC_MIXED ? minimize_impl<float>(ctx, pos, n_steps, max_disp_A, e)
                                         : minimize_impl<double>(ctx, pos, n_steps, max_disp_A, e);
}

sibfa_status sibfa_md_steps(sibfa_ctx *ctx, double *pos, double *vel, const double *masses, double dt_fs, int n_steps,
                            sibfa_energy_terms *e) {
    if (!ctx || !pos || !vel || !masses || n_steps < 0) return SIBFA_E_INVALID;
    return ctx->prec == SIBFA_PREC_MIXED ? md_impl<float>(ctx, pos, vel, masses, dt_fs, n_steps, e)
                                         : md_impl<double>(ctx, pos, vel, masses, dt_fs, n_steps, e);
}

sibfa_status sibfa_cluster_terms(sibfa_ctx *ctx, sibfa_energy_terms *terms) {
    if (!ctx || !terms) return SIBFA_E_INVALID;
    const int nc = ctx->kp.n_cl;
    std::vector<double> h((size_t)nc * (NTERM + 1));
    const double *src = ctx->d_energy;
    if (nc > 1) src = ctx->prec == SIBFA_PREC_MIXED ? ctx->df.cl_energy : ctx->dd.cl_energy;
    CK(cudaMemcpyAsync(h.data(), src, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int c = 0; c < nc; ++c) {
        const double *v = h.data() + (size_t)c * (NTERM + 1);
        sibfa_energy_terms &e = terms[c];
        e.elec = v[T_ELEC]; e.pen = v[T_PEN]; e.rep = v[T_REP]; e.disp = v[T_DISP];
        e.xdisp = v[T_XDISP]; e.pol = v[T_POL]; e.ct = v[T_CT]; e.total = v[NTERM];
    }
    return SIBFA_OK;
}

sibfa_status sibfa_last_stats(const sibfa_ctx *ctx, int *pcg_iters, double *pcg_resid_D) {
    if (!ctx) return SIBFA_E_INVALID;
    if (pcg_iters) *pcg_iters = ctx->last_iters;
    if (pcg_resid_D) *pcg_resid_D = ctx->last_resid;
    return SIBFA_OK;
}

void sibfa_set_profiling(sibfa_ctx *ctx, int on) {
    if (!ctx) return;
    ctx->profiling = on != 0;
    ctx->serial = on == 2;
}

/* Sum of the recorded phase durations (ms) and their count for `name`; the
 * spans are consumed (their events return to the pool).  Synchronizes the
 * context stream. */
sibfa_status sibfa_profile_get(sibfa_ctx *ctx, const char *name, double *ms, int *count) {
    if (!ctx || !name) return SIBFA_E_INVALID;
    if (cudaStreamSynchronize(ctx->s) != cudaSuccess) return SIBFA_E_CUDA;
    double tot = 0;
    int n = 0;
    std::vector<sibfa_ctx::Span> keep;
    for (auto &s : ctx->spans) {
        if (s.name == name) {
            float t = 0;
            cudaEventElapsedTime(&t, s.a, s.b);
            tot += t;
            ++n;
            ctx->event_pool.push_back(s.a);
            ctx->event_pool.push_back(s.b);
        } else {
            keep.push_back(s);
        }
    }
    ctx->spans.swap(keep);
    if (ms) *ms = tot;
    if (count) *count = n;
    return SIBFA_OK;
}

void sibfa_profile_clear(sibfa_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->s);
    for (auto &s : ctx->spans) {
        ctx->event_pool.push_back(s.a);
        ctx->event_pool.push_back(s.b);
    }
    ctx->spans.clear();
}

uint64_t sibfa_kernel_launches(const sibfa_ctx *ctx) { return ctx ? ctx->launches : 0; }

sibfa_status sibfa_tuned_shape(const sibfa_ctx *ctx, int *blocks_per_sm, int *done) {
    if (!ctx) return SIBFA_E_INVALID;
    if (blocks_per_sm) *blocks_per_sm = short_cap(ctx);
    if (done) *done = (!ctx->tune.on || ctx->tune.choice >= 0) ? 1 : 0;
    return SIBFA_OK;
}

sibfa_status sibfa_tuned_schedule(const sibfa_ctx *ctx, int *blocks_per_sm, int *join_before_solve, int *done,
                                  double *cand_ms, int n_cand) {
    if (!ctx || n_cand < 0) return SIBFA_E_INVALID;
    const ShortSched s = short_sched(ctx);
    if (blocks_per_sm) *blocks_per_sm = s.cap;
    if (join_before_solve) *join_before_solve = s.join_before_solve ? 1 : 0;
    if (done) *done = (!ctx->tune.on || ctx->tune.choice >= 0) ? 1 : 0;
    if (cand_ms)
        for (int c = 0; c < n_cand; ++c)
            cand_ms[c] = (c < kNSched && ctx->tune.tmin[c] < 1e29f) ? (double)ctx->tune.tmin[c] : 0.0;
    return SIBFA_OK;
}

void sibfa_destroy(sibfa_ctx *ctx) {
    if (!ctx) return;
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    if (ctx->s2) cudaStreamSynchronize(ctx->s2);
    if (ctx->s3) cudaStreamSynchronize(ctx->s3);
    if (ctx->s4) cudaStreamSynchronize(ctx->s4);
    if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
    if (ctx->ev_fork4) cudaEventDestroy(ctx->ev_fork4);
    if (ctx->tune.e0) cudaEventDestroy(ctx->tune.e0);
    if (ctx->tune.e1) cudaEventDestroy(ctx->tune.e1);
    if (ctx->ev_join4) cudaEventDestroy(ctx->ev_join4);
    if (ctx->ev_fork3) cudaEventDestroy(ctx->ev_fork3);
    if (ctx->ev_join3) cudaEventDestroy(ctx->ev_join3);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    else cudaDeviceSynchronize();
    if (ctx->have_fft) {
        cufftDestroy(ctx->r2c1);
        cufftDestroy(ctx->c2r1);
        cufftDestroy(ctx->r2c2);
        cufftDestroy(ctx->c2r2);
    }
    for (auto &s : ctx->spans) {
        cudaEventDestroy(s.a);
        cudaEventDestroy(s.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->s) cudaStreamDestroy(ctx->s);
    if (ctx->s2) cudaStreamDestroy(ctx->s2);
    if (ctx->s3) cudaStreamDestroy(ctx->s3);
    if (ctx->s4) cudaStreamDestroy(ctx->s4);
    delete ctx;
}

const char *sibfa_last_error(const sibfa_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Hooks for the request server (server.cu): regrouping a gas-phase batch
// context in place and reading its device arrays.
// ---------------------------------------------------------------------------
namespace sibfa {

template <typename R>
static sibfa_status set_batch_impl(sibfa_ctx *ctx, int M, int n_cl, const int *cluster_start) {
    DevState<R> &d = state<R>(ctx);
    std::vector<int> start(n_cl + 1), of(M);
    for (int c = 0; c <= n_cl; ++c) start[c] = cluster_start[c];
    for (int c = 0; c < n_cl; ++c)
        for (int m = start[c]; m < start[c + 1]; ++m) of[m] = c;
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaMemcpyAsync(d.cl_start, start.data(), (n_cl + 1) * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(d.cl_of, of.data(), M * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));   // the host vectors are freed on return
    return SIBFA_OK;
}

sibfa_status ctx_set_batch(sibfa_ctx *ctx, int M, int n_cl, const int *cluster_start) {
    if (!ctx || M < 1 || M > ctx->capacity || n_cl < 1 || n_cl > M || ctx->opts.periodic) return SIBFA_E_INVALID;
    if (cluster_start[0] != 0 || cluster_start[n_cl] != M) return SIBFA_E_INVALID;
    for (int c = 0; c < n_cl; ++c) {
        const int n = cluster_start[c + 1] - cluster_start[c];
        if (n < 1 || n > ctx->kp.tls / 3 + 1) return SIBFA_E_INVALID;
    }
    sibfa_status st = ctx->prec == SIBFA_PREC_MIXED ? set_batch_impl<float>(ctx, M, n_cl, cluster_start)
                                                     : set_batch_impl<double>(ctx, M, n_cl, cluster_start);
    if (st) return st;
    ctx->M = M;
    ctx->kp.M = M;
    ctx->kp.n_cl = n_cl;
    ctx->md_forces_valid = false;
    ctx->hist_n = 0;   // stored dipoles belong to the previous batch
    // the device-side PCG loop is captured for one size: drive the loop from the host
    if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
    ctx->pcg_exec = nullptr;
    ctx->pcg_graph_state = -1;
    return SIBFA_OK;
}

BatchArrays ctx_batch_arrays(sibfa_ctx *ctx) {
    BatchArrays b{};
    if (!ctx) return b;
    if (ctx->prec == SIBFA_PREC_MIXED) {
        b.mp_local = ctx->df.mp_local;
        b.mu = ctx->df.mu;
    } else {
        b.mp_local = ctx->dd.mp_local;
        b.mu = ctx->dd.mu;
    }
    b.forces = ctx->d_forces;
    b.capacity = ctx->capacity;
    return b;
}

cudaStream_t ctx_stream(sibfa_ctx *ctx) { return ctx ? ctx->s : nullptr; }
size_t ctx_device_bytes(const sibfa_ctx *ctx) { return ctx ? ctx->dev_bytes : 0; }

}  // namespace sibfa
