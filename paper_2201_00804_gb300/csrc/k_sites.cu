// Sites and frames (multipoles rotated from the molecular local frames to the
// global frame each step, section "Multipolar Electrostatics"; explicit
// lone-pair extra centres, section "Exchange-Repulsion"), the molecular cell
// list and the full neighbour list.
#include "sibfa_internal.cuh"

namespace sibfa {

// Eight lanes per molecule.  Lane t < 7 owns point t (offset from O, SPME
// grid coordinates) and builds the one local frame it needs (points 5 and 6,
// the lone pairs, hang on frame 0); lane t < 5 rotates the multipoles of site
// t into the global frame; lane t < 3 forms V_int of atom t; lane 7 wraps O;
// the lanes share the clearing of the per-molecule accumulators.  Geometry
// and rotation in the working precision R (the results are stored in R);
// the SPME grid coordinates and the wrap in FP64.
template <typename R>
__global__ void __launch_bounds__(128) k_sites(KParams p, DevState<R> d) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = g >> 3, t = g & 7;
    const bool live = m < p.M;
    float ext = 0.f;
    // bond vectors r1 = H1 - O, r2 = H2 - O: lane t < 6 takes one FP64
    // difference (rounded once to R) and the molecule's 8 lanes share them
    R bc = R(0);
    if (live && t < 6) {
        const double *x = d.pos + m * 9;
        bc = R(x[3 + t] - x[t % 3]);
    }
    V3<R> r1, r2;
    r1.x = __shfl_sync(0xffffffffu, bc, 0, 8);
    r1.y = __shfl_sync(0xffffffffu, bc, 1, 8);
    r1.z = __shfl_sync(0xffffffffu, bc, 2, 8);
    r2.x = __shfl_sync(0xffffffffu, bc, 3, 8);
    r2.y = __shfl_sync(0xffffffffu, bc, 4, 8);
    r2.z = __shfl_sync(0xffffffffu, bc, 5, 8);
    if (live) {
        const double *x = d.pos + m * 9;
        const R s1 = rsqrt_<R>(dot(r1, r1)), s2 = rsqrt_<R>(dot(r2, r2));
        const int f = t < NS ? site_frame(t) : 0;
        V3<R> zv, xv, ex, ey, ez;
        frame_generators(f, r1, r2, s1, s2, zv, xv);
        frame_axes(zv, xv, ex, ey, ez);
        const R hz = R(-p.d_lp * p.lp_cos), hy = R(p.d_lp * p.lp_sin);
        // offsets of the sites O, H1, H2, M1, M2 (needed by every V_int lane)
        const V3<R> so[NS] = {mk(R(0), R(0), R(0)), r1, r2, R(0.5) * r1, R(0.5) * r2};
        const double *ml = d.mp_local + m * NS * NMP;
        if (t < NP) {
            V3<R> o = hz * ez + (t == 5 ? hy : -hy) * ey;
#pragma unroll
            for (int k = 0; k < NS; ++k)
                if (k == t) o = so[k];
            d.off[(m * NP + t) * 3 + 0] = o.x;
            d.off[(m * NP + t) * 3 + 1] = o.y;
            d.off[(m * NP + t) * 3 + 2] = o.z;
            ext = (float)sqrt_<R>(dot(o, o));
            // SPME grid coordinates of the point, from the FP64 O position
            // and the stored offset (the spread and gather kernels build their
            // B-spline weights from the fraction)
            if (p.periodic) {
                const double pk[3] = {x[0] + (double)o.x, x[1] + (double)o.y, x[2] + (double)o.z};
                for (int c = 0; c < 3; ++c) {
                    const double u = pk[c] * p.ibox[c] * (double)p.K[c];
                    const double fl = floor(u);
                    int b = (int)fl % p.K[c];
                    if (b < 0) b += p.K[c];
                    d.sbase[(m * NP + t) * 3 + c] = b;
                    d.sfrac[(m * NP + t) * 3 + c] = R(u - fl);
                }
            }
        }
        if (t < NS) {
            const double *l = ml + t * NMP;
            const R q = R(l[0]), m1 = R(l[1]), m2 = R(l[2]), m3 = R(l[3]);
            const V3<R> mu = m1 * ex + m2 * ey + m3 * ez;
            // Theta = Rm Th_l Rm^T; Th_l symmetric (xx yy zz xy xz yz), Rm columns = frame axes
            const R tl[3][3] = {{R(l[4]), R(l[7]), R(l[8])}, {R(l[7]), R(l[5]), R(l[9])}, {R(l[8]), R(l[9]), R(l[6])}};
            const V3<R> e[3] = {ex, ey, ez};
            // A_k = sum_c Th_l[k][c] e_c (column k of Rm Th_l); Theta = sum_k e_k A_k^T
            V3<R> A[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) A[k] = tl[k][0] * e[0] + tl[k][1] * e[1] + tl[k][2] * e[2];
            R T[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T[0] += e[k].x * A[k].x;
                T[1] += e[k].y * A[k].y;
                T[2] += e[k].z * A[k].z;
                T[3] += e[k].x * A[k].y;
                T[4] += e[k].x * A[k].z;
                T[5] += e[k].y * A[k].z;
            }
            R *gm = d.gmp + (m * NS + t) * GMP;
            gm[0] = q;
            gm[1] = mu.x;
            gm[2] = mu.y;
            gm[3] = mu.z;
#pragma unroll
            for (int k = 0; k < 6; ++k) gm[4 + k] = T[k];
            gm[10] = R(0);
            gm[11] = R(0);
        }
        if (t < 3) {
            // intramolecular potential on atom t from the charges of the other sites
            V3<R> ot = so[0];
#pragma unroll
            for (int k = 1; k < 3; ++k)
                if (k == t) ot = so[k];
            R v = R(0);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (s == t) continue;
                const V3<R> dd = ot - so[s];
                v += R(ml[s * NMP]) * rsqrt_<R>(dot(dd, dd));
            }
            d.vint[m * 3 + t] = p.ke * (double)v;
        }
        if (t == 7) {
            // O wrapped into the box in single precision (cell binning) and as
            // 32-bit fixed-point fractional coordinates: the difference of two
            // of those, read as a signed integer, is the minimum-image
            // displacement in units of box / 2^32.
            for (int k = 0; k < 3; ++k) {
                double v = x[k];
                if (p.periodic) {
                    const double f = v * p.ibox[k];
                    const double fr = f - floor(f);
                    d.ufx[m * 3 + k] = (unsigned)(long long)(fr * 4294967296.0);   // fr -> 1 wraps to 0
                    v = fr * p.box[k];
                }
                d.ofw[m * 3 + k] = (float)v;
            }
        }
        // clear the per-molecule accumulators of this evaluation
        for (int k = t; k < NP * 3; k += 8)
            d.gpt[m * NP * 3 + k] = 0.0, d.gpt_r[m * NP * 3 + k] = 0.0, d.gpt_s[m * NP * 3 + k] = 0.0;
        for (int k = t; k < NS * 3; k += 8) d.gmu[m * NS * 3 + k] = 0.0, d.gmu_r[m * NS * 3 + k] = 0.0;
        for (int k = t; k < NS * 6; k += 8) d.gth[m * NS * 6 + k] = 0.0, d.gth_r[m * NS * 6 + k] = 0.0;
        for (int k = t; k < 9; k += 8) d.efield[m * 9 + k] = 0.0, d.efield_r[m * 9 + k] = 0.0;
        for (int k = t; k < 18; k += 8) d.d2rec[m * 18 + k] = 0.0;
        if (t < 2) d.vlp[m * 2 + t] = 0.0, d.vlp_r[m * 2 + t] = 0.0, d.lam[m * 2 + t] = 0.0;
        if (t < 6) d.dvlp[m * 6 + t] = 0.0, d.dvlp_r[m * 6 + t] = 0.0;
        if (t < 3) d.kap[m * 3 + t] = 0.0;
        if (p.ct_orig) {
            if (t < 3) d.va[m * 3 + t] = 0.0, d.va_r[m * 3 + t] = 0.0, d.lama[m * 3 + t] = 0.0;
            for (int k = t; k < 9; k += 8) d.dva[m * 9 + k] = 0.0, d.dva_r[m * 9 + k] = 0.0;
        }
        if (t < NTERM) d.epart[m * NTERM + t] = 0.0, d.epart_r[m * NTERM + t] = 0.0;
        if (p.vir)
            for (int k = t; k < 9; k += 8) d.vir[m * 9 + k] = 0.0, d.vir_r[m * 9 + k] = 0.0;
    }
    // largest point distance from its O (list margin): one atomic per warp
    const int e = __reduce_max_sync(0xffffffffu, __float_as_int(ext));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)d.ext, e);
}

template <typename R>
void launch_sites(const KParams &p, DevState<R> &d, Launch L) {
    cudaMemsetAsync(d.ext, 0, sizeof(float), L.s);
    const long long n = (long long)p.M * 8;
    k_sites<R><<<(unsigned)((n + 127) / 128), 128, 0, L.s>>>(p, d);
    count(L);
}

// ---------------------------------------------------------------------------
// Neighbour list: molecule pairs whose O-O distance (minimum image) is below
// rc + 2 * ext, ext = largest point distance from its own O this step.  The
// list is full (both orders), ordered by cell and molecule index, so every
// pair sum over it has a fixed order.  Each entry stores the minimum-image
// displacement O_j - O_i (computed in FP64, stored in R), so the pair
// kernels do no FP64 work.  Candidates are tested in FP32 with a small
// margin; only accepted pairs pay the FP64 displacement.
// ---------------------------------------------------------------------------
__device__ inline double list_cut(const KParams &p, const float *ext) {
    return p.periodic ? p.rc + 2.0 * (double)(*ext) : 1e300;
}
// the radius of a build: rc + 2 ext + the skin chosen at that build
template <typename R>
__device__ inline double build_cut(const KParams &p, const DevState<R> &d) {
    return p.periodic ? p.rc + 2.0 * (double)d.lst[0] + (double)d.lst[1] : 1e300;
}

// Verlet skin (periodic systems).  The largest O displacement since the last
// build (squared, as float bits: non-negative floats order like their bits).
template <typename R>
__global__ void k_skin_disp(KParams p, DevState<R> d) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double v = d.pos[m * 9 + k] - d.oref[m * 3 + k];
        d2 += v * v;
    }
    atomicMax((int *)(d.lst + 2), __float_as_int((float)fmin(d2, 1e30)));
}
// Rebuild when no list exists yet, when the skin is zero, or when twice the
// largest move plus twice the growth of the site extent reaches the skin (a
// pair can then have come from outside the listed radius to inside rc +
// 2 ext).  A rebuild takes the current extent and the largest skin that keeps
// the list radius below half the box (minimum image).
template <typename R>
__global__ void k_skin_decide(KParams p, DevState<R> d) {
    const float ext = *d.ext;
    const float md = sqrtf(__int_as_float(*(const int *)(d.lst + 2)));
    const bool rebuild = d.lflag[1] == 0 || d.lst[1] <= 0.f || 2.f * md + 2.f * fmaxf(0.f, ext - d.lst[0]) >= d.lst[1];
    if (rebuild) {
        const double half = 0.5 * fmin(p.box[0], fmin(p.box[1], p.box[2]));
        d.lst[0] = ext;
        d.lst[1] = (float)fmax(0.0, fmin(p.skin, half - p.rc - 2.0 * (double)ext - 1e-3));
        d.lflag[1] = 1;
    }
    d.lflag[0] = rebuild ? 1 : 0;
    *(int *)(d.lst + 2) = 0;
}


template <typename R>
__global__ void k_check_ext(KParams p, DevState<R> d) {
    if (!p.periodic) return;
    double cut = list_cut(p, d.ext);
    double half = 0.5 * fmin(p.box[0], fmin(p.box[1], p.box[2]));
    if (cut > half || *d.ext > 1.3f) atomicOr(d.flags, F_CUTOFF);
}

// Minimum-image O_j - O_i from the fixed-point fractional coordinates (FP32).
template <typename R>
__device__ inline V3<float> fx_disp(const KParams &p, const DevState<R> &d, int i, int j) {
    const int ax = (int)(d.ufx[j * 3] - d.ufx[i * 3]);
    const int ay = (int)(d.ufx[j * 3 + 1] - d.ufx[i * 3 + 1]);
    const int az = (int)(d.ufx[j * 3 + 2] - d.ufx[i * 3 + 2]);
    return mk((float)ax * p.fxs[0], (float)ay * p.fxs[1], (float)az * p.fxs[2]);
}

// FP32 candidate test
template <typename R>
__device__ inline bool near_f(const KParams &p, const DevState<R> &d, int i, int j, float cut2f) {
    if (!p.periodic) {
        const float dx = d.ofw[j * 3] - d.ofw[i * 3], dy = d.ofw[j * 3 + 1] - d.ofw[i * 3 + 1],
                    dz = d.ofw[j * 3 + 2] - d.ofw[i * 3 + 2];
        return dx * dx + dy * dy + dz * dz < cut2f;
    }
    const V3<float> v = fx_disp(p, d, i, j);
    return dot(v, v) < cut2f;
}

// Stored displacement: FP32 path in a periodic box from the fixed-point
// coordinates (relative error ~1e-7, like rounding an exact value to FP32);
// otherwise the FP64 minimum image.
template <typename R>
__device__ inline void store_entry(const KParams &p, DevState<R> &d, int i, int slot, int j) {
    if (slot >= MAXN) return;
    d.nbr[i * MAXN + slot] = j;
    R *o = d.ndo + ((size_t)i * MAXN + slot) * 3;
    if (sizeof(R) == 4 && p.periodic) {
        const V3<float> v = fx_disp(p, d, i, j);
        o[0] = R(v.x);
        o[1] = R(v.y);
        o[2] = R(v.z);
        return;
    }
    double dx, dy, dz;
    min_image(p, d.pos, i, j, dx, dy, dz);
    o[0] = R(dx);
    o[1] = R(dy);
    o[2] = R(dz);
}

// Without a rebuild: the listed pairs' displacements at the current positions.
template <typename R>
__global__ void k_nbr_refresh(KParams p, DevState<R> d) {
    if (d.lflag[0]) return;
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= p.M) return;
    const int nn = d.nnbr[i];
    for (int slot = lane; slot < nn; slot += 32) store_entry(p, d, i, slot, d.nbr[i * MAXN + slot]);
}

template <typename R>
__global__ void k_nbr_all(KParams p, DevState<R> d) {
    if (!d.lflag[0]) return;
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= p.M) return;
    if (lane < 3) d.oref[i * 3 + lane] = d.pos[i * 9 + lane];
    const double cut = build_cut(p, d) + 1e-3;
    const float cut2f = p.periodic ? (float)(cut * cut) : 3.0e38f;
    // partners: the molecules of i's own cluster (the whole system when n_cl = 1)
    const int c = d.cl_of[i], j_lo = d.cl_start[c], j_hi = d.cl_start[c + 1];
    int n = 0;
    for (int j0 = j_lo; j0 < j_hi; j0 += 32) {
        const int j = j0 + lane;
        const bool ok = (j < j_hi && j != i) && near_f(p, d, i, j, cut2f);
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (ok) store_entry(p, d, i, n + __popc(b & ((1u << lane) - 1u)), j);
        n += __popc(b);
    }
    if (lane == 0) {
        d.nnbr[i] = min(n, MAXN);
        if (n > MAXN) atomicOr(d.flags, F_NEIGHBOR);
    }
}

__device__ inline int cell_index(const KParams &p, const int nc[3], float x, float y, float z) {
    const float f[3] = {x / (float)p.box[0], y / (float)p.box[1], z / (float)p.box[2]};
    int c[3];
    for (int k = 0; k < 3; ++k) {
        int ci = (int)(f[k] * nc[k]);
        c[k] = min(max(ci, 0), nc[k] - 1);
    }
    return (c[0] * nc[1] + c[1]) * nc[2] + c[2];
}

template <typename R>
__global__ void k_cell_count(KParams p, DevState<R> d, int nc0, int nc1, int nc2) {
    if (!d.lflag[0]) return;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    const int nc[3] = {nc0, nc1, nc2};
    const int c = cell_index(p, nc, d.ofw[m * 3], d.ofw[m * 3 + 1], d.ofw[m * 3 + 2]);
    d.cell_of[m] = c;
    atomicAdd(&d.cell_cursor[c], 1);
}

// exclusive scan of the cell counts (one block of 1024 threads): every thread
// sums a contiguous chunk, the chunk sums are scanned with warp shuffles and
// one pass over the warp totals, and each thread writes its chunk's starts
template <typename R>
__global__ void __launch_bounds__(1024) k_cell_scan(DevState<R> d, int ncell) {
    __shared__ int wsum[32];
    if (!d.lflag[0]) return;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (ncell + blockDim.x - 1) / blockDim.x;
    const int a = t * per, b = min(ncell, a + per);
    int s = 0;
    for (int k = a; k < b; ++k) s += d.cell_cursor[k];
    int incl = s;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = (int)(blockDim.x >> 5);
        int v = lane < nw ? wsum[lane] : 0, iv = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, iv, o);
            if (lane >= o) iv += u;
        }
        if (lane < nw) wsum[lane] = iv - v;   // exclusive warp offsets
        if (lane == nw - 1) d.cell_start[ncell] = iv;
    }
    __syncthreads();
    int acc = wsum[w] + incl - s;
    for (int k = a; k < b; ++k) {
        const int v = d.cell_cursor[k];
        d.cell_start[k] = acc;
        acc += v;
        d.cell_cursor[k] = 0;
    }
}

template <typename R>
__global__ void k_cell_fill(KParams p, DevState<R> d) {
    if (!d.lflag[0]) return;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    int c = d.cell_of[m];
    int k = atomicAdd(&d.cell_cursor[c], 1);
    d.cell_mol[d.cell_start[c] + k] = m;
}

// Order the members of every cell by molecule index: one warp per cell, each
// member's rank is the number of smaller members (indices are distinct).
constexpr int SORT_CAP = 256;
template <typename R>
__global__ void k_cell_sort(DevState<R> d, int ncell) {
    __shared__ int buf[4][SORT_CAP];
    if (!d.lflag[0]) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + w;
    if (c >= ncell) return;
    const int a = d.cell_start[c], n = d.cell_start[c + 1] - a;
    if (n <= SORT_CAP) {
        for (int k = lane; k < n; k += 32) buf[w][k] = d.cell_mol[a + k];
        __syncwarp();
        for (int k = lane; k < n; k += 32) {
            const int v = buf[w][k];
            int r = 0;
            for (int q = 0; q < n; ++q) r += buf[w][q] < v;
            d.cell_mol[a + r] = v;
        }
    } else if (lane == 0) {
        for (int k = a + 1; k < a + n; ++k) {
            int v = d.cell_mol[k], j = k - 1;
            while (j >= a && d.cell_mol[j] > v) {
                d.cell_mol[j + 1] = d.cell_mol[j];
                --j;
            }
            d.cell_mol[j + 1] = v;
        }
    }
}

template <typename R>
__global__ void k_nbr_cell(KParams p, DevState<R> d, int nc0, int nc1, int nc2) {
    if (!d.lflag[0]) return;
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= p.M) return;
    if (lane < 3) d.oref[i * 3 + lane] = d.pos[i * 9 + lane];
    const double cut = build_cut(p, d) + 1e-3;
    const float cut2f = (float)(cut * cut);
    const int ci = d.cell_of[i];
    const int cz = ci % nc2, cy = (ci / nc2) % nc1, cx = ci / (nc1 * nc2);
    int n = 0;
    for (int o = 0; o < 27; ++o) {
        const int ox = o / 9 - 1, oy = (o / 3) % 3 - 1, oz = o % 3 - 1;
        const int c = (((cx + ox + nc0) % nc0) * nc1 + (cy + oy + nc1) % nc1) * nc2 + (cz + oz + nc2) % nc2;
        const int a = d.cell_start[c], b = d.cell_start[c + 1];
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            int j = -1;
            bool ok = false;
            if (k < b) {
                j = d.cell_mol[k];
                ok = (j != i) && near_f(p, d, i, j, cut2f);
            }
            const unsigned bl = __ballot_sync(0xffffffffu, ok);
            if (ok) store_entry(p, d, i, n + __popc(bl & ((1u << lane) - 1u)), j);
            n += __popc(bl);
        }
    }
    if (lane == 0) {
        d.nnbr[i] = min(n, MAXN);
        if (n > MAXN) atomicOr(d.flags, F_NEIGHBOR);
    }
}

template <typename R>
void launch_neighbors(const KParams &p, DevState<R> &d, int nc[3], Launch L) {
    k_check_ext<R><<<1, 1, 0, L.s>>>(p, d);
    k_skin_disp<R><<<(p.M + 255) / 256, 256, 0, L.s>>>(p, d);
    k_skin_decide<R><<<1, 1, 0, L.s>>>(p, d);
    count(L, 3);
    const int wpb = 4;
    // either the refresh or the build kernels do work, as the decision says
    k_nbr_refresh<R><<<(p.M + wpb - 1) / wpb, 32 * wpb, 0, L.s>>>(p, d);
    count(L);
    if (!p.periodic || nc[0] < 3 || nc[1] < 3 || nc[2] < 3) {
        k_nbr_all<R><<<(p.M + wpb - 1) / wpb, 32 * wpb, 0, L.s>>>(p, d);
        count(L);
        return;
    }
    const int ncell = nc[0] * nc[1] * nc[2];
    cudaMemsetAsync(d.cell_cursor, 0, sizeof(int) * ncell, L.s);
    k_cell_count<R><<<(p.M + 255) / 256, 256, 0, L.s>>>(p, d, nc[0], nc[1], nc[2]);
    k_cell_scan<R><<<1, 1024, 0, L.s>>>(d, ncell);
    k_cell_fill<R><<<(p.M + 255) / 256, 256, 0, L.s>>>(p, d);
    k_cell_sort<R><<<(ncell + 3) / 4, 128, 0, L.s>>>(d, ncell);
    k_nbr_cell<R><<<(p.M + wpb - 1) / wpb, 32 * wpb, 0, L.s>>>(p, d, nc[0], nc[1], nc[2]);
    count(L, 5);
}

template void launch_sites<float>(const KParams &, DevState<float> &, Launch);
template void launch_sites<double>(const KParams &, DevState<double> &, Launch);
template void launch_neighbors<float>(const KParams &, DevState<float> &, int *, Launch);
template void launch_neighbors<double>(const KParams &, DevState<double> &, int *, Launch);

}  // namespace sibfa
