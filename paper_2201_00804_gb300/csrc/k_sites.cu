// Sites and frames (multipoles rotated from the molecular local frames to the
// global frame each step, section "Multipolar Electrostatics"; explicit
// lone-pair extra centres, section "Exchange-Repulsion"), the molecular cell
// list and the full neighbour list.
#include "sibfa_internal.cuh"

namespace sibfa {

// Orthonormal frame with z along zv and x in the (z, xv) plane; y = z x x.
__device__ inline void frame_d(V3<double> zv, V3<double> xv, V3<double> &ex, V3<double> &ey, V3<double> &ez) {
    ez = (1.0 / sqrt(dot(zv, zv))) * zv;
    V3<double> xp = xv - dot(xv, ez) * ez;
    ex = (1.0 / sqrt(dot(xp, xp))) * xp;
    ey = cross(ez, ex);
}

template <typename R>
__global__ void k_sites(KParams p, DevState<R> d) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    const double *x = d.pos + m * 9;
    V3<double> O = mk(x[0], x[1], x[2]), H1 = mk(x[3], x[4], x[5]), H2 = mk(x[6], x[7], x[8]);
    V3<double> r1 = H1 - O, r2 = H2 - O;
    V3<double> u1 = (1.0 / sqrt(dot(r1, r1))) * r1, u2 = (1.0 / sqrt(dot(r2, r2))) * r2;
    V3<double> F[3][3];  // frames: [frame][axis]
    frame_d(u1 + u2, r1, F[0][0], F[0][1], F[0][2]);
    frame_d(O - H1, H2 - H1, F[1][0], F[1][1], F[1][2]);
    frame_d(O - H2, H1 - H2, F[2][0], F[2][1], F[2][2]);
    const int fr_of[5] = {0, 1, 2, 1, 2};
    V3<double> offs[NP];
    offs[0] = mk(0.0, 0.0, 0.0);
    offs[1] = r1;
    offs[2] = r2;
    offs[3] = 0.5 * r1;
    offs[4] = 0.5 * r2;
    offs[5] = p.d_lp * ((-p.lp_cos) * F[0][2] + p.lp_sin * F[0][1]);
    offs[6] = p.d_lp * ((-p.lp_cos) * F[0][2] - p.lp_sin * F[0][1]);
    float ext = 0.f;
    for (int k = 0; k < NP; ++k) {
        d.off[(m * NP + k) * 3 + 0] = R(offs[k].x);
        d.off[(m * NP + k) * 3 + 1] = R(offs[k].y);
        d.off[(m * NP + k) * 3 + 2] = R(offs[k].z);
        ext = fmaxf(ext, (float)sqrt(dot(offs[k], offs[k])));
    }
    atomicMax((int *)d.ext, __float_as_int(ext));
    // O wrapped into the box in single precision (candidate tests of the list build)
    for (int k = 0; k < 3; ++k) {
        double v = x[k];
        if (p.periodic) v -= p.box[k] * floor(v / p.box[k]);
        d.ofw[m * 3 + k] = (float)v;
    }
    const double *ml = d.mp_local + m * NS * NMP;
    double qs[NS];
    for (int s = 0; s < NS; ++s) {
        const double *l = ml + s * NMP;
        const V3<double> *e = F[fr_of[s]];
        V3<double> mu = l[1] * e[0] + l[2] * e[1] + l[3] * e[2];
        // Theta = R Th_l R^T ; Th_l symmetric (xx yy zz xy xz yz)
        double tl[3][3] = {{l[4], l[7], l[8]}, {l[7], l[5], l[9]}, {l[8], l[9], l[6]}};
        double Rm[3][3] = {{e[0].x, e[1].x, e[2].x}, {e[0].y, e[1].y, e[2].y}, {e[0].z, e[1].z, e[2].z}};
        double A[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int c = 0; c < 3; ++c) acc += Rm[a][c] * tl[c][b];
                A[a][b] = acc;
            }
        double T[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int c = 0; c < 3; ++c) acc += A[a][c] * Rm[b][c];
                T[a][b] = acc;
            }
        R *g = d.gmp + (m * NS + s) * NMP;
        g[0] = R(l[0]);
        g[1] = R(mu.x);
        g[2] = R(mu.y);
        g[3] = R(mu.z);
        g[4] = R(T[0][0]);
        g[5] = R(T[1][1]);
        g[6] = R(T[2][2]);
        g[7] = R(T[0][1]);
        g[8] = R(T[0][2]);
        g[9] = R(T[1][2]);
        qs[s] = l[0];
    }
    // intramolecular potential on O, H1, H2 from the charges of the other sites
    for (int a = 0; a < 3; ++a) {
        double v = 0;
        for (int s = 0; s < NS; ++s) {
            if (s == a) continue;
            V3<double> dd = offs[a] - offs[s];
            v += qs[s] / sqrt(dot(dd, dd));
        }
        d.vint[m * 3 + a] = p.ke * v;
    }
    // clear the per-molecule accumulators of this evaluation
    for (int k = 0; k < NP * 3; ++k) d.gpt[m * NP * 3 + k] = 0.0;
    for (int k = 0; k < NS * 3; ++k) d.gmu[m * NS * 3 + k] = 0.0;
    for (int k = 0; k < NS * 6; ++k) d.gth[m * NS * 6 + k] = 0.0;
    for (int k = 0; k < 9; ++k) d.efield[m * 9 + k] = 0.0;
    for (int k = 0; k < 18; ++k) d.d2rec[m * 18 + k] = 0.0;
    for (int k = 0; k < 2; ++k) d.vlp[m * 2 + k] = 0.0, d.lam[m * 2 + k] = 0.0;
    for (int k = 0; k < 6; ++k) d.dvlp[m * 6 + k] = 0.0;
    for (int k = 0; k < 3; ++k) d.kap[m * 3 + k] = 0.0;
    for (int k = 0; k < NTERM; ++k) d.epart[m * NTERM + k] = 0.0;
}

template <typename R>
void launch_sites(const KParams &p, DevState<R> &d, Launch L) {
    cudaMemsetAsync(d.ext, 0, sizeof(float), L.s);
    k_sites<R><<<(p.M + 127) / 128, 128, 0, L.s>>>(p, d);
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

template <typename R>
__global__ void k_check_ext(KParams p, DevState<R> d) {
    if (!p.periodic) return;
    double cut = list_cut(p, d.ext);
    double half = 0.5 * fmin(p.box[0], fmin(p.box[1], p.box[2]));
    if (cut > half || *d.ext > 1.3f) atomicOr(d.flags, F_CUTOFF);
}

// FP32 candidate test on wrapped O positions
template <typename R>
__device__ inline bool near_f(const KParams &p, const DevState<R> &d, int i, int j, float cut2f) {
    float dx = d.ofw[j * 3] - d.ofw[i * 3], dy = d.ofw[j * 3 + 1] - d.ofw[i * 3 + 1], dz = d.ofw[j * 3 + 2] - d.ofw[i * 3 + 2];
    if (p.periodic) {
        const float L0 = (float)p.box[0], L1 = (float)p.box[1], L2 = (float)p.box[2];
        dx -= L0 * rintf(dx / L0);
        dy -= L1 * rintf(dy / L1);
        dz -= L2 * rintf(dz / L2);
    }
    return dx * dx + dy * dy + dz * dz < cut2f;
}

template <typename R>
__device__ inline void store_entry(const KParams &p, DevState<R> &d, int i, int slot, int j) {
    if (slot >= MAXN) return;
    double dx, dy, dz;
    min_image(p, d.pos, i, j, dx, dy, dz);
    d.nbr[i * MAXN + slot] = j;
    R *o = d.ndo + ((size_t)i * MAXN + slot) * 3;
    o[0] = R(dx);
    o[1] = R(dy);
    o[2] = R(dz);
}

template <typename R>
__global__ void k_nbr_all(KParams p, DevState<R> d) {
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= p.M) return;
    const double cut = list_cut(p, d.ext) + 1e-3;
    const float cut2f = p.periodic ? (float)(cut * cut) : 3.0e38f;
    int n = 0;
    for (int j0 = 0; j0 < p.M; j0 += 32) {
        const int j = j0 + lane;
        const bool ok = (j < p.M && j != i) && near_f(p, d, i, j, cut2f);
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
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    const int nc[3] = {nc0, nc1, nc2};
    const int c = cell_index(p, nc, d.ofw[m * 3], d.ofw[m * 3 + 1], d.ofw[m * 3 + 2]);
    d.cell_of[m] = c;
    atomicAdd(&d.cell_cursor[c], 1);
}

// exclusive scan of the cell counts (one block)
template <typename R>
__global__ void k_cell_scan(DevState<R> d, int ncell) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (ncell + blockDim.x - 1) / blockDim.x;
    const int a = t * per, b = min(ncell, a + per);
    int s = 0;
    for (int k = a; k < b; ++k) s += d.cell_cursor[k];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            int v = part[k];
            part[k] = acc;
            acc += v;
        }
        d.cell_start[ncell] = acc;
    }
    __syncthreads();
    int acc = part[t];
    for (int k = a; k < b; ++k) {
        int v = d.cell_cursor[k];
        d.cell_start[k] = acc;
        acc += v;
        d.cell_cursor[k] = 0;
    }
}

template <typename R>
__global__ void k_cell_fill(KParams p, DevState<R> d) {
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
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= p.M) return;
    const double cut = list_cut(p, d.ext) + 1e-3;
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
    count(L);
    const int wpb = 4;
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
