// Allocation-free variant of the real-space permanent electrostatics kernel
// for gas-phase clusters (multipole energy and its penetration correction),
// for callers that may not allocate device memory.
//
// All scratch (rotated site offsets, global multipoles, per-molecule energy
// partials) lives in one file-scope __device__ array of fixed size, so the
// entry point calls no cudaMalloc, cudaFree or allocating library routine.
// Host code cannot use the array's name as a device address; the device
// address is looked up once per device with cudaGetSymbolAddress.
#include <cmath>
#include <mutex>
#include <string>

#include "sibfa_internal.cuh"

using namespace sibfa;

namespace {

constexpr int NA_MAX_MOL = 512;                  // largest cluster accepted
constexpr int NA_OFF = 0;                        // [mol][5][3] site offsets from O
constexpr int NA_GMP = NA_MAX_MOL * NS * 3;      // [mol][5][10] global multipoles
constexpr int NA_E = NA_GMP + NA_MAX_MOL * NS * NMP;   // [mol][2] elec, pen partials
constexpr int NA_SIZE = NA_E + NA_MAX_MOL * 2;   // doubles (about 270 KB)
constexpr int NA_MAX_DEV = 64;

// Scratch shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) double g_na_scratch[NA_SIZE];

std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEV] = {nullptr};
thread_local std::string g_na_error = "no error";

__device__ inline void na_frame(V3<double> zv, V3<double> xv, V3<double> &ex, V3<double> &ey, V3<double> &ez) {
    ez = (1.0 / sqrt(dot(zv, zv))) * zv;
    V3<double> xp = xv - dot(xv, ez) * ez;
    ex = (1.0 / sqrt(dot(xp, xp))) * xp;
    ey = cross(ez, ex);
}

// Site offsets and global multipoles of every molecule (FP64).
__global__ void k_na_sites(int M, const double *pos, const double *mp_local, double *scr) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double *x = pos + m * 9;
    const V3<double> O = mk(x[0], x[1], x[2]), H1 = mk(x[3], x[4], x[5]), H2 = mk(x[6], x[7], x[8]);
    const V3<double> r1 = H1 - O, r2 = H2 - O;
    const V3<double> u1 = (1.0 / sqrt(dot(r1, r1))) * r1, u2 = (1.0 / sqrt(dot(r2, r2))) * r2;
    V3<double> F[3][3];
    na_frame(u1 + u2, r1, F[0][0], F[0][1], F[0][2]);
    na_frame(O - H1, H2 - H1, F[1][0], F[1][1], F[1][2]);
    na_frame(O - H2, H1 - H2, F[2][0], F[2][1], F[2][2]);
    const int fr_of[NS] = {0, 1, 2, 1, 2};
    const V3<double> offs[NS] = {mk(0.0, 0.0, 0.0), r1, r2, 0.5 * r1, 0.5 * r2};
    for (int s = 0; s < NS; ++s) {
        double *o = scr + NA_OFF + (m * NS + s) * 3;
        o[0] = offs[s].x;
        o[1] = offs[s].y;
        o[2] = offs[s].z;
        const double *l = mp_local + (m * NS + s) * NMP;
        const V3<double> *e = F[fr_of[s]];
        const V3<double> mu = l[1] * e[0] + l[2] * e[1] + l[3] * e[2];
        const double tl[3][3] = {{l[4], l[7], l[8]}, {l[7], l[5], l[9]}, {l[8], l[9], l[6]}};
        const double R[3][3] = {{e[0].x, e[1].x, e[2].x}, {e[0].y, e[1].y, e[2].y}, {e[0].z, e[1].z, e[2].z}};
        double T[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) acc += R[a][c] * tl[c][d] * R[b][d];
                T[a][b] = acc;
            }
        double *g = scr + NA_GMP + (m * NS + s) * NMP;
        g[0] = l[0];
        g[1] = mu.x;
        g[2] = mu.y;
        g[3] = mu.z;
        g[4] = T[0][0];
        g[5] = T[1][1];
        g[6] = T[2][2];
        g[7] = T[0][1];
        g[8] = T[0][2];
        g[9] = T[1][2];
    }
}

// Multipole energy and penetration correction of molecule i with all other
// molecules (bare 1/r kernels, no cutoff): one warp per target site, lanes
// over the other molecules; half of every pair energy is credited to i.
__global__ void __launch_bounds__(160) k_na_elec(KParams p, int M, const double *pos, double *scr) {
    __shared__ double s_e[NS][2];
    const int i = blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double *ot_ = scr + NA_OFF + (i * NS + w) * 3;
    const V3<double> ot = mk(ot_[0], ot_[1], ot_[2]);
    const Mp<double> mt = load_mp(scr + NA_GMP + (i * NS + w) * NMP);
    const double Nt = (w < 3) ? p.z[w] - mt.q : 0.0;
    const double bt = (w < 3) ? p.b[w] : 0.0;
    double ue = 0.0, up = 0.0;
    for (int j = lane; j < M; j += 32) {
        if (j == i) continue;
        const V3<double> dO = mk(pos[j * 9] - pos[i * 9], pos[j * 9 + 1] - pos[i * 9 + 1], pos[j * 9 + 2] - pos[i * 9 + 2]);
        for (int s = 0; s < NS; ++s) {
            const double *os = scr + NA_OFF + (j * NS + s) * 3;
            const V3<double> x = ot - (dO + mk(os[0], os[1], os[2]));
            const double rinv = 1.0 / sqrt(dot(x, x));
            const double r = 1.0 / rinv;
            const Mp<double> ms = load_mp(scr + NA_GMP + (j * NS + s) * NMP);
            double g[6];
            g_bare<double, 5>(rinv, g);
            FieldTerms<double> f;
            source_field<double, 2>(ms, x, g, f);
            ue += 0.5 * (mt.q * f.phi + dot(mt.mu, f.d1) + symdd(mt.th, f.d2) / 3.0);
            const double Ns = (s < 3) ? p.z[s] - ms.q : 0.0;
            if (Nt == 0.0 && Ns == 0.0) continue;
            const double bs = (s < 3) ? p.b[s] : 0.0;
            double pen = (mt.q * Ns * exp(-bs * r) + ms.q * Nt * exp(-bt * r) + Nt * Ns * exp(-(bt + bs) * r)) * rinv;
            if (Nt != 0.0) {
                double ge[4];
                g_exp<double, 3>(r, rinv, bt, ge);
                Mp<double> m0 = ms;
                m0.q = 0.0;
                FieldTerms<double> f2;
                source_field<double, 0>(m0, x, ge, f2);
                pen += Nt * f2.phi;
            }
            if (Ns != 0.0) {
                double ge[4];
                g_exp<double, 3>(r, rinv, bs, ge);
                Mp<double> m0 = mt;
                m0.q = 0.0;
                FieldTerms<double> f3;
                source_field<double, 0>(m0, -x, ge, f3);
                pen += Ns * f3.phi;
            }
            up += 0.5 * pen;
        }
    }
    ue = warp_sum(ue);
    up = warp_sum(up);
    if (lane == 0) {
        s_e[w][0] = ue;
        s_e[w][1] = up;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int k = 0; k < NS; ++k) a += s_e[k][0], b += s_e[k][1];
        scr[NA_E + i * 2] = a;       // written, not accumulated: no clearing needed
        scr[NA_E + i * 2 + 1] = b;
    }
}

// out[0] = ke * sum elec partials, out[1] = ke * sum pen partials (fixed order)
__global__ void k_na_reduce(int M, double ke, const double *scr, double *out) {
    __shared__ double sh[2][256];
    double a = 0, b = 0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        a += scr[NA_E + m * 2];
        b += scr[NA_E + m * 2 + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ke * sh[0][0];
        out[1] = ke * sh[1][0];
    }
}

// The current device, or an error.
sibfa_status na_device(int *dev) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess || *dev < 0 || *dev >= NA_MAX_DEV) {
        g_na_error = std::string("sibfa_cluster_elec_noalloc: no usable current device: ") + cudaGetErrorString(e);
        return SIBFA_E_CUDA;
    }
    return SIBFA_OK;
}

// A caller buffer must be device (or managed) memory of the current device:
// a host address handed to the kernels would be read as a device address.
// cudaPointerGetAttributes allocates nothing.
sibfa_status na_check_ptr(const void *p, int dev, const char *name) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_na_error = std::string("sibfa_cluster_elec_noalloc: ") + name + " is not a CUDA pointer: " +
                     cudaGetErrorString(e);
        return SIBFA_E_INVALID;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        g_na_error = std::string("sibfa_cluster_elec_noalloc: ") + name + " must be device or managed memory";
        return SIBFA_E_INVALID;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev) {
        g_na_error = std::string("sibfa_cluster_elec_noalloc: ") + name + " lives on device " +
                     std::to_string(a.device) + ", not on the current device " + std::to_string(dev);
        return SIBFA_E_INVALID;
    }
    return SIBFA_OK;
}

// Device address of the scratch array on device `dev` (looked up once per
// device, with that device current, and kept until the process exits).
sibfa_status na_scratch(int dev, double **ptr) {
    cudaError_t e = cudaSuccess;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            g_na_error = std::string("sibfa_cluster_elec_noalloc: cudaGetSymbolAddress failed: ") +
                         cudaGetErrorString(e);
            return SIBFA_E_CUDA;
        }
        g_na_ptr[dev] = (double *)p;
    }
    *ptr = g_na_ptr[dev];
    return SIBFA_OK;
}

}  // namespace

extern "C" {

sibfa_status sibfa_cluster_elec_noalloc(const sibfa_params *params, int n_mol, const double *pos,
                                        const double *mp_local, double *elec_pen, void *stream) {
    if (!params || !pos || !mp_local || !elec_pen || n_mol < 1) {
        g_na_error = "sibfa_cluster_elec_noalloc: null pointer or n_mol < 1";
        return SIBFA_E_INVALID;
    }
    if (n_mol > NA_MAX_MOL) {
        g_na_error = "sibfa_cluster_elec_noalloc: n_mol " + std::to_string(n_mol) + " exceeds the maximum of " +
                     std::to_string(NA_MAX_MOL) + " molecules of the static scratch array";
        return SIBFA_E_INVALID;
    }
    int dev = 0;
    sibfa_status st = na_device(&dev);
    if (st) return st;
    if ((st = na_check_ptr(pos, dev, "pos")) || (st = na_check_ptr(mp_local, dev, "mp_local")) ||
        (st = na_check_ptr(elec_pen, dev, "elec_pen")))
        return st;
    double *scr = nullptr;
    if ((st = na_scratch(dev, &scr))) return st;
    KParams p{};
    p.z[0] = params->z_o;
    p.z[1] = p.z[2] = params->z_h;
    p.b[0] = params->b_o;
    p.b[1] = p.b[2] = params->b_h;
    cudaStream_t s = (cudaStream_t)stream;
    k_na_sites<<<(n_mol + 127) / 128, 128, 0, s>>>(n_mol, pos, mp_local, scr);
    k_na_elec<<<n_mol, 160, 0, s>>>(p, n_mol, pos, scr);
    k_na_reduce<<<1, 256, 0, s>>>(n_mol, params->ke, scr, elec_pen);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_na_error = std::string("sibfa_cluster_elec_noalloc: launch failed: ") + cudaGetErrorString(e);
        return SIBFA_E_CUDA;
    }
    return SIBFA_OK;
}

const char *sibfa_noalloc_last_error(void) { return g_na_error.c_str(); }

}  // extern "C"
