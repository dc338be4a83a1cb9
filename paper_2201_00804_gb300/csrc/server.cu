// Request server: energy/force jobs (MD runs of periodic water boxes and of
// gas-phase clusters) that arrive over time.
//
// * Box jobs run in `slots` worker threads, each with its own stream and up
//   to four contexts of distinct shapes kept for later jobs of those shapes
//   (positions, velocities and multipoles are replaced; the previous induced
//   dipoles serve as the first warm start); a slot prefers queued jobs of a
//   shape it holds.  Work of different slots overlaps on the device.
// * Gas-phase clusters are batched continuously: one resident batch context
//   (a cluster batch, see sibfa_topology) advances all admitted clusters by one
//   velocity-Verlet step per tick; jobs that reach their step count leave and
//   queued ones join at the next tick.  Leaving and joining regroup the batch
//   in place: one gather kernel per array moves the remaining molecules'
//   positions, velocities, multipoles and induced dipoles (their warm start).
// * Admission: a job starts when the device memory it needs (estimated from
//   its size) fits under the cap; the queue is bounded and sibfa_submit
//   returns SIBFA_E_BUSY when it is full.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "server_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr double MASS_O = 15.999, MASS_H = 1.008;

struct Job {
    uint64_t id = 0;
    sibfa_job spec{};
    std::vector<double> pos, vel, mp;
    int state = 0;          // 0 queued, 1 running, 2 done
    bool batch = false;     // runs in the cluster batch
    size_t mem = 0;         // estimated device bytes (slot jobs)
    int steps_done = 0;
    Clock::time_point t_submit, t_start, t_done;
    sibfa_energy_terms terms{};
    std::vector<double> forces, pos_out;
    int status = SIBFA_OK, iters = 0;
};

struct Shape {
    int n_mol = 0, periodic = 0, grid[3] = {0, 0, 0};
    double box[3] = {0, 0, 0}, rc = 0, alpha = 0;
    bool operator==(const Shape &o) const {
        return n_mol == o.n_mol && periodic == o.periodic && grid[0] == o.grid[0] && grid[1] == o.grid[1] &&
               grid[2] == o.grid[2] && box[0] == o.box[0] && box[1] == o.box[1] && box[2] == o.box[2] &&
               rc == o.rc && alpha == o.alpha;
    }
};

Shape shape_of(const sibfa_job &j) {
    Shape s;
    s.n_mol = j.n_mol;
    s.periodic = j.periodic;
    for (int k = 0; k < 3; ++k) {
        s.grid[k] = j.periodic ? j.grid[k] : 0;
        s.box[k] = j.periodic ? j.box[k] : 0;
    }
    s.rc = j.periodic ? j.rc : 0;
    s.alpha = j.periodic ? j.ewald_alpha : 0;
    return s;
}

// Device memory a context for the job needs: the polarization pair list and
// the neighbour list per molecule, the per-molecule state, the SPME grids and
// a fixed allowance for the context and cuFFT.  An estimate with margin.
size_t estimate_bytes(const sibfa_job &j, int precision) {
    const int nb = j.periodic ? 384 : std::max(1, std::min(384, j.n_mol - 1));
    const size_t entry = precision == SIBFA_PREC_FP64 ? 36 : 20;
    const size_t per_mol =
        (size_t)3 * 3 * nb * entry + (size_t)nb * (precision == SIBFA_PREC_FP64 ? 28 : 16) + 6144;
    size_t b = (size_t)j.n_mol * per_mol;
    if (j.periodic) b += (size_t)j.grid[0] * j.grid[1] * j.grid[2] * (precision == SIBFA_PREC_FP64 ? 80 : 44);
    return b + ((size_t)96 << 20);
}

// dst[m] = src[idx[m]] for molecule records of `width` doubles
__global__ void k_gather_rows(int n, int width, const int *idx, const double *src, double *dst) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * width) return;
    const int m = (int)(t / width), c = (int)(t % width);
    dst[(size_t)m * width + c] = src[(size_t)idx[m] * width + c];
}

// atom masses, 3 per molecule (O, H1, H2): the layout sibfa_md_steps reads
void fill_masses(std::vector<double> &h, int n) {
    h.resize((size_t)n * 3);
    for (int m = 0; m < n; ++m)
        for (int a = 0; a < 3; ++a) h[(size_t)m * 3 + a] = a == 0 ? MASS_O : MASS_H;
}

}  // namespace

struct sibfa_server {
    sibfa_server_opts o{};
    sibfa_params params{};
    int device = 0;
    std::mutex m;
    std::condition_variable cv;
    std::deque<Job *> queue;
    std::unordered_map<uint64_t, Job *> jobs;
    uint64_t next_id = 1;
    std::vector<size_t> resident;   // device bytes held by each slot's cached contexts
    size_t batch_bytes = 0;
    size_t running_bytes = 0;       // estimates of slot jobs whose context is being built
    bool stop = false;
    std::vector<std::thread> workers;
    std::thread batcher;

    size_t used() const {
        size_t u = batch_bytes + running_bytes;
        for (size_t r : resident) u += r;
        return u;
    }
    void finish(Job *j) {
        j->t_done = Clock::now();
        j->state = 2;
    }
};

namespace {

sibfa_run_opts run_opts_for(const sibfa_server &S, const sibfa_job &j, cudaStream_t st) {
    sibfa_run_opts r{};
    r.periodic = j.periodic;
    for (int k = 0; k < 3; ++k) {
        r.box[k] = j.box[k];
        r.grid[k] = j.grid[k];
    }
    r.rc = j.rc;
    r.order = 5;
    r.ewald_alpha = j.ewald_alpha;
    r.pcg_tol_D = S.o.pcg_tol_D;
    r.pcg_max_iter = 200;
    r.precision = S.o.precision;
    r.warm_start = 1;
    r.stream = st;
    r.md_k_bond = 529.6;
    r.md_r0 = 0.9572;
    r.md_k_angle = 34.05;
    r.md_theta0_deg = 104.52;
    return r;
}

// A context a slot keeps for later jobs of the same shape, with its device
// arrays (positions, velocities, masses, forces).
struct SlotCtx {
    Shape shape;
    sibfa_ctx *ctx = nullptr;
    double *dpos = nullptr, *dvel = nullptr, *dmass = nullptr, *dF = nullptr;
    size_t bytes = 0;     // device bytes: the context and the four arrays
    uint64_t last = 0;    // use stamp; the least recently used is evicted first
};
constexpr int SLOT_CACHE = 4;   // contexts (distinct shapes) a slot keeps
constexpr int SLOT_LOOK = 8;    // queued slot jobs a slot looks through for a shape it holds
constexpr int SLOT_WAIT_MS = 250;   // the oldest slot job waiting longer is taken first

void release(SlotCtx &c) {
    if (c.ctx) sibfa_destroy(c.ctx);
    cudaFree(c.dpos), cudaFree(c.dvel), cudaFree(c.dmass), cudaFree(c.dF);
    c = SlotCtx{};
}

int find_shape(const std::vector<SlotCtx> &cache, const Shape &s) {
    for (size_t c = 0; c < cache.size(); ++c)
        if (cache[c].shape == s) return (int)c;
    return -1;
}

// Box jobs (and clusters that do not join the batch) in slot k.  The slot
// keeps up to SLOT_CACHE contexts of distinct shapes.  It takes the oldest of
// the first SLOT_LOOK queued slot jobs whose shape it holds (no context to
// build: allocations, FFT plans, solver graph and launch-shape tuning are
// done once per shape and slot), unless the oldest slot job has waited
// longer than SLOT_WAIT_MS; otherwise the oldest job whose context fits under
// the memory cap, evicting the slot's least recently used contexts as needed.
void slot_worker(sibfa_server *S, int k) {
    cudaSetDevice(S->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<SlotCtx> cache;
    uint64_t stamp = 0;
    std::vector<double> hmass;
    for (;;) {
        Job *j = nullptr;
        int hit = -1;
        std::vector<int> evict;   // cache entries to release before building the job's context
        {
            std::unique_lock<std::mutex> lk(S->m);
            for (;;) {
                if (S->stop) break;
                int seen = 0;
                Job *head = nullptr;
                for (Job *c : S->queue)
                    if (!c->batch) {
                        head = c;
                        break;
                    }
                if (head && Clock::now() - head->t_submit > std::chrono::milliseconds(SLOT_WAIT_MS))
                    seen = SLOT_LOOK;   // no reordering: the oldest job goes next
                for (auto it = S->queue.begin(); it != S->queue.end() && seen < SLOT_LOOK; ++it) {
                    if ((*it)->batch) continue;
                    ++seen;
                    const int c = find_shape(cache, shape_of((*it)->spec));
                    if (c >= 0) {
                        j = *it;
                        hit = c;
                        S->queue.erase(it);
                        break;
                    }
                }
                if (!j) {
                    std::vector<int> order(cache.size());
                    for (size_t c = 0; c < cache.size(); ++c) order[c] = (int)c;
                    std::sort(order.begin(), order.end(), [&](int a, int b) { return cache[a].last < cache[b].last; });
                    const size_t used = S->used();
                    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
                        Job *c = *it;
                        if (c->batch) continue;
                        evict.clear();
                        size_t freed = 0;
                        const size_t must = cache.size() >= (size_t)SLOT_CACHE ? 1 : 0;
                        for (int e : order) {
                            if (evict.size() >= must && used - freed + c->mem <= S->o.device_mem_bytes) break;
                            evict.push_back(e);
                            freed += cache[e].bytes;
                        }
                        if (evict.size() >= must && used - freed + c->mem <= S->o.device_mem_bytes) {
                            j = c;
                            S->queue.erase(it);
                            break;
                        }
                    }
                    if (!j) evict.clear();
                }
                if (j) break;
                S->cv.wait(lk);
            }
            if (!j) break;
            j->state = 1;
            j->t_start = Clock::now();
            if (hit < 0) {
                for (int e : evict) S->resident[k] -= cache[e].bytes;
                S->running_bytes += j->mem;
            }
        }
        const sibfa_job &J = j->spec;
        const size_t nb = (size_t)J.n_mol * 9 * sizeof(double);
        int status = SIBFA_OK;
        if (hit < 0) {
            std::sort(evict.begin(), evict.end(), [](int a, int b) { return a > b; });
            for (int e : evict) {
                release(cache[e]);
                cache.erase(cache.begin() + e);
            }
            SlotCtx c;
            sibfa_topology topo{};
            topo.n_mol = J.n_mol;
            topo.mp_local = j->mp.data();
            const sibfa_run_opts ro = run_opts_for(*S, J, st);
            status = sibfa_create(&S->params, &topo, &ro, &c.ctx);
            if (status == SIBFA_OK) {
                if (cudaMalloc(&c.dpos, nb) != cudaSuccess || cudaMalloc(&c.dvel, nb) != cudaSuccess ||
                    cudaMalloc(&c.dmass, nb) != cudaSuccess || cudaMalloc(&c.dF, nb) != cudaSuccess)
                    status = SIBFA_E_OOM;
                fill_masses(hmass, J.n_mol);
                if (status == SIBFA_OK)
                    cudaMemcpyAsync(c.dmass, hmass.data(), hmass.size() * sizeof(double), cudaMemcpyHostToDevice, st);
                c.shape = shape_of(J);
                c.bytes = c.ctx ? sibfa::ctx_device_bytes(c.ctx) + 4 * nb : 0;
            }
            if (status != SIBFA_OK) release(c);
            std::lock_guard<std::mutex> lk(S->m);
            S->running_bytes -= j->mem;
            if (status == SIBFA_OK) {
                S->resident[k] += c.bytes;
                cache.push_back(c);
                hit = (int)cache.size() - 1;
            }
        } else {
            // same shape: new multipoles; the previous dipoles are the first warm start
            const sibfa::BatchArrays b = sibfa::ctx_batch_arrays(cache[hit].ctx);
            cudaMemcpyAsync(b.mp_local, j->mp.data(), (size_t)J.n_mol * 50 * sizeof(double), cudaMemcpyHostToDevice,
                            sibfa::ctx_stream(cache[hit].ctx));
            cudaStreamSynchronize(sibfa::ctx_stream(cache[hit].ctx));
        }
        if (status == SIBFA_OK) {
            SlotCtx &c = cache[hit];
            c.last = ++stamp;
            cudaMemcpyAsync(c.dpos, j->pos.data(), nb, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(c.dvel, j->vel.data(), nb, cudaMemcpyHostToDevice, st);
            cudaStreamSynchronize(st);
            if (J.n_steps <= 0) status = sibfa_energy_forces(c.ctx, c.dpos, nullptr, &j->terms, c.dF, nullptr);
            else status = sibfa_md_steps(c.ctx, c.dpos, c.dvel, c.dmass, J.dt_fs, J.n_steps, &j->terms);
            j->forces.resize((size_t)J.n_mol * 9);
            j->pos_out.resize((size_t)J.n_mol * 9);
            const double *fsrc = J.n_steps <= 0 ? c.dF : sibfa::ctx_batch_arrays(c.ctx).forces;
            cudaMemcpyAsync(j->forces.data(), fsrc, nb, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(j->pos_out.data(), c.dpos, nb, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            double res = 0;
            sibfa_last_stats(c.ctx, &j->iters, &res);
        }
        {
            std::lock_guard<std::mutex> lk(S->m);
            j->status = status;
            S->finish(j);
        }
        S->cv.notify_all();
    }
    for (SlotCtx &c : cache) release(c);
    cudaStreamDestroy(st);
}

// Regroup the batch: molecules idx (old positions) move to the front of the
// device arrays, in order.
void regroup(cudaStream_t st, const std::vector<int> &idx, int *didx, double *scratch, double *const arrays[4]) {
    const int n = (int)idx.size();
    if (n == 0) return;
    const int width[4] = {9, 9, 50, 9};
    cudaMemcpyAsync(didx, idx.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
    for (int r = 0; r < 4; ++r) {
        const long long cnt = (long long)n * width[r];
        k_gather_rows<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(n, width[r], didx, arrays[r], scratch);
        cudaMemcpyAsync(arrays[r], scratch, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    cudaStreamSynchronize(st);   // idx (host) is reused by the caller
}

// Continuous batching of gas-phase clusters.
void batch_worker(sibfa_server *S) {
    cudaSetDevice(S->device);
    const int B = S->o.batch_waters;
    const int maxc = std::max(2, std::min(S->o.batch_max_cluster, 385));
    // the batch context: capacity B waters; its pair-list stride fits clusters of maxc
    std::vector<double> mp0((size_t)B * 50, 0.0);
    std::vector<int> start0;
    for (int s = 0; s < B; s += maxc) start0.push_back(s);
    start0.push_back(B);
    sibfa_topology topo{};
    topo.n_mol = B;
    topo.mp_local = mp0.data();
    topo.n_clusters = (int)start0.size() - 1;
    topo.cluster_start = start0.data();
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    sibfa_job proto{};
    const sibfa_run_opts ro = run_opts_for(*S, proto, st);
    sibfa_ctx *ctx = nullptr;
    if (sibfa_create(&S->params, &topo, &ro, &ctx) != SIBFA_OK) ctx = nullptr;
    const size_t nb = (size_t)B * 9 * sizeof(double);
    double *dpos = nullptr, *dvel = nullptr, *dmass = nullptr, *scratch = nullptr;
    int *didx = nullptr;
    bool ok = ctx && cudaMalloc(&dpos, nb) == cudaSuccess && cudaMalloc(&dvel, nb) == cudaSuccess &&
              cudaMalloc(&dmass, nb) == cudaSuccess &&
              cudaMalloc(&scratch, (size_t)B * 50 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&didx, (size_t)B * sizeof(int)) == cudaSuccess;
    std::vector<double> hmass;
    fill_masses(hmass, B);
    if (ok) cudaMemcpyAsync(dmass, hmass.data(), hmass.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->batch_bytes = ok ? sibfa::ctx_device_bytes(ctx) + 3 * nb + (size_t)B * (50 * 8 + 4) : 0;
        if (!ok) {
            // no batch: its jobs go to the slots
            for (Job *j : S->queue) j->batch = false;
            S->o.batch_waters = 0;
        }
    }
    S->cv.notify_all();
    std::vector<Job *> active;   // in batch order
    std::vector<int> offset;     // first molecule of each active job
    std::vector<sibfa_energy_terms> terms;
    std::vector<int> idx;
    while (ok) {
        // 1. admission
        std::vector<Job *> joined;
        {
            std::unique_lock<std::mutex> lk(S->m);
            for (;;) {
                int used = 0;
                for (Job *a : active) used += a->spec.n_mol;
                for (auto it = S->queue.begin(); it != S->queue.end();) {
                    Job *c = *it;
                    if (c->batch && used + c->spec.n_mol <= B) {
                        used += c->spec.n_mol;
                        c->state = 1;
                        c->t_start = Clock::now();
                        joined.push_back(c);
                        it = S->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                if (!active.empty() || !joined.empty() || S->stop) break;
                S->cv.wait(lk);
            }
            if (S->stop && active.empty() && joined.empty()) break;
        }
        const sibfa::BatchArrays b = sibfa::ctx_batch_arrays(ctx);
        double *const arrays[4] = {dpos, dvel, b.mp_local, b.mu};
        // 2. regroup: the jobs already in the batch first, the new ones appended
        if (!joined.empty()) {
            int M = 0;
            idx.clear();
            std::vector<int> new_off;
            for (size_t a = 0; a < active.size(); ++a) {
                new_off.push_back(M);
                for (int q = 0; q < active[a]->spec.n_mol; ++q) idx.push_back(offset[a] + q);
                M += active[a]->spec.n_mol;
            }
            regroup(st, idx, didx, scratch, arrays);
            for (Job *j : joined) {
                const size_t nbj = (size_t)j->spec.n_mol * 9 * sizeof(double);
                cudaMemcpyAsync(dpos + (size_t)M * 9, j->pos.data(), nbj, cudaMemcpyHostToDevice, st);
                cudaMemcpyAsync(dvel + (size_t)M * 9, j->vel.data(), nbj, cudaMemcpyHostToDevice, st);
                cudaMemcpyAsync(b.mp_local + (size_t)M * 50, j->mp.data(),
                                (size_t)j->spec.n_mol * 50 * sizeof(double), cudaMemcpyHostToDevice, st);
                cudaMemsetAsync(b.mu + (size_t)M * 9, 0, nbj, st);
                new_off.push_back(M);
                active.push_back(j);
                M += j->spec.n_mol;
            }
            offset = new_off;
            cudaStreamSynchronize(st);
            std::vector<int> cs(1, 0);
            for (Job *a : active) cs.push_back(cs.back() + a->spec.n_mol);
            if (sibfa::ctx_set_batch(ctx, M, (int)active.size(), cs.data()) != SIBFA_OK) ok = false;
        }
        if (!ok) break;
        // 3. one velocity-Verlet step, or one evaluation for newly joined jobs that ask for none
        bool want_eval = false;
        for (Job *a : active) want_eval |= a->spec.n_steps <= 0 && a->steps_done == 0;
        int status;
        sibfa_energy_terms tot{};
        const int n_act = (int)active.size();
        if (want_eval) {
            status = sibfa_energy_forces(ctx, dpos, nullptr, &tot, scratch, nullptr);
        } else {
            status = sibfa_md_steps(ctx, dpos, dvel, dmass, S->o.batch_dt_fs, 1, &tot);
            for (Job *a : active) a->steps_done += 1;
        }
        terms.assign(n_act, sibfa_energy_terms{});
        if (status == SIBFA_OK || status == SIBFA_E_NOT_CONVERGED) sibfa_cluster_terms(ctx, terms.data());
        int iters = 0;
        double res = 0;
        sibfa_last_stats(ctx, &iters, &res);
        // 4. jobs that reached their step count (or failed with the batch) leave
        std::vector<Job *> left, keep;
        std::vector<int> left_off, keep_off;
        for (int a = 0; a < n_act; ++a) {
            Job *j = active[a];
            const bool done = status != SIBFA_OK || j->steps_done >= std::max(0, j->spec.n_steps);
            if (done) {
                left.push_back(j);
                left_off.push_back(offset[a]);
                j->terms = terms[a];
            } else {
                keep.push_back(j);
                keep_off.push_back(offset[a]);
            }
        }
        if (left.empty()) continue;
        // forces of the last evaluation: the integrator's (step) or the explicit output (evaluation)
        const double *fsrc = want_eval ? scratch : b.forces;
        for (size_t q = 0; q < left.size(); ++q) {
            Job *j = left[q];
            const size_t nbj = (size_t)j->spec.n_mol * 9 * sizeof(double);
            j->forces.resize((size_t)j->spec.n_mol * 9);
            j->pos_out.resize((size_t)j->spec.n_mol * 9);
            cudaMemcpyAsync(j->forces.data(), fsrc + (size_t)left_off[q] * 9, nbj, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(j->pos_out.data(), dpos + (size_t)left_off[q] * 9, nbj, cudaMemcpyDeviceToHost, st);
        }
        cudaStreamSynchronize(st);
        {
            std::lock_guard<std::mutex> lk(S->m);
            for (Job *j : left) {
                j->status = status;
                j->iters = iters;
                S->finish(j);
            }
        }
        S->cv.notify_all();
        if (!keep.empty()) {
            int M = 0;
            idx.clear();
            std::vector<int> new_off;
            for (size_t a = 0; a < keep.size(); ++a) {
                new_off.push_back(M);
                for (int q = 0; q < keep[a]->spec.n_mol; ++q) idx.push_back(keep_off[a] + q);
                M += keep[a]->spec.n_mol;
            }
            regroup(st, idx, didx, scratch, arrays);
            std::vector<int> cs(1, 0);
            for (Job *a : keep) cs.push_back(cs.back() + a->spec.n_mol);
            if (sibfa::ctx_set_batch(ctx, M, (int)keep.size(), cs.data()) != SIBFA_OK) ok = false;
            keep_off = new_off;
        }
        active = keep;
        offset = keep_off;
    }
    if (!ok) {
        // the batch failed: finish its jobs with an error, and send the queued
        // cluster jobs to the slots rather than leave them waiting
        std::lock_guard<std::mutex> lk(S->m);
        for (Job *j : active) {
            j->status = SIBFA_E_CUDA;
            S->finish(j);
        }
        for (Job *j : S->queue) j->batch = false;
        S->o.batch_waters = 0;
    }
    S->cv.notify_all();
    if (ctx) sibfa_destroy(ctx);
    cudaFree(dpos), cudaFree(dvel), cudaFree(dmass), cudaFree(scratch), cudaFree(didx);
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

sibfa_status sibfa_server_create(const sibfa_server_opts *opts, sibfa_server **out) {
    if (out) *out = nullptr;
    if (!opts || !out || !opts->params || opts->slots < 1 || opts->max_pending < 1 || opts->batch_waters < 0 ||
        (opts->precision != SIBFA_PREC_MIXED && opts->precision != SIBFA_PREC_FP64))
        return SIBFA_E_INVALID;
    sibfa_server *S = new sibfa_server();
    S->o = *opts;
    S->params = *opts->params;
    S->o.params = &S->params;
    if (S->o.batch_dt_fs <= 0) S->o.batch_dt_fs = 0.5;
    if (S->o.pcg_tol_D <= 0) S->o.pcg_tol_D = 1e-6;
    if (S->o.batch_max_cluster <= 0) S->o.batch_max_cluster = 32;
    cudaGetDevice(&S->device);
    S->resident.assign(S->o.slots, 0);
    for (int k = 0; k < S->o.slots; ++k) S->workers.emplace_back(slot_worker, S, k);
    if (S->o.batch_waters > 0) S->batcher = std::thread(batch_worker, S);
    *out = S;
    return SIBFA_OK;
}

sibfa_status sibfa_submit(sibfa_server *S, const sibfa_job *job, uint64_t *ticket) {
    if (!S || !job || !ticket || job->n_mol < 1 || !job->pos || !job->mp_local) return SIBFA_E_INVALID;
    Job *j = new Job();
    j->spec = *job;
    const size_t n9 = (size_t)job->n_mol * 9;
    j->pos.assign(job->pos, job->pos + n9);
    if (job->vel) j->vel.assign(job->vel, job->vel + n9);
    else j->vel.assign(n9, 0.0);
    j->mp.assign(job->mp_local, job->mp_local + (size_t)job->n_mol * 50);
    j->spec.pos = j->spec.vel = j->spec.mp_local = nullptr;
    j->mem = estimate_bytes(*job, S->o.precision);
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->m);
        j->batch = !job->periodic && S->o.batch_waters > 0 && job->n_mol <= S->o.batch_max_cluster &&
                   job->n_mol <= S->o.batch_waters;
        if (S->stop || (!j->batch && j->mem > S->o.device_mem_bytes)) {
            const bool stopped = S->stop;
            delete j;
            return stopped ? SIBFA_E_BUSY : SIBFA_E_INVALID;
        }
        if ((int)S->queue.size() >= S->o.max_pending) {
            delete j;
            return SIBFA_E_BUSY;
        }
        j->id = S->next_id++;
        S->jobs[j->id] = j;
        S->queue.push_back(j);
        *ticket = j->id;
    }
    S->cv.notify_all();
    return SIBFA_OK;
}

sibfa_status sibfa_poll(sibfa_server *S, uint64_t ticket, sibfa_result *out, int *done) {
    if (!S || !done) return SIBFA_E_INVALID;
    Job *j = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->m);
        auto it = S->jobs.find(ticket);
        if (it == S->jobs.end()) return SIBFA_E_INVALID;
        j = it->second;
        if (j->state != 2) {
            *done = 0;
            return SIBFA_OK;
        }
        S->jobs.erase(it);
    }
    *done = 1;
    if (out) {
        out->terms = j->terms;
        out->status = j->status;
        out->pcg_iters = j->iters;
        out->batched = j->batch ? 1 : 0;
        out->queue_ms = std::chrono::duration<double, std::milli>(j->t_start - j->t_submit).count();
        out->latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
        const size_t n9 = (size_t)j->spec.n_mol * 9;
        if (out->forces && j->forces.size() == n9) std::memcpy(out->forces, j->forces.data(), n9 * sizeof(double));
        if (out->pos && j->pos_out.size() == n9) std::memcpy(out->pos, j->pos_out.data(), n9 * sizeof(double));
    }
    delete j;
    return SIBFA_OK;
}

void sibfa_server_destroy(sibfa_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &t : S->workers) t.join();
    if (S->batcher.joinable()) S->batcher.join();
    for (auto &kv : S->jobs) delete kv.second;
    delete S;
}

}  // extern "C"
