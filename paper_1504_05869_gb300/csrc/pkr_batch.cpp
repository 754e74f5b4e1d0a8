// pkr_batch.cpp -- batches and serving (pkr_ctx_*, pkr_submit, pkr_poll).
//
// A context owns the device-resident batch state: one descriptor per live
// grid, the batch-wide tile partials and per-grid residuals.  One K-step
// "window" is a captured CUDA graph: K x (persistent batch sweep, step
// counter increment), the per-grid residual reduction and the copy of the
// residuals to pinned host memory.  Between windows the host admits queued
// requests that fit the HBM budget (first fit; source preparation on the
// context's stream; they start at the window boundary) and retires the grids
// whose check at the end of the window passed.  A worker thread drives the
// windows in threaded contexts; pkr_ctx_run does in the others.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "pkr_internal.h"

namespace pkr {
template <class L, typename T> int launch_batch_t(int, BatchState*, int, int, void*);
template <class L, typename T> int batch_occupancy_t(int, int*);
template <class L> int variant_count_t();

namespace {

template <class L>
int batch_launch_l(int prec, int var, BatchState* st, int K, int grid, void* s)
{
    return prec == PKR_FP64 ? launch_batch_t<L, double>(var, st, K, grid, s)
                            : launch_batch_t<L, float>(var, st, K, grid, s);
}
template <class L>
int batch_occ_l(int prec, int var, int* b)
{
    return prec == PKR_FP64 ? batch_occupancy_t<L, double>(var, b)
                            : batch_occupancy_t<L, float>(var, b);
}

}  // namespace

int launch_batch_step(int lattice, int precision, int variant, BatchState* st, int K, int grid,
                      void* stream)
{
    switch (lattice) {
    case PKR_D1Q5: return batch_launch_l<D1Q5>(precision, variant, st, K, grid, stream);
    case PKR_D1Q9: return batch_launch_l<D1Q9>(precision, variant, st, K, grid, stream);
    case PKR_D1Q13: return batch_launch_l<D1Q13>(precision, variant, st, K, grid, stream);
    case PKR_D2Q25: return batch_launch_l<D2Q25>(precision, variant, st, K, grid, stream);
    case PKR_D2Q81: return batch_launch_l<D2Q81>(precision, variant, st, K, grid, stream);
    case PKR_D2Q169: return batch_launch_l<D2Q169>(precision, variant, st, K, grid, stream);
    case PKR_D3Q19: return batch_launch_l<D3Q19>(precision, variant, st, K, grid, stream);
    case PKR_D3Q111: return batch_launch_l<D3Q111>(precision, variant, st, K, grid, stream);
    }
    return (int)cudaErrorInvalidValue;
}

int batch_occupancy(int lattice, int precision, int variant, int* blocks)
{
    switch (lattice) {
    case PKR_D1Q5: return batch_occ_l<D1Q5>(precision, variant, blocks);
    case PKR_D1Q9: return batch_occ_l<D1Q9>(precision, variant, blocks);
    case PKR_D1Q13: return batch_occ_l<D1Q13>(precision, variant, blocks);
    case PKR_D2Q25: return batch_occ_l<D2Q25>(precision, variant, blocks);
    case PKR_D2Q81: return batch_occ_l<D2Q81>(precision, variant, blocks);
    case PKR_D2Q169: return batch_occ_l<D2Q169>(precision, variant, blocks);
    case PKR_D3Q19: return batch_occ_l<D3Q19>(precision, variant, blocks);
    case PKR_D3Q111: return batch_occ_l<D3Q111>(precision, variant, blocks);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace pkr

using namespace pkr;

namespace {

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket = 0;
    pkr_problem prob{};
    const double* rho = nullptr;
    double* phi = nullptr;
    int host = 0;
    int status = PKR_EBUSY;
    pkr_stats st{};
    void* pop[2] = {nullptr, nullptr};
    void* S = nullptr;
    double* Phi = nullptr;
    size_t bytes = 0;
    int64_t V = 0;
    int ntiles = 0;
    long long join = 0;
    double tau = 0, omega = 0, mean = 0;
    double t_submit = 0;
    int small = 0;
};

}  // namespace

struct pkr_ctx {
    pkr_ctx_config cfg{};
    LatticeInfo li{};
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 0, elem = 8, variant = 0, grid = 0, K = 32, max_grids = 4096;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::deque<Job*> queue;
    std::vector<Job*> live;
    std::map<uint64_t, Job*> jobs;
    uint64_t next_ticket = 1;
    // device state
    BatchState* d_state = nullptr;
    BatchState h_state{};
    unsigned char* d_grids = nullptr;
    std::vector<unsigned char> h_grids;
    int grid_stride = 0;
    double* d_tile_partials = nullptr;
    int64_t tiles_cap = 0;
    double* d_res = nullptr;
    double* h_res = nullptr;   // pinned, 3 per grid slot
    double* d_scratch = nullptr;
    int* d_flag = nullptr;
    double* d_mean = nullptr;
    int* h_flag = nullptr;     // pinned
    double* h_mean = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    long long step = 0;
    bool dirty = true;
    int64_t finished = 0, windows = 0;
    double site_updates = 0;
};

namespace {

constexpr int kScratchBlocks = 152 * 4;

template <typename R>
void fill_grid(unsigned char* dst, const Job* j, const LatticeInfo& li, int tile_begin)
{
    BatchGrid<R> g{};
    g.pop[0] = j->pop[0];
    g.pop[1] = j->pop[1];
    g.S = j->S;
    g.Phi = j->Phi;
    g.V = j->V;
    g.nx = (int)j->prob.n[0];
    g.ny = (int)j->prob.n[1];
    g.nz = (int)j->prob.n[2];
    g.small = j->small;
    g.tile_begin = tile_begin;
    g.join = j->join;
    g.c.om1 = (R)(1.0 - j->omega);
    for (int c = 0; c < li.ncls; ++c) {
        g.c.wphi[c] = (R)(j->omega * li.cls_phi[c]);
        g.c.chi[c] = (R)li.cls_chi[c];
    }
    std::memcpy(dst, &g, sizeof(g));
}

size_t job_bytes(const pkr_ctx* C, int64_t V)
{
    const size_t e = (size_t)C->elem;
    return 2 * (size_t)C->li.Q * (size_t)V * e + (size_t)V * e + (size_t)V * 8;
}

void free_job_memory(pkr_ctx* C, Job* j)
{
    for (int k = 0; k < 2; ++k)
        if (j->pop[k]) cudaFreeAsync(j->pop[k], C->stream);
    if (j->S) cudaFreeAsync(j->S, C->stream);
    if (j->Phi) cudaFreeAsync(j->Phi, C->stream);
    j->pop[0] = j->pop[1] = j->S = nullptr;
    j->Phi = nullptr;
    C->used -= j->bytes;
    j->bytes = 0;
}

void finish(pkr_ctx* C, Job* j, int status)
{
    j->status = status;
    j->st.wall_ms = now_ms() - j->t_submit;
    C->finished += 1;
    C->cv_done.notify_all();
}

// Allocate and prepare a request (context stream; caller holds the lock).
// Returns PKR_OK, PKR_ENOMEM (try later) or a final error status.
int admit(pkr_ctx* C, Job* j)
{
    const size_t b = job_bytes(C, j->V);
    const size_t popb = (size_t)C->li.Q * (size_t)j->V * (size_t)C->elem;
    if (cudaMallocAsync(&j->pop[0], popb, C->stream) != cudaSuccess ||
        cudaMallocAsync(&j->pop[1], popb, C->stream) != cudaSuccess ||
        cudaMallocAsync(&j->S, (size_t)j->V * C->elem, C->stream) != cudaSuccess ||
        cudaMallocAsync((void**)&j->Phi, (size_t)j->V * 8, C->stream) != cudaSuccess) {
        cudaGetLastError();
        j->bytes = 0;
        for (int k = 0; k < 2; ++k)
            if (j->pop[k]) cudaFreeAsync(j->pop[k], C->stream);
        if (j->S) cudaFreeAsync(j->S, C->stream);
        if (j->Phi) cudaFreeAsync(j->Phi, C->stream);
        j->pop[0] = j->pop[1] = j->S = nullptr;
        j->Phi = nullptr;
        return PKR_ENOMEM;
    }
    j->bytes = b;
    C->used += b;
    const double* rd = j->rho;
    if (j->host) {
        if (cudaMemcpyAsync(j->Phi, j->rho, (size_t)j->V * 8, cudaMemcpyHostToDevice,
                            C->stream) != cudaSuccess)
            return PKR_ECUDA;
        rd = j->Phi;
    }
    const double scale = C->li.cs2 * (j->tau - 0.5) / j->prob.epsilon;
    if (cudaMemsetAsync(C->d_flag, 0, sizeof(int), C->stream) != cudaSuccess ||
        launch_rho_partials(rd, j->V, C->d_scratch, kScratchBlocks, C->d_flag, C->stream) != 0 ||
        launch_finalize_mean(C->d_scratch, kScratchBlocks, j->V, C->d_mean, C->stream) != 0 ||
        launch_make_source(rd, C->d_mean, scale, j->V, j->S, C->cfg.precision, C->stream) != 0 ||
        cudaMemcpyAsync(C->h_flag, C->d_flag, sizeof(int), cudaMemcpyDeviceToHost, C->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(C->h_mean, C->d_mean, sizeof(double), cudaMemcpyDeviceToHost,
                        C->stream) != cudaSuccess ||
        cudaMemsetAsync(j->Phi, 0, (size_t)j->V * 8, C->stream) != cudaSuccess ||
        cudaStreamSynchronize(C->stream) != cudaSuccess)
        return PKR_ECUDA;
    if (*C->h_flag) return PKR_EINVAL;
    j->mean = *C->h_mean;
    j->join = C->step;
    return PKR_OK;
}

// Upload the descriptors of the live grids (and grow the tile partials).
int rebuild(pkr_ctx* C)
{
    int64_t tiles = 0;
    for (Job* j : C->live) tiles += j->ntiles;
    if (tiles > 0x7fffffff) return PKR_EINVAL;
    if (tiles > C->tiles_cap) {
        if (C->d_tile_partials) cudaFreeAsync(C->d_tile_partials, C->stream);
        C->d_tile_partials = nullptr;
        int64_t cap = tiles + tiles / 4 + 1024;
        if (cudaMallocAsync((void**)&C->d_tile_partials, (size_t)cap * 3 * sizeof(double),
                            C->stream) != cudaSuccess) {
            C->tiles_cap = 0;
            return PKR_ENOMEM;
        }
        C->tiles_cap = cap;
    }
    int tb = 0;
    for (size_t k = 0; k < C->live.size(); ++k) {
        unsigned char* dst = C->h_grids.data() + k * (size_t)C->grid_stride;
        if (C->cfg.precision == PKR_FP64) fill_grid<double>(dst, C->live[k], C->li, tb);
        else fill_grid<float>(dst, C->live[k], C->li, tb);
        tb += C->live[k]->ntiles;
    }
    C->h_state.grids = C->d_grids;
    C->h_state.tile_partials = C->d_tile_partials;
    C->h_state.grid_res = C->d_res;
    C->h_state.step = C->step;
    C->h_state.ngrids = (int)C->live.size();
    C->h_state.ntiles = (int)tiles;
    if (!C->live.empty() &&
        cudaMemcpyAsync(C->d_grids, C->h_grids.data(), C->live.size() * (size_t)C->grid_stride,
                        cudaMemcpyHostToDevice, C->stream) != cudaSuccess)
        return PKR_ECUDA;
    if (cudaMemcpyAsync(C->d_state, &C->h_state, sizeof(BatchState), cudaMemcpyHostToDevice,
                        C->stream) != cudaSuccess ||
        cudaStreamSynchronize(C->stream) != cudaSuccess)
        return PKR_ECUDA;
    C->dirty = false;
    return PKR_OK;
}

// Queue one window (K steps + reduction + residual copy) on the stream.
int enqueue_window(pkr_ctx* C)
{
    for (int k = 0; k < C->K; ++k) {
        if (launch_batch_step(C->cfg.lattice, C->cfg.precision, C->variant, C->d_state, C->K,
                              C->grid, C->stream) != 0 ||
            launch_batch_increment(C->d_state, C->stream) != 0)
            return PKR_ECUDA;
    }
    if (launch_batch_reduce(C->d_state, C->max_grids, C->grid_stride, C->stream) != 0 ||
        cudaMemcpyAsync(C->h_res, C->d_res, (size_t)C->max_grids * 3 * sizeof(double),
                        cudaMemcpyDeviceToHost, C->stream) != cudaSuccess)
        return PKR_ECUDA;
    return PKR_OK;
}

int run_window(pkr_ctx* C)
{
    if (!C->graph) {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal) ==
                  cudaSuccess;
        int rc = ok ? enqueue_window(C) : PKR_ECUDA;
        if (ok) ok = cudaStreamEndCapture(C->stream, &g) == cudaSuccess && rc == PKR_OK;
        if (ok) ok = cudaGraphInstantiate(&C->graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            C->graph = nullptr;
        }
    }
    if (C->graph) {
        if (cudaGraphLaunch(C->graph, C->stream) != cudaSuccess) return PKR_ECUDA;
    } else if (enqueue_window(C) != PKR_OK) {
        return PKR_ECUDA;
    }
    if (cudaStreamSynchronize(C->stream) != cudaSuccess) return PKR_ECUDA;
    C->windows += 1;
    return PKR_OK;
}

// One scheduling round (caller holds the lock): admit, run a window, retire.
// Returns 1 if work was done, 0 if idle, < 0 on a CUDA error.
int round(pkr_ctx* C, std::unique_lock<std::mutex>& lk)
{
    // admit (first fit, FIFO order) while memory and descriptor slots allow
    for (auto it = C->queue.begin(); it != C->queue.end();) {
        Job* j = *it;
        if ((int)C->live.size() >= C->max_grids) break;
        if (C->used + job_bytes(C, j->V) > C->budget) {
            ++it;
            continue;
        }
        int rc = admit(C, j);
        if (rc == PKR_ENOMEM) {
            ++it;
            continue;
        }
        it = C->queue.erase(it);
        if (rc != PKR_OK) {
            free_job_memory(C, j);
            finish(C, j, rc);
            continue;
        }
        C->live.push_back(j);
        C->dirty = true;
    }
    if (C->live.empty()) {
        // nothing runs, so nothing will free memory: a queued request that
        // could not be allocated now never will be
        if (!C->queue.empty()) {
            Job* j = C->queue.front();
            C->queue.pop_front();
            finish(C, j, PKR_ENOMEM);
            return 1;
        }
        return 0;
    }
    if (C->dirty && rebuild(C) != PKR_OK) return -1;
    // the window runs without the lock so that submissions and polls proceed
    lk.unlock();
    int rc = run_window(C);
    lk.lock();
    if (rc != PKR_OK) return -1;
    const long long step0 = C->step;
    C->step += C->K;
    // retire
    std::vector<Job*> keep;
    bool changed = false;
    for (size_t k = 0; k < C->live.size(); ++k) {
        Job* j = C->live[k];
        const long long age_end = C->step - 1 - j->join;    // age of the window's last step
        C->site_updates += (double)j->V * (double)(C->step - (step0 > j->join ? step0 : j->join));
        const bool checked = age_end >= 1;
        const double* r = C->h_res + 3 * k;
        const double res = r[j->prob.tol_kind == PKR_TOL_MAX_ABS_DPHI ? 0 : 1];
        int status = PKR_EBUSY;
        if (checked) {
            if (!std::isfinite(r[0]) || !std::isfinite(r[2])) status = PKR_EDIVERGED;
            else if (j->prob.tol > 0.0 && res < j->prob.tol) status = PKR_OK;
            else if (age_end >= j->prob.max_sweeps)
                status = (j->prob.tol > 0.0) ? PKR_ENOCONV : PKR_OK;
        }
        if (status == PKR_EBUSY) {
            keep.push_back(j);
            continue;
        }
        j->st.sweeps = age_end;
        j->st.launches = age_end + 1;
        j->st.residual = res;
        j->st.rho_mean_removed = j->mean;
        j->st.tau_lb = j->tau;
        j->st.cs2 = C->li.cs2;
        if (status == PKR_OK || status == PKR_ENOCONV) {
            if (cudaMemcpyAsync(j->phi, j->Phi, (size_t)j->V * 8,
                                j->host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                C->stream) != cudaSuccess ||
                cudaStreamSynchronize(C->stream) != cudaSuccess)
                status = PKR_ECUDA;
        }
        free_job_memory(C, j);
        finish(C, j, status);
        changed = true;
    }
    C->live.swap(keep);
    if (changed) C->dirty = true;
    return 1;
}

void worker_main(pkr_ctx* C)
{
    cudaSetDevice(C->device);
    std::unique_lock<std::mutex> lk(C->mu);
    while (!C->stop) {
        int r = round(C, lk);
        if (r < 0) {
            // a CUDA error: fail everything that is queued or live
            for (Job* j : C->live) finish(C, j, PKR_ECUDA);
            for (Job* j : C->queue) finish(C, j, PKR_ECUDA);
            C->live.clear();
            C->queue.clear();
            continue;
        }
        if (r == 0) C->cv_work.wait(lk, [&] { return C->stop || !C->queue.empty(); });
    }
}

int tune_variant(pkr_ctx* C, int edge);

}  // namespace

extern "C" {

int pkr_ctx_create(const pkr_ctx_config* cfg, void* stream, pkr_ctx** out)
{
    if (!cfg || !out) return PKR_EINVAL;
    *out = nullptr;
    if (cfg->check_every < 1 || cfg->hbm_budget_bytes == 0) return PKR_EINVAL;
    if (cfg->precision != PKR_FP64 && cfg->precision != PKR_FP32) return PKR_EINVAL;
    LatticeInfo li;
    int rc = build_lattice(cfg->lattice, cfg->order, &li);
    if (rc != PKR_OK) return rc;
    pkr_ctx* C = new (std::nothrow) pkr_ctx();
    if (!C) return PKR_ENOMEM;
    C->cfg = *cfg;
    C->li = li;
    C->stream = (cudaStream_t)stream;
    C->elem = cfg->precision == PKR_FP64 ? 8 : 4;
    C->K = cfg->check_every;
    C->budget = cfg->hbm_budget_bytes;
    C->max_grids = cfg->max_grids > 0 ? cfg->max_grids : 4096;
    C->grid_stride = cfg->precision == PKR_FP64 ? (int)sizeof(BatchGrid<double>)
                                                : (int)sizeof(BatchGrid<float>);
    C->h_grids.assign((size_t)C->max_grids * C->grid_stride, 0);
    bool ok = cudaGetDevice(&C->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&C->nsm, cudaDevAttrMultiProcessorCount, C->device) ==
                  cudaSuccess &&
              cudaMalloc((void**)&C->d_state, sizeof(BatchState)) == cudaSuccess &&
              cudaMalloc((void**)&C->d_grids, (size_t)C->max_grids * C->grid_stride) ==
                  cudaSuccess &&
              cudaMalloc((void**)&C->d_res, (size_t)C->max_grids * 3 * sizeof(double)) ==
                  cudaSuccess &&
              cudaMalloc((void**)&C->d_scratch, kScratchBlocks * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&C->d_flag, sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&C->d_mean, sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void**)&C->h_res, (size_t)C->max_grids * 3 * sizeof(double)) ==
                  cudaSuccess &&
              cudaMallocHost((void**)&C->h_flag, sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void**)&C->h_mean, sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pkr_ctx_destroy(C);
        return PKR_ENOMEM;
    }
    std::memset(&C->h_state, 0, sizeof(BatchState));
    if (cudaMemcpy(C->d_state, &C->h_state, sizeof(BatchState), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        pkr_ctx_destroy(C);
        return PKR_ECUDA;
    }
    const int nvar = pkr_variant_count(cfg->lattice);
    int var = cfg->variant;
    if (var >= nvar || var < -2) {
        pkr_ctx_destroy(C);
        return PKR_EINVAL;
    }
    if (var == -2) {
        var = tune_variant(C, cfg->probe_edge > 0 ? cfg->probe_edge : 64);
        if (var < 0) {
            pkr_ctx_destroy(C);
            return PKR_ECUDA;
        }
    } else if (var == -1) {
        var = nvar > 2 ? 2 : 0;
    }
    C->variant = var;
    int bps = 0;
    if (batch_occupancy(cfg->lattice, cfg->precision, var, &bps) != 0 || bps < 1) {
        pkr_ctx_destroy(C);
        return PKR_ECUDA;
    }
    C->grid = C->nsm * bps;
    if (cfg->threaded) C->worker = std::thread(worker_main, C);
    *out = C;
    return PKR_OK;
}

int pkr_submit(pkr_ctx* C, const pkr_problem* p, const double* rho, double* phi, int host_buffers,
               uint64_t* ticket)
{
    if (!C || !p || !rho || !phi || !ticket) return PKR_EINVAL;
    if (p->lattice != C->cfg.lattice || p->order != C->cfg.order ||
        p->precision != C->cfg.precision || p->dim != C->li.dim)
        return PKR_EINVAL;
    int64_t V = 1;
    for (int k = 0; k < 3; ++k) {
        if (p->n[k] < 1 || (k >= p->dim && p->n[k] != 1)) return PKR_EINVAL;
        V *= p->n[k];
        if (V > (int64_t)0x7fffffff) return PKR_EINVAL;
    }
    if (p->max_sweeps < 1 || (p->tol_kind != 0 && p->tol_kind != 1)) return PKR_EINVAL;
    double tau = p->tau_lb;
    if (!(tau > 0.0) && pkr_tau_from_knudsen(p->lattice, p->knudsen, p->n, &tau) != PKR_OK)
        return PKR_EINVAL;
    if (!(tau > 0.5) || !std::isfinite(tau)) return PKR_EINVAL;
    if (unstable(C->li, 1.0 / tau)) return PKR_EUNSTABLE;
    if (job_bytes(C, V) > C->budget) return PKR_ENOMEM;
    Job* j = new (std::nothrow) Job();
    if (!j) return PKR_ENOMEM;
    j->prob = *p;
    if (j->prob.epsilon == 0.0) j->prob.epsilon = 1.0;
    j->rho = rho;
    j->phi = phi;
    j->host = host_buffers ? 1 : 0;
    j->V = V;
    j->ntiles = (int)((V + 31) / 32);
    j->tau = tau;
    j->omega = 1.0 / tau;
    for (int k = 0; k < C->li.dim; ++k)
        if (p->n[k] < C->li.reach) j->small = 1;
    j->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(C->mu);
        j->ticket = C->next_ticket++;
        C->jobs[j->ticket] = j;
        C->queue.push_back(j);
    }
    C->cv_work.notify_all();
    *ticket = j->ticket;
    return PKR_OK;
}

int pkr_poll(pkr_ctx* C, uint64_t ticket, pkr_stats* st)
{
    if (!C) return PKR_EINVAL;
    std::lock_guard<std::mutex> lk(C->mu);
    auto it = C->jobs.find(ticket);
    if (it == C->jobs.end()) return PKR_EINVAL;
    Job* j = it->second;
    if (j->status != PKR_EBUSY && st) *st = j->st;
    return j->status;
}

int pkr_ctx_wait(pkr_ctx* C, uint64_t ticket, pkr_stats* st)
{
    if (!C) return PKR_EINVAL;
    std::unique_lock<std::mutex> lk(C->mu);
    auto it = C->jobs.find(ticket);
    if (it == C->jobs.end()) return PKR_EINVAL;
    Job* j = it->second;
    if (!C->cfg.threaded) {
        while (j->status == PKR_EBUSY) {
            int r = round(C, lk);
            if (r < 0) return PKR_ECUDA;
            if (r == 0 && j->status == PKR_EBUSY) return PKR_EINVAL;
        }
    } else {
        C->cv_done.wait(lk, [&] { return j->status != PKR_EBUSY || C->stop; });
    }
    if (st && j->status != PKR_EBUSY) *st = j->st;
    return j->status;
}

int pkr_ctx_run(pkr_ctx* C, int64_t max_windows)
{
    if (!C || C->cfg.threaded) return PKR_EINVAL;
    std::unique_lock<std::mutex> lk(C->mu);
    int64_t n = 0;
    while (max_windows <= 0 || n < max_windows) {
        int r = round(C, lk);
        if (r < 0) return PKR_ECUDA;
        if (r == 0) break;
        ++n;
    }
    return PKR_OK;
}

int pkr_ctx_info(pkr_ctx* C, int64_t* finished, double* site_updates, int64_t* windows,
                 size_t* bytes_in_use, int32_t* variant)
{
    if (!C) return PKR_EINVAL;
    std::lock_guard<std::mutex> lk(C->mu);
    if (finished) *finished = C->finished;
    if (site_updates) *site_updates = C->site_updates;
    if (windows) *windows = C->windows;
    if (bytes_in_use) *bytes_in_use = C->used;
    if (variant) *variant = C->variant;
    return PKR_OK;
}

int pkr_ctx_destroy(pkr_ctx* C)
{
    if (!C) return PKR_OK;
    {
        std::lock_guard<std::mutex> lk(C->mu);
        C->stop = true;
    }
    C->cv_work.notify_all();
    C->cv_done.notify_all();
    if (C->worker.joinable()) C->worker.join();
    if (C->stream || C->d_state) cudaStreamSynchronize(C->stream);
    for (auto& kv : C->jobs) {
        Job* j = kv.second;
        for (int k = 0; k < 2; ++k)
            if (j->pop[k]) cudaFree(j->pop[k]);
        if (j->S) cudaFree(j->S);
        if (j->Phi) cudaFree(j->Phi);
        delete j;
    }
    if (C->graph) cudaGraphExecDestroy(C->graph);
    cudaFree(C->d_state);
    cudaFree(C->d_grids);
    cudaFree(C->d_res);
    cudaFree(C->d_scratch);
    cudaFree(C->d_flag);
    cudaFree(C->d_mean);
    if (C->d_tile_partials) cudaFree(C->d_tile_partials);
    if (C->h_res) cudaFreeHost(C->h_res);
    if (C->h_flag) cudaFreeHost(C->h_flag);
    if (C->h_mean) cudaFreeHost(C->h_mean);
    delete C;
    return PKR_OK;
}

}  // extern "C"

namespace {

// Autotuner of the batch geometry: time one step of every compiled variant on
// a probe grid (edge^3, zero source) in this context's batch layout, keep
// the fastest.  Runs at context creation, before any request, so that every
// request of the context sees the same kernel.
int tune_variant(pkr_ctx* C, int edge)
{
    const int nvar = pkr_variant_count(C->cfg.lattice);
    Job probe;
    probe.prob.n[0] = edge;
    probe.prob.n[1] = C->li.dim >= 2 ? edge : 1;
    probe.prob.n[2] = C->li.dim >= 3 ? edge : 1;
    probe.V = probe.prob.n[0] * probe.prob.n[1] * probe.prob.n[2];
    probe.ntiles = (int)((probe.V + 31) / 32);
    probe.omega = 0.5;
    for (int k = 0; k < C->li.dim; ++k)
        if (probe.prob.n[k] < C->li.reach) probe.small = 1;
    const size_t popb = (size_t)C->li.Q * (size_t)probe.V * (size_t)C->elem;
    if (cudaMalloc(&probe.pop[0], popb) != cudaSuccess ||
        cudaMalloc(&probe.pop[1], popb) != cudaSuccess ||
        cudaMalloc(&probe.S, (size_t)probe.V * C->elem) != cudaSuccess ||
        cudaMalloc((void**)&probe.Phi, (size_t)probe.V * 8) != cudaSuccess) {
        cudaGetLastError();
        for (int k = 0; k < 2; ++k) cudaFree(probe.pop[k]);
        cudaFree(probe.S);
        cudaFree(probe.Phi);
        return -1;
    }
    cudaMemset(probe.pop[0], 0, popb);
    cudaMemset(probe.pop[1], 0, popb);
    cudaMemset(probe.S, 0, (size_t)probe.V * C->elem);
    probe.join = -1;   // never the zero-in step: the timed steps pull real data
    C->live.push_back(&probe);
    int best = -1;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (rebuild(C) == PKR_OK) {
        for (int v = 0; v < nvar; ++v) {
            int bps = 0;
            if (batch_occupancy(C->cfg.lattice, C->cfg.precision, v, &bps) != 0 || bps < 1)
                continue;
            const int grid = C->nsm * bps;
            launch_batch_step(C->cfg.lattice, C->cfg.precision, v, C->d_state, 1 << 30, grid,
                              C->stream);
            cudaEventRecord(e0, C->stream);
            for (int k = 0; k < 3; ++k)
                launch_batch_step(C->cfg.lattice, C->cfg.precision, v, C->d_state, 1 << 30,
                                  grid, C->stream);
            cudaEventRecord(e1, C->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    C->live.clear();
    C->dirty = true;
    C->step = 0;
    std::memset(&C->h_state, 0, sizeof(BatchState));
    cudaMemcpy(C->d_state, &C->h_state, sizeof(BatchState), cudaMemcpyHostToDevice);
    for (int k = 0; k < 2; ++k) cudaFree(probe.pop[k]);
    cudaFree(probe.S);
    cudaFree(probe.Phi);
    probe.pop[0] = probe.pop[1] = probe.S = nullptr;
    probe.Phi = nullptr;
    return best;
}

}  // namespace
