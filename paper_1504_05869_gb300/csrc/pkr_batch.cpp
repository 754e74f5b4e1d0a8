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
//
// A MIXED context runs two such batches ("lanes"): binary32 and binary64.
// Requests start in the binary32 lane; when a request's own residual passes
// PKR_MIXED_SWITCH_TOL (or stops falling at the binary32 rounding floor) its
// state is converted to binary64 and it continues in the binary64 lane, with
// its age and check schedule unchanged, until its tolerance.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

#include "pkr_internal.h"

namespace pkr {
template <class L, typename T> int launch_batch_t(int, BatchState*, int, int, void*);
template <class L, typename T> int batch_occupancy_t(int, int*);
template <class L> int batch_variant_count_t();

namespace {

// Compiled geometries of the batch sweep (the staged ones; the plan sweep's
// warp-specialised variants have no batch form).
int batch_variant_count(int lattice)
{
    switch (lattice) {
    case PKR_D1Q5: return batch_variant_count_t<D1Q5>();
    case PKR_D1Q9: return batch_variant_count_t<D1Q9>();
    case PKR_D1Q13: return batch_variant_count_t<D1Q13>();
    case PKR_D2Q25: return batch_variant_count_t<D2Q25>();
    case PKR_D2Q81: return batch_variant_count_t<D2Q81>();
    case PKR_D2Q169: return batch_variant_count_t<D2Q169>();
    case PKR_D3Q19: return batch_variant_count_t<D3Q19>();
    case PKR_D3Q111: return batch_variant_count_t<D3Q111>();
    }
    return -1;
}

template <class L>
int batch_launch_l(int prec, int var, BatchState* st, int K, int grid, void* s)
{
    if (prec == PKR_FP64) return launch_batch_t<L, double>(var, st, K, grid, s);
    if (prec == PKR_FX64) return launch_batch_t<L, long long>(var, st, K, grid, s);
    return launch_batch_t<L, float>(var, st, K, grid, s);
}
template <class L>
int batch_occ_l(int prec, int var, int* b)
{
    if (prec == PKR_FP64) return batch_occupancy_t<L, double>(var, b);
    if (prec == PKR_FX64) return batch_occupancy_t<L, long long>(var, b);
    return batch_occupancy_t<L, float>(var, b);
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
    void* pop[2] = {nullptr, nullptr};   // populations in the precision of the job's lane
    void* S = nullptr;                   // source, same precision
    double* Phi = nullptr;               // density (binary64)
    void* fx = nullptr;                  // 16 B of per-grid device state: fixed-point lanes
                                         // int F[2], then the OR bound (u64); binary32
                                         // lanes the source offset (double)
    size_t bytes = 0;                    // bytes counted against the budget (reservation)
    int64_t V = 0;
    int ntiles = 0;
    int lane = 0;                        // 0: first (or only) lane; 1: binary64 lane of MIXED
    long long join = 0;                  // lane step at which the job's age was 0
    double tau = 0, omega = 0, mean = 0;
    double prev_res = INFINITY;          // residual at the previous check (binary32 lane)
    double t_submit = 0;
    int small = 0;
    int waiters = 0;                     // threads blocked in pkr_ctx_wait on this ticket
};

// One batch of grids stored in one precision, advanced by one persistent
// kernel per step and one captured graph per window.
struct Lane {
    int prec = PKR_FP32, elem = 4, grid_stride = 0, variant = 0, grid = 0;
    BatchState* d_state = nullptr;
    BatchState h_state{};
    unsigned char* d_grids = nullptr;
    std::vector<unsigned char> h_grids;
    double* d_tile_partials = nullptr;
    int64_t tiles_cap = 0;
    double* d_res = nullptr;
    double* h_res = nullptr;   // pinned, 4 per grid slot
    cudaGraphExec_t graph = nullptr;
    long long step = 0;
    bool dirty = true;
    std::vector<Job*> live;
};

}  // namespace

struct pkr_ctx {
    pkr_ctx_config cfg{};
    LatticeInfo li{};
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 0, K = 32, max_grids = 4096;
    bool mixed = false;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::deque<Job*> queue;
    std::map<uint64_t, Job*> jobs;
    uint64_t next_ticket = 1;
    Lane lane[2];
    int nlanes = 1;
    double* d_scratch = nullptr;
    int* d_flag = nullptr;
    double* d_mean = nullptr;
    int* h_flag = nullptr;     // pinned
    double* h_mean = nullptr;  // pinned
    int64_t finished = 0, windows = 0;
    double site_updates = 0;
    // non-threaded contexts: set while one thread runs a round (round()
    // drops the lock while the windows run), so that no second thread
    // drives the same lanes at the same time
    bool driving = false;
    // rounds that ran windows; a test may name one (environment variable
    // PKR_TEST_FAIL_ROUND, read at creation) whose window launch then
    // reports a CUDA error without launching anything
    int64_t rounds = 0, fail_round = -1;
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
    if constexpr (std::is_same<R, float>::value) g.soff = static_cast<double*>(j->fx);
    if (j->fx) {
        g.fxF = static_cast<int*>(j->fx);
        g.fxmax = reinterpret_cast<unsigned long long*>(static_cast<char*>(j->fx) + 8);
        g.cfx = std::llround(std::ldexp(1.0 - j->omega, 62));
    }
    g.c.om1 = (R)(1.0 - j->omega);
    for (int c = 0; c < li.ncls; ++c) {
        g.c.wphi[c] = (R)(j->omega * li.cls_phi[c]);
        g.c.chi[c] = (R)li.cls_chi[c];
    }
    std::memcpy(dst, &g, sizeof(g));
}

// Populations and source of one grid in one lane's precision.
size_t lane_bytes(const pkr_ctx* C, int ln, int64_t V)
{
    const size_t e = (size_t)C->lane[ln].elem;
    return 2 * (size_t)C->li.Q * (size_t)V * e + (size_t)V * e;
}

// Budget reservation of a request: its lane-0 state plus Phi; in a MIXED
// context also its binary64 state, which coexists with the binary32 one
// while the state is converted.
size_t job_bytes(const pkr_ctx* C, int64_t V)
{
    size_t b = lane_bytes(C, 0, V) + (size_t)V * 8;
    if (C->mixed) b += lane_bytes(C, 1, V);
    return b;
}

void free_lane_state(pkr_ctx* C, Job* j)
{
    for (int k = 0; k < 2; ++k)
        if (j->pop[k]) cudaFreeAsync(j->pop[k], C->stream);
    if (j->S) cudaFreeAsync(j->S, C->stream);
    j->pop[0] = j->pop[1] = j->S = nullptr;
}

void free_job_memory(pkr_ctx* C, Job* j)
{
    free_lane_state(C, j);
    if (j->Phi) cudaFreeAsync(j->Phi, C->stream);
    if (j->fx) cudaFreeAsync(j->fx, C->stream);
    j->Phi = nullptr;
    j->fx = nullptr;
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

// Allocate the populations and source of a job in lane ln's precision.
bool alloc_lane_state(pkr_ctx* C, Job* j, int ln)
{
    const size_t popb = (size_t)C->li.Q * (size_t)j->V * (size_t)C->lane[ln].elem;
    if (cudaMallocAsync(&j->pop[0], popb, C->stream) != cudaSuccess ||
        cudaMallocAsync(&j->pop[1], popb, C->stream) != cudaSuccess ||
        cudaMallocAsync(&j->S, (size_t)j->V * C->lane[ln].elem, C->stream) != cudaSuccess) {
        cudaGetLastError();
        free_lane_state(C, j);
        return false;
    }
    return true;
}

// S = (rho - <rho>) c_s^2 (tau_lb - 1/2) / eps in lane ln's precision, from
// rho on the device (rd); the mean goes to C->h_mean.  Synchronises.
int make_job_source(pkr_ctx* C, Job* j, const double* rd, int ln)
{
    const double scale = C->li.cs2 * (j->tau - 0.5) / j->prob.epsilon;
    if (cudaMemsetAsync(C->d_flag, 0, sizeof(int), C->stream) != cudaSuccess ||
        launch_rho_partials(rd, j->V, C->d_scratch, kScratchBlocks, C->d_flag, C->stream) != 0 ||
        launch_finalize_mean(C->d_scratch, kScratchBlocks, j->V, C->d_mean, C->stream) != 0 ||
        launch_make_source(rd, C->d_mean, scale, j->V, j->S,
                           C->lane[ln].prec == PKR_FX64 ? PKR_FP64 : C->lane[ln].prec,
                           C->stream) != 0 ||
        cudaMemcpyAsync(C->h_flag, C->d_flag, sizeof(int), cudaMemcpyDeviceToHost, C->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(C->h_mean, C->d_mean, sizeof(double), cudaMemcpyDeviceToHost,
                        C->stream) != cudaSuccess ||
        cudaStreamSynchronize(C->stream) != cudaSuccess)
        return PKR_ECUDA;
    return *C->h_flag ? PKR_EINVAL : PKR_OK;
}

// Allocate and prepare a request in lane 0 (context stream; caller holds
// the lock).  Returns PKR_OK, PKR_ENOMEM (try later; the request then holds no
// memory and no share of the budget) or a final error status.
int admit(pkr_ctx* C, Job* j)
{
    if (!alloc_lane_state(C, j, 0)) return PKR_ENOMEM;
    if (cudaMallocAsync((void**)&j->Phi, (size_t)j->V * 8, C->stream) != cudaSuccess) {
        cudaGetLastError();
        free_lane_state(C, j);
        return PKR_ENOMEM;
    }
    j->bytes = job_bytes(C, j->V);
    C->used += j->bytes;
    const double* rd = j->rho;
    if (j->host) {
        if (cudaMemcpyAsync(j->Phi, j->rho, (size_t)j->V * 8, cudaMemcpyHostToDevice,
                            C->stream) != cudaSuccess)
            return PKR_ECUDA;
        rd = j->Phi;
    }
    int rc = make_job_source(C, j, rd, 0);
    if (rc != PKR_OK) return rc;
    if (cudaMemsetAsync(j->Phi, 0, (size_t)j->V * 8, C->stream) != cudaSuccess) return PKR_ECUDA;
    if (C->lane[0].prec == PKR_FP32) {
        // the source offset of the binary32 mass correction (0 until a check)
        if (cudaMallocAsync(&j->fx, 16, C->stream) != cudaSuccess) {
            cudaGetLastError();
            j->fx = nullptr;
            free_job_memory(C, j);   // the request stays queued: hold nothing
            return PKR_ENOMEM;
        }
        if (cudaMemsetAsync(j->fx, 0, 16, C->stream) != cudaSuccess) return PKR_ECUDA;
    }
    if (C->lane[0].prec == PKR_FX64) {
        // exponent of the first write (the step from zero stores chi_i S): its
        // largest value lands near 2^52, as for a plan
        if (cudaMallocAsync(&j->fx, 16, C->stream) != cudaSuccess) {
            cudaGetLastError();
            j->fx = nullptr;
            free_job_memory(C, j);   // the request stays queued: hold nothing
            return PKR_ENOMEM;
        }
        unsigned long long* mb = reinterpret_cast<unsigned long long*>(static_cast<char*>(j->fx) + 8);
        unsigned long long hm = 0;
        if (cudaMemsetAsync(mb, 0, 8, C->stream) != cudaSuccess ||
            launch_absmax_f64(static_cast<const double*>(j->S), j->V, mb, C->stream) != 0 ||
            cudaMemcpyAsync(&hm, mb, 8, cudaMemcpyDeviceToHost, C->stream) != cudaSuccess ||
            cudaStreamSynchronize(C->stream) != cudaSuccess)
            return PKR_ECUDA;
        double ms = 0.0;
        std::memcpy(&ms, &hm, sizeof(ms));
        double mchi = 0.0;
        for (int i = 0; i < C->li.Q; ++i) mchi = std::fmax(mchi, std::fabs(C->li.chi[i]));
        const double m = ms * mchi;
        int F = 0;
        if (m > 0.0 && std::isfinite(m)) F = 52 - (std::ilogb(m) + 1);
        const int F2[2] = {F, F};
        if (cudaMemcpyAsync(j->fx, F2, sizeof(F2), cudaMemcpyHostToDevice, C->stream) !=
                cudaSuccess ||
            cudaMemsetAsync(mb, 0, 8, C->stream) != cudaSuccess ||
            cudaStreamSynchronize(C->stream) != cudaSuccess)
            return PKR_ECUDA;
    }
    j->mean = *C->h_mean;
    j->lane = 0;
    j->join = C->lane[0].step;
    return PKR_OK;
}

// MIXED: move a job from the binary32 lane to the binary64 lane at a window
// boundary.  The state the next step reads is converted to binary64 and
// projected onto the zero-mass gauge (with c the mean of the latest Phi,
// c phi_i is subtracted from every population and c from Phi: the k = 0
// equilibrium mode, sum_i phi_i = 1), which removes the mass drift of the
// binary32 steps; the source is rebuilt in binary64 from rho.  The job keeps
// its age, so its check schedule and step count continue.  Its reservation
// already covers both states.  Caller holds the lock.
int promote(pkr_ctx* C, Job* j)
{
    Lane& L0 = C->lane[0];
    Lane& L1 = C->lane[1];
    const long long age = L0.step - j->join;   // age of the next step
    const int cur = (int)(age & 1);
    void* old_pop[2] = {j->pop[0], j->pop[1]};
    void* old_S = j->S;
    j->pop[0] = j->pop[1] = j->S = nullptr;
    if (!alloc_lane_state(C, j, 1)) {
        j->pop[0] = old_pop[0];
        j->pop[1] = old_pop[1];
        j->S = old_S;
        return PKR_ENOMEM;
    }
    int rc = PKR_OK;
    // mean of Phi, then the shift table c phi_i
    if (launch_rho_partials(j->Phi, j->V, C->d_scratch, kScratchBlocks, C->d_flag, C->stream) !=
            0 ||
        launch_finalize_mean(C->d_scratch, kScratchBlocks, j->V, C->d_mean, C->stream) != 0 ||
        cudaMemcpyAsync(C->h_mean, C->d_mean, sizeof(double), cudaMemcpyDeviceToHost,
                        C->stream) != cudaSuccess ||
        cudaStreamSynchronize(C->stream) != cudaSuccess)
        rc = PKR_ECUDA;
    if (rc == PKR_OK) {
        const double c = std::isfinite(*C->h_mean) ? *C->h_mean : 0.0;
        std::vector<double> shift(C->li.Q);
        for (int i = 0; i < C->li.Q; ++i) shift[i] = c * C->li.phi[i];
        if (cudaMemcpyAsync(C->d_scratch, shift.data(), shift.size() * 8, cudaMemcpyHostToDevice,
                            C->stream) != cudaSuccess)
            rc = PKR_ECUDA;
        if (rc == PKR_OK && L1.prec == PKR_FX64) {
            // into fixed point: exponent from the largest converted magnitude
            if (!j->fx && cudaMallocAsync(&j->fx, 16, C->stream) != cudaSuccess) {
                cudaGetLastError();
                j->fx = nullptr;
                rc = PKR_ECUDA;
            }
            unsigned long long* mb =
                j->fx ? reinterpret_cast<unsigned long long*>(static_cast<char*>(j->fx) + 8)
                      : nullptr;
            unsigned long long hm = 0;
            if (rc == PKR_OK &&
                (cudaMemsetAsync(mb, 0, 8, C->stream) != cudaSuccess ||
                 launch_absmax_shift(old_pop[cur], PKR_FP32, C->li.Q, j->V, C->d_scratch, nullptr,
                                     mb, C->stream) != 0 ||
                 cudaMemcpyAsync(&hm, mb, 8, cudaMemcpyDeviceToHost, C->stream) != cudaSuccess ||
                 cudaStreamSynchronize(C->stream) != cudaSuccess))
                rc = PKR_ECUDA;
            if (rc == PKR_OK) {
                double m = 0.0;
                std::memcpy(&m, &hm, sizeof(m));
                const int Fx = fx_exponent(m);
                const int F2[2] = {Fx, Fx};
                if (cudaMemcpyAsync(j->fx, F2, sizeof(F2), cudaMemcpyHostToDevice, C->stream) !=
                        cudaSuccess ||
                    cudaMemsetAsync(mb, 0, 8, C->stream) != cudaSuccess ||
                    launch_convert_fx(old_pop[cur], PKR_FP32, static_cast<long long*>(j->pop[cur]),
                                      C->li.Q, j->V, C->d_scratch, nullptr, Fx, C->stream) != 0)
                    rc = PKR_ECUDA;
            }
        } else if (rc == PKR_OK &&
                   launch_convert_shift(old_pop[cur], PKR_FP32, j->pop[cur], PKR_FP64, C->li.Q,
                                        j->V, C->d_scratch, C->stream) != 0) {
            rc = PKR_ECUDA;
        }
        if (rc == PKR_OK &&
            (launch_make_source(j->Phi, C->d_mean, 1.0, j->V, j->Phi, PKR_FP64, C->stream) != 0 ||
             cudaStreamSynchronize(C->stream) != cudaSuccess))
            rc = PKR_ECUDA;
    }
    if (rc == PKR_OK) {
        // binary64 source from rho (host rho staged in the array the next step writes)
        const double* rd = j->rho;
        if (j->host) {
            if (cudaMemcpyAsync(j->pop[cur ^ 1], j->rho, (size_t)j->V * 8,
                                cudaMemcpyHostToDevice, C->stream) != cudaSuccess)
                rc = PKR_ECUDA;
            rd = static_cast<const double*>(j->pop[cur ^ 1]);
        }
        if (rc == PKR_OK) rc = make_job_source(C, j, rd, 1);
    }
    // the binary32 state goes in every case (on an error the job fails with
    // the binary64 arrays, which free_job_memory releases)
    for (int k = 0; k < 2; ++k) cudaFreeAsync(old_pop[k], C->stream);
    cudaFreeAsync(old_S, C->stream);
    if (rc != PKR_OK) return rc;
    // release the binary32 share of the reservation
    C->used -= lane_bytes(C, 0, j->V);
    j->bytes -= lane_bytes(C, 0, j->V);
    j->lane = 1;
    j->join = L1.step - age;
    L1.live.push_back(j);
    L1.dirty = true;
    return PKR_OK;
}

// Upload the descriptors of a lane's live grids (and grow its tile partials).
int rebuild(pkr_ctx* C, Lane& L)
{
    int64_t tiles = 0;
    for (Job* j : L.live) tiles += j->ntiles;
    if (tiles > 0x7fffffff) return PKR_EINVAL;
    if (tiles > L.tiles_cap) {
        if (L.d_tile_partials) cudaFreeAsync(L.d_tile_partials, C->stream);
        L.d_tile_partials = nullptr;
        int64_t cap = tiles + tiles / 4 + 1024;
        if (cudaMallocAsync((void**)&L.d_tile_partials, (size_t)cap * 4 * sizeof(double),
                            C->stream) != cudaSuccess) {
            L.tiles_cap = 0;
            return PKR_ENOMEM;
        }
        L.tiles_cap = cap;
    }
    int tb = 0;
    for (size_t k = 0; k < L.live.size(); ++k) {
        unsigned char* dst = L.h_grids.data() + k * (size_t)L.grid_stride;
        if (L.prec == PKR_FP32) fill_grid<float>(dst, L.live[k], C->li, tb);
        else fill_grid<double>(dst, L.live[k], C->li, tb);
        tb += L.live[k]->ntiles;
    }
    L.h_state.grids = L.d_grids;
    L.h_state.tile_partials = L.d_tile_partials;
    L.h_state.grid_res = L.d_res;
    L.h_state.step = L.step;
    L.h_state.ngrids = (int)L.live.size();
    L.h_state.ntiles = (int)tiles;
    if (!L.live.empty() &&
        cudaMemcpyAsync(L.d_grids, L.h_grids.data(), L.live.size() * (size_t)L.grid_stride,
                        cudaMemcpyHostToDevice, C->stream) != cudaSuccess)
        return PKR_ECUDA;
    if (cudaMemcpyAsync(L.d_state, &L.h_state, sizeof(BatchState), cudaMemcpyHostToDevice,
                        C->stream) != cudaSuccess ||
        cudaStreamSynchronize(C->stream) != cudaSuccess)
        return PKR_ECUDA;
    L.dirty = false;
    return PKR_OK;
}

// Queue one window of a lane (K steps + reduction + residual copy).
int enqueue_window(pkr_ctx* C, Lane& L)
{
    for (int k = 0; k < C->K; ++k) {
        if (launch_batch_step(C->cfg.lattice, L.prec, L.variant, L.d_state, C->K, L.grid,
                              C->stream) != 0 ||
            (L.prec == PKR_FX64 &&
             launch_batch_fx_rescale(L.d_state, C->max_grids, C->stream) != 0) ||
            launch_batch_increment(L.d_state, C->stream) != 0)
            return PKR_ECUDA;
    }
    if (launch_batch_reduce(L.d_state, C->max_grids, L.grid_stride, C->stream) != 0 ||
        cudaMemcpyAsync(L.h_res, L.d_res, (size_t)C->max_grids * 4 * sizeof(double),
                        cudaMemcpyDeviceToHost, C->stream) != cudaSuccess)
        return PKR_ECUDA;
    return PKR_OK;
}

// Launch a lane's window (its captured graph; captured on first use).
int launch_window(pkr_ctx* C, Lane& L)
{
    if (!L.graph) {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal) ==
                  cudaSuccess;
        int rc = ok ? enqueue_window(C, L) : PKR_ECUDA;
        if (ok) ok = cudaStreamEndCapture(C->stream, &g) == cudaSuccess && rc == PKR_OK;
        if (ok) ok = cudaGraphInstantiate(&L.graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            L.graph = nullptr;
        }
    }
    if (L.graph) return cudaGraphLaunch(L.graph, C->stream) == cudaSuccess ? PKR_OK : PKR_ECUDA;
    return enqueue_window(C, L);
}

// Retire (or promote) the grids of lane ln whose check at the end of the
// window just run decided them.  Caller holds the lock.
int retire(pkr_ctx* C, int ln, long long step0)
{
    Lane& L = C->lane[ln];
    std::vector<Job*> keep;
    bool changed = false;
    for (size_t k = 0; k < L.live.size(); ++k) {
        Job* j = L.live[k];
        const long long age_end = L.step - 1 - j->join;    // age of the window's last step
        C->site_updates += (double)j->V * (double)(L.step - (step0 > j->join ? step0 : j->join));
        const bool checked = age_end >= 1;
        const double* r = L.h_res + 4 * k;
        const double res = r[j->prob.tol_kind == PKR_TOL_MAX_ABS_DPHI ? 0 : 1];
        const double tol = j->prob.tol;
        int status = PKR_EBUSY;
        bool move = false;
        if (checked) {
            if (!std::isfinite(r[0]) || !std::isfinite(r[2])) {
                status = PKR_EDIVERGED;
            } else if (C->mixed && ln == 0 && tol > 0.0 && tol < PKR_MIXED_SWITCH_TOL) {
                // binary32 lane: hand over at the switch tolerance, or once
                // the residual stops falling (the binary32 rounding floor)
                if ((res < PKR_MIXED_SWITCH_TOL || (res >= j->prev_res && res < 1e-3)) &&
                    age_end < j->prob.max_sweeps)
                    move = true;
                j->prev_res = res;
            } else if (tol > 0.0 && res < tol) {
                status = PKR_OK;
            }
            if (status == PKR_EBUSY && !move && age_end >= j->prob.max_sweeps)
                status = (tol > 0.0) ? PKR_ENOCONV : PKR_OK;
        }
        if (move) {
            const int rc = promote(C, j);
            if (rc == PKR_OK) {
                changed = true;
                continue;
            }
            if (rc != PKR_ENOMEM) status = rc;   // else: device memory short, stay in binary32
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
        j->st.variant = L.variant;
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
    L.live.swap(keep);
    if (changed) L.dirty = true;
    return PKR_OK;
}

// One scheduling round (caller holds the lock): admit, run a window of every
// lane with live grids, retire/promote.  Returns 1 if work was done, 0 if
// idle, < 0 on a CUDA error.
int round(pkr_ctx* C, std::unique_lock<std::mutex>& lk)
{
    // admit (first fit, FIFO order) while memory and descriptor slots allow
    Lane& L0 = C->lane[0];
    for (auto it = C->queue.begin(); it != C->queue.end();) {
        Job* j = *it;
        // descriptor slots: a job lives in one lane at a time, so the lanes
        // together never hold more than max_grids
        if ((int)(L0.live.size() + C->lane[1].live.size()) >= C->max_grids) break;
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
        L0.live.push_back(j);
        L0.dirty = true;
    }
    bool any = false;
    for (int ln = 0; ln < C->nlanes; ++ln) any = any || !C->lane[ln].live.empty();
    if (!any) {
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
    bool ran[2] = {false, false};
    for (int ln = 0; ln < C->nlanes; ++ln) {
        Lane& L = C->lane[ln];
        if (L.live.empty()) continue;
        if (L.dirty && rebuild(C, L) != PKR_OK) return -1;
        ran[ln] = true;
    }
    // the windows run without the lock so that submissions and polls proceed
    const bool inject = C->rounds++ == C->fail_round;
    lk.unlock();
    int rc = inject ? PKR_ECUDA : PKR_OK;
    for (int ln = 0; ln < C->nlanes && rc == PKR_OK; ++ln)
        if (ran[ln]) rc = launch_window(C, C->lane[ln]);
    if (rc == PKR_OK && cudaStreamSynchronize(C->stream) != cudaSuccess) rc = PKR_ECUDA;
    lk.lock();
    if (rc != PKR_OK) return -1;
    // binary64 lane first, so that grids promoted in this scheduling round wait for the next window
    for (int ln = C->nlanes - 1; ln >= 0; --ln) {
        if (!ran[ln]) continue;
        Lane& L = C->lane[ln];
        const long long step0 = L.step;
        L.step += C->K;
        C->windows += 1;
        retire(C, ln, step0);
    }
    return 1;
}

// After a failed round: every live and queued request finishes with
// PKR_ECUDA, and the live ones give their device memory (and their share of
// the budget) back, so that a finished request holds nothing.  The stream is
// drained first; after a sticky error nothing more runs on it anyway.
void fail_all(pkr_ctx* C)
{
    cudaStreamSynchronize(C->stream);
    for (int ln = 0; ln < C->nlanes; ++ln) {
        for (Job* j : C->lane[ln].live) {
            free_job_memory(C, j);
            finish(C, j, PKR_ECUDA);
        }
        C->lane[ln].live.clear();
        C->lane[ln].dirty = true;
    }
    for (Job* j : C->queue) finish(C, j, PKR_ECUDA);   // queued requests hold no memory
    C->queue.clear();
    cudaStreamSynchronize(C->stream);
    cudaGetLastError();
}

// One round of a non-threaded context, driven by the calling thread (the
// caller holds the lock and has checked that no other thread drives).
int drive_round(pkr_ctx* C, std::unique_lock<std::mutex>& lk)
{
    C->driving = true;
    int r = round(C, lk);
    if (r < 0) fail_all(C);
    C->driving = false;
    C->cv_done.notify_all();
    return r;
}

void worker_main(pkr_ctx* C)
{
    cudaSetDevice(C->device);
    std::unique_lock<std::mutex> lk(C->mu);
    while (!C->stop) {
        int r = round(C, lk);
        if (r < 0) {
            // a CUDA error: fail everything that is queued or live
            fail_all(C);
            continue;
        }
        if (r == 0) C->cv_work.wait(lk, [&] { return C->stop || !C->queue.empty(); });
    }
}

int tune_variant(pkr_ctx* C, Lane& L, int edge);

bool init_lane(pkr_ctx* C, Lane& L, int prec)
{
    L.prec = prec;
    L.elem = prec == PKR_FP32 ? 4 : 8;
    L.grid_stride = prec == PKR_FP32 ? (int)sizeof(BatchGrid<float>)
                                     : (int)sizeof(BatchGrid<double>);
    L.h_grids.assign((size_t)C->max_grids * L.grid_stride, 0);
    std::memset(&L.h_state, 0, sizeof(BatchState));
    return cudaMalloc((void**)&L.d_state, sizeof(BatchState)) == cudaSuccess &&
           cudaMalloc((void**)&L.d_grids, (size_t)C->max_grids * L.grid_stride) == cudaSuccess &&
           cudaMalloc((void**)&L.d_res, (size_t)C->max_grids * 4 * sizeof(double)) ==
               cudaSuccess &&
           cudaMallocHost((void**)&L.h_res, (size_t)C->max_grids * 4 * sizeof(double)) ==
               cudaSuccess &&
           cudaMemcpy(L.d_state, &L.h_state, sizeof(BatchState), cudaMemcpyHostToDevice) ==
               cudaSuccess;
}

void free_lane(Lane& L)
{
    if (L.graph) cudaGraphExecDestroy(L.graph);
    cudaFree(L.d_state);
    cudaFree(L.d_grids);
    cudaFree(L.d_res);
    if (L.d_tile_partials) cudaFree(L.d_tile_partials);
    if (L.h_res) cudaFreeHost(L.h_res);
    L = Lane();
}

}  // namespace

extern "C" {

int pkr_ctx_create(const pkr_ctx_config* cfg, void* stream, pkr_ctx** out)
{
    if (!cfg || !out) return PKR_EINVAL;
    *out = nullptr;
    if (cfg->check_every < 1 || cfg->hbm_budget_bytes == 0) return PKR_EINVAL;
    if (cfg->precision != PKR_FP64 && cfg->precision != PKR_FP32 &&
        cfg->precision != PKR_MIXED && cfg->precision != PKR_FX64 &&
        cfg->precision != PKR_MIXED_FX64)
        return PKR_EINVAL;
    LatticeInfo li;
    int rc = build_lattice(cfg->lattice, cfg->order, &li);
    if (rc != PKR_OK) return rc;
    const int nvar = batch_variant_count(cfg->lattice);
    if (cfg->variant >= nvar || cfg->variant < -2) return PKR_EINVAL;
    pkr_ctx* C = new (std::nothrow) pkr_ctx();
    if (!C) return PKR_ENOMEM;
    C->cfg = *cfg;
    C->li = li;
    C->stream = (cudaStream_t)stream;
    C->K = cfg->check_every;
    C->budget = cfg->hbm_budget_bytes;
    C->max_grids = cfg->max_grids > 0 ? cfg->max_grids : 4096;
    C->mixed = cfg->precision == PKR_MIXED || cfg->precision == PKR_MIXED_FX64;
    if (const char* fr = std::getenv("PKR_TEST_FAIL_ROUND")) C->fail_round = std::atoll(fr);
    C->nlanes = C->mixed ? 2 : 1;
    bool ok = cudaGetDevice(&C->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&C->nsm, cudaDevAttrMultiProcessorCount, C->device) ==
                  cudaSuccess &&
              cudaMalloc((void**)&C->d_scratch, kScratchBlocks * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&C->d_flag, sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&C->d_mean, sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void**)&C->h_flag, sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void**)&C->h_mean, sizeof(double)) == cudaSuccess;
    const int precs[2] = {C->mixed ? PKR_FP32 : cfg->precision,
                          cfg->precision == PKR_MIXED_FX64 ? PKR_FX64 : PKR_FP64};
    for (int ln = 0; ok && ln < C->nlanes; ++ln) ok = init_lane(C, C->lane[ln], precs[ln]);
    if (!ok) {
        cudaGetLastError();
        pkr_ctx_destroy(C);
        return PKR_ENOMEM;
    }
    for (int ln = 0; ln < C->nlanes; ++ln) {
        Lane& L = C->lane[ln];
        int var = cfg->variant;
        if (var == -2) {
            var = tune_variant(C, L, cfg->probe_edge > 0 ? cfg->probe_edge : 64);
            if (var < 0) {
                pkr_ctx_destroy(C);
                return PKR_ECUDA;
            }
        } else if (var == -1) {
            var = nvar > 2 ? 2 : 0;
        }
        L.variant = var;
        int bps = 0;
        if (batch_occupancy(cfg->lattice, L.prec, var, &bps) != 0 || bps < 1) {
            pkr_ctx_destroy(C);
            return PKR_ECUDA;
        }
        L.grid = C->nsm * bps;
    }
    if (cfg->threaded) C->worker = std::thread(worker_main, C);
    *out = C;
    return PKR_OK;
}

int pkr_batch_variant_count(int lattice) { return batch_variant_count(lattice); }

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
        // drive rounds until the request finishes; while another thread
        // drives, wait for its round to end (the request stays registered as
        // waited on, so that pkr_ctx_release cannot delete it meanwhile)
        j->waiters += 1;
        while (j->status == PKR_EBUSY) {
            if (C->driving) {
                C->cv_done.wait(lk);
                continue;
            }
            const int r = drive_round(C, lk);
            if (r == 0 && j->status == PKR_EBUSY) {
                j->waiters -= 1;
                return PKR_EINVAL;
            }
        }
        j->waiters -= 1;
    } else {
        j->waiters += 1;
        C->cv_done.wait(lk, [&] { return j->status != PKR_EBUSY || C->stop; });
        j->waiters -= 1;
    }
    if (st && j->status != PKR_EBUSY) *st = j->st;
    return j->status;
}
int pkr_ctx_release(pkr_ctx* C, uint64_t ticket)
{
    if (!C) return PKR_EINVAL;
    std::lock_guard<std::mutex> lk(C->mu);
    auto it = C->jobs.find(ticket);
    if (it == C->jobs.end()) return PKR_EINVAL;
    Job* j = it->second;
    // a finished request holds no device memory (retire and fail_all free
    // it) and sits in no queue or lane
    if (j->status == PKR_EBUSY || j->waiters > 0) return PKR_EBUSY;
    C->jobs.erase(it);
    delete j;
    return PKR_OK;
}

int pkr_ctx_run(pkr_ctx* C, int64_t max_windows)
{
    if (!C || C->cfg.threaded) return PKR_EINVAL;
    std::unique_lock<std::mutex> lk(C->mu);
    int64_t n = 0;
    while (max_windows <= 0 || n < max_windows) {
        if (C->driving) {   // another thread runs a round: wait for it to end
            C->cv_done.wait(lk);
            continue;
        }
        const int r = drive_round(C, lk);
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
    if (variant) *variant = C->lane[0].variant;
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
    if (C->stream || C->lane[0].d_state) cudaStreamSynchronize(C->stream);
    for (auto& kv : C->jobs) {
        Job* j = kv.second;
        for (int k = 0; k < 2; ++k)
            if (j->pop[k]) cudaFree(j->pop[k]);
        if (j->S) cudaFree(j->S);
        if (j->Phi) cudaFree(j->Phi);
        if (j->fx) cudaFree(j->fx);
        delete j;
    }
    for (int ln = 0; ln < 2; ++ln) free_lane(C->lane[ln]);
    cudaFree(C->d_scratch);
    cudaFree(C->d_flag);
    cudaFree(C->d_mean);
    if (C->h_flag) cudaFreeHost(C->h_flag);
    if (C->h_mean) cudaFreeHost(C->h_mean);
    delete C;
    return PKR_OK;
}

}  // extern "C"

namespace {

// Autotuner of a lane's batch geometry: time three steps of every compiled
// variant on a probe grid (edge^3, zero source) in the lane's batch layout,
// keep the fastest.  Runs at context creation, before any request, so that
// every request of the context sees the same kernels.
int tune_variant(pkr_ctx* C, Lane& L, int edge)
{
    const int nvar = batch_variant_count(C->cfg.lattice);
    Job probe;
    probe.prob.n[0] = edge;
    probe.prob.n[1] = C->li.dim >= 2 ? edge : 1;
    probe.prob.n[2] = C->li.dim >= 3 ? edge : 1;
    probe.V = probe.prob.n[0] * probe.prob.n[1] * probe.prob.n[2];
    probe.ntiles = (int)((probe.V + 31) / 32);
    probe.omega = 0.5;
    for (int k = 0; k < C->li.dim; ++k)
        if (probe.prob.n[k] < C->li.reach) probe.small = 1;
    const size_t popb = (size_t)C->li.Q * (size_t)probe.V * (size_t)L.elem;
    if (cudaMalloc(&probe.pop[0], popb) != cudaSuccess ||
        cudaMalloc(&probe.pop[1], popb) != cudaSuccess ||
        cudaMalloc(&probe.S, (size_t)probe.V * L.elem) != cudaSuccess ||
        cudaMalloc((void**)&probe.Phi, (size_t)probe.V * 8) != cudaSuccess) {
        cudaGetLastError();
        for (int k = 0; k < 2; ++k) cudaFree(probe.pop[k]);
        cudaFree(probe.S);
        cudaFree(probe.Phi);
        return -1;
    }
    cudaMemset(probe.pop[0], 0, popb);
    cudaMemset(probe.pop[1], 0, popb);
    cudaMemset(probe.S, 0, (size_t)probe.V * L.elem);
    if (L.prec == PKR_FX64) {   // zero exponents and bound for the probe's fixed-point steps
        if (cudaMalloc(&probe.fx, 16) != cudaSuccess) {
            cudaGetLastError();
            for (int k = 0; k < 2; ++k) cudaFree(probe.pop[k]);
            cudaFree(probe.S);
            cudaFree(probe.Phi);
            return -1;
        }
        cudaMemset(probe.fx, 0, 16);
    }
    probe.join = -1;   // never the zero-in step: the timed steps pull real data
    L.live.push_back(&probe);
    int best = -1;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (rebuild(C, L) == PKR_OK) {
        for (int v = 0; v < nvar; ++v) {
            int bps = 0;
            if (batch_occupancy(C->cfg.lattice, L.prec, v, &bps) != 0 || bps < 1) continue;
            const int grid = C->nsm * bps;
            launch_batch_step(C->cfg.lattice, L.prec, v, L.d_state, 1 << 30, grid, C->stream);
            cudaEventRecord(e0, C->stream);
            for (int k = 0; k < 3; ++k)
                launch_batch_step(C->cfg.lattice, L.prec, v, L.d_state, 1 << 30, grid,
                                  C->stream);
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
    L.live.clear();
    L.dirty = true;
    L.step = 0;
    std::memset(&L.h_state, 0, sizeof(BatchState));
    cudaMemcpy(L.d_state, &L.h_state, sizeof(BatchState), cudaMemcpyHostToDevice);
    for (int k = 0; k < 2; ++k) cudaFree(probe.pop[k]);
    cudaFree(probe.S);
    cudaFree(probe.Phi);
    cudaFree(probe.fx);
    probe.pop[0] = probe.pop[1] = probe.S = nullptr;
    probe.Phi = nullptr;
    probe.fx = nullptr;
    return best;
}

}  // namespace
