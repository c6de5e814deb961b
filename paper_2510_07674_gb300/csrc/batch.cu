// Batched form of the two-stage solve (not in the paper: the throughput form of the hot path
// for many independent problems).  The first attempt of stage 1 of every problem is one CUDA
// graph; stage 2 (lift of every problem, one persistent launch of the trajectory kernel over
// the particles of all problems, selection and FP64 check of every problem) is a second
// graph.  The rare problem that needs a further attempt continues alone on its own stream
// with the code of spasm_optimize.  Every particle runs the same arithmetic as in the
// single-problem launches, so each problem's result equals its spasm_optimize result.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "problem.h"

using namespace spasm;

namespace {

// Capture what `enqueue` puts on stream s into a graph, run it once and wait for it.
template <typename F>
spasm_status run_as_graph(cudaStream_t s, F enqueue) {
    SPASM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    const spasm_status st = enqueue();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != SPASM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (x) cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return SPASM_OK;
}

struct PinnedInts {
    int* p = nullptr;
    ~PinnedInts() {
        if (p) cudaFreeHost(p);
    }
};

spasm_status check_batch(spasm_problem_t* prs, int n, void* stream) {
    if (!prs || n < 1 || n > 4096) return fail(SPASM_ERR_INVALID, "batch of 1..4096 problems expected");
    if (!stream) return fail(SPASM_ERR_INVALID, "the batched form needs a created (non-default) stream for graph capture");
    for (int i = 0; i < n; ++i) {
        if (!prs[i]) return fail(SPASM_ERR_INVALID, "null problem in the batch");
        if (prs[i]->sc.kind == kKindPack)
            return fail(SPASM_ERR_INVALID, "the batched form solves tower and point-to-point problems");
        for (int j = 0; j < i; ++j)
            if (prs[j] == prs[i]) return fail(SPASM_ERR_INVALID, "a problem appears twice in the batch");
    }
    return SPASM_OK;
}

// Stage 1 of every problem not yet placed: attempt 0 of all of them as one graph, then any
// further attempts per problem.  status[i] records each problem's outcome.
spasm_status place_all(spasm_problem_t* prs, int n, cudaStream_t s, std::vector<spasm_status>& status) {
    std::vector<int> todo;
    for (int i = 0; i < n; ++i)
        if (!prs[i]->placed) todo.push_back(i);
    status.assign(n, SPASM_OK);
    if (todo.empty()) return SPASM_OK;
    PinnedInts h;
    SPASM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h.p), sizeof(int) * n));
    SPASM_TRY(run_as_graph(s, [&]() -> spasm_status {
        for (int i : todo) {
            SPASM_TRY(place_attempt(prs[i], 0u, s));
            SPASM_CUDA(cudaMemcpyAsync(&h.p[i], prs[i]->d_nsat, sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        return SPASM_OK;
    }));
    for (int i : todo) {
        spasm_problem* pr = prs[i];
        pr->stats.d2h_bytes += sizeof(int);
        const spasm_status st = place_continue(pr, 1, pr->sc.K_lin + pr->sc.K_quad, h.p[i]);
        if (st != SPASM_OK && st != SPASM_ERR_NOSOLUTION) return st;
        status[i] = st;
    }
    return SPASM_OK;
}

// Work list of a batched trajectory launch over the problems `live` (in `order`).
struct JobList {
    std::vector<TrajJob> jobs;
    int n_items = 0;
    size_t smem = 0;
};

JobList make_jobs(spasm_problem_t* prs, const std::vector<int>& live, int per_fetch, int mode, int k_steps,
                  bool init_multipliers) {
    JobList L;
    for (int i : live) {
        spasm_problem* pr = prs[i];
        TrajJob j{};
        j.sc = pr->d_sc;
        j.tab = pr->tab;
        j.io.q = pr->d_q;
        if (mode == kTrajModeDescend) {
            j.io.lam = pr->d_lam; j.io.mu = pr->d_mu; j.io.metrics = pr->d_metrics; j.io.sat = pr->d_tsat;
            j.io.tests = pr->d_tests;
        }
        j.io.k_steps = k_steps;
        j.io.init_multipliers = init_multipliers ? 1 : 0;
        j.err = pr->d_err;
        j.n = pr->sc.Q;
        j.first = L.n_items;
        L.n_items += (pr->sc.Q + per_fetch - 1) / per_fetch;
        L.smem = std::max(L.smem, traj_smem_bytes(pr->sc));
        L.jobs.push_back(j);
    }
    return L;
}

// Problems in the order the schedule takes them: as given, or largest trajectory work
// (particles x configurations) first, so that small problems fill the tail of the launch.
std::vector<int> job_order(spasm_problem_t* prs, const std::vector<int>& live, int order) {
    std::vector<int> v = live;
    if (order == 0)
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
            return (long long)prs[a]->sc.Q * prs[a]->sc.C > (long long)prs[b]->sc.Q * prs[b]->sc.C;
        });
    return v;
}

struct DeviceJobs {
    TrajJob* jobs = nullptr;
    int* next = nullptr;
    cudaStream_t s = nullptr;
    ~DeviceJobs() {
        if (jobs) cudaFreeAsync(jobs, s);
        if (next) cudaFreeAsync(next, s);
    }
};

spasm_status upload_jobs(const JobList& L, cudaStream_t s, DeviceJobs& d) {
    d.s = s;
    SPASM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d.jobs), sizeof(TrajJob) * L.jobs.size(), s));
    SPASM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d.next), sizeof(int), s));
    SPASM_CUDA(cudaMemcpyAsync(d.jobs, L.jobs.data(), sizeof(TrajJob) * L.jobs.size(), cudaMemcpyHostToDevice, s));
    SPASM_CUDA(cudaStreamSynchronize(s));
    return SPASM_OK;
}

spasm_status batch_grid(const spasm_batch_config& cfg, size_t smem, int* grid) {
    int dev = 0, sms = 0;
    SPASM_CUDA(cudaGetDevice(&dev));
    SPASM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int resident = traj_batch_ctas_per_sm(smem);
    if (resident < 1) return fail(SPASM_ERR_INVALID, "batched trajectory kernel does not fit this shared-memory size");
    const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, resident) : resident;
    *grid = per_sm * sms;
    return SPASM_OK;
}

spasm_status check_config(const spasm_batch_config& c) {
    if (c.per_fetch < 1 || c.per_fetch > 64 || c.ctas_per_sm < 0 || c.ctas_per_sm > 8 || c.order < 0 || c.order > 1)
        return fail(SPASM_ERR_INVALID, "batch config outside per_fetch 1..64, ctas_per_sm 0..8, order 0..1");
    return SPASM_OK;
}

}  // namespace

extern "C" spasm_status spasm_batch_default_config(spasm_batch_config* cfg) {
    if (!cfg) return fail(SPASM_ERR_INVALID, "null config");
    cfg->per_fetch = 1;
    cfg->ctas_per_sm = 0;
    cfg->order = 0;
    return SPASM_OK;
}

extern "C" spasm_status spasm_optimize_batch(spasm_problem_t* prs, int n, void* cuda_stream,
                                             const spasm_batch_config* cfg_in) {
    SPASM_TRY(check_batch(prs, n, cuda_stream));
    spasm_batch_config cfg;
    spasm_batch_default_config(&cfg);
    if (cfg_in) cfg = *cfg_in;
    SPASM_TRY(check_config(cfg));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    for (int i = 0; i < n; ++i) SPASM_CUDA(cudaStreamSynchronize(prs[i]->stream));

    std::vector<spasm_status> status;
    SPASM_TRY(place_all(prs, n, s, status));
    std::vector<int> live;
    for (int i = 0; i < n; ++i)
        if (status[i] == SPASM_OK && prs[i]->n_place > 0) live.push_back(i);
    if (live.empty()) return SPASM_OK;

    const std::vector<int> order = job_order(prs, live, cfg.order);
    JobList L = make_jobs(prs, order, cfg.per_fetch, kTrajModeDescend, 0, true);
    for (size_t k = 0; k < order.size(); ++k) L.jobs[k].io.k_steps = prs[order[k]]->sc.K_traj;
    int grid = 0;
    SPASM_TRY(batch_grid(cfg, L.smem, &grid));
    DeviceJobs dj;
    SPASM_TRY(upload_jobs(L, s, dj));
    PinnedInts h;
    SPASM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h.p), sizeof(int) * n));
    SPASM_TRY(run_as_graph(s, [&]() -> spasm_status {
        for (int i : live) {
            spasm_problem* pr = prs[i];
            SPASM_CUDA(cudaMemsetAsync(pr->d_tests, 0, 3 * sizeof(unsigned long long), s));
            SPASM_CUDA(launch_lift(pr->sc, pr->sc.Q, pr->d_place, pr->n_place, 0u, pr->d_q, s));
        }
        SPASM_CUDA(cudaMemsetAsync(dj.next, 0, sizeof(int), s));
        SPASM_CUDA(launch_traj_batch(dj.jobs, (int)L.jobs.size(), L.n_items, cfg.per_fetch, kTrajModeDescend, dj.next,
                                     L.smem, grid, s));
        for (int i : live) {
            spasm_problem* pr = prs[i];
            SPASM_TRY(traj_select(pr, s));
            SPASM_CUDA(cudaMemcpyAsync(&h.p[i], pr->d_tnsat, sizeof(int), cudaMemcpyDeviceToHost, s));
            SPASM_TRY(finish_enqueue(pr, s));
        }
        return SPASM_OK;
    }));
    for (int i : live) {
        spasm_problem* pr = prs[i];
        const Scalars& sc = pr->sc;
        count_launches(pr, 2);   // its lift; the shared trajectory launch belongs to no single problem
        pr->stats.traj_launches += 1;
        pr->stats.particle_iters += (long long)sc.Q * sc.K_traj;
        pr->stats.d2h_bytes += sizeof(int);
        int found = 0;
        spasm_status st;
        if (h.p[i] > 0) {
            found = h.p[i] < sc.P ? h.p[i] : sc.P;
            pr->traj_attempts = 1;
            pr->stats.traj_attempts += 1;
            st = finish_record(pr, found, true);
        } else {
            pr->stats.traj_attempts -= 1;   // traj_continue counts the batched attempt again
            SPASM_TRY(traj_continue(pr, 1, sc.K_traj, 0, &found));
            st = finish_record(pr, found, false);
        }
        if (st != SPASM_OK && st != SPASM_ERR_NOSOLUTION) return st;
    }
    return SPASM_OK;
}

extern "C" spasm_status spasm_batch_autotune(spasm_problem_t* prs, int n, void* cuda_stream, spasm_batch_config* best,
                                             double* best_ms) {
    SPASM_TRY(check_batch(prs, n, cuda_stream));
    if (!best) return fail(SPASM_ERR_INVALID, "null config");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    for (int i = 0; i < n; ++i) SPASM_CUDA(cudaStreamSynchronize(prs[i]->stream));
    std::vector<spasm_status> status;
    SPASM_TRY(place_all(prs, n, s, status));
    std::vector<int> live;
    for (int i = 0; i < n; ++i)
        if (status[i] == SPASM_OK && prs[i]->n_place > 0) live.push_back(i);
    spasm_batch_default_config(best);
    if (best_ms) *best_ms = 0.0;
    if (live.empty()) return SPASM_OK;
    // the candidates run one evaluation of every lifted particle (no writes besides q's reads)
    for (int i : live) {
        spasm_problem* pr = prs[i];
        SPASM_CUDA(launch_lift(pr->sc, pr->sc.Q, pr->d_place, pr->n_place, 0u, pr->d_q, s));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPASM_CUDA(cudaEventCreate(&e0));
    SPASM_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    double best_t = 1e300;
    const int fetches[] = {1, 2, 4};
    for (int order = 0; order <= 1; ++order) {
        for (int pf : fetches) {
            for (int per_sm : {0, 1}) {
                spasm_batch_config c{pf, per_sm, order};
                JobList L = make_jobs(prs, job_order(prs, live, order), pf, kTrajModeEval, 0, true);
                int grid = 0;
                SPASM_TRY(batch_grid(c, L.smem, &grid));
                DeviceJobs dj;
                SPASM_TRY(upload_jobs(L, s, dj));
                double t = 1e300;
                for (int rep = 0; rep < 2; ++rep) {   // the first repetition warms caches
                    SPASM_CUDA(cudaMemsetAsync(dj.next, 0, sizeof(int), s));
                    SPASM_CUDA(cudaEventRecord(e0, s));
                    SPASM_CUDA(launch_traj_batch(dj.jobs, (int)L.jobs.size(), L.n_items, pf, kTrajModeEval, dj.next,
                                                 L.smem, grid, s));
                    SPASM_CUDA(cudaEventRecord(e1, s));
                    SPASM_CUDA(cudaEventSynchronize(e1));
                    if (rep > 0) t = ev_ms(e0, e1);
                }
                if (t < best_t) { best_t = t; *best = c; }
            }
        }
    }
    for (int i : live) SPASM_TRY(check_device_error(prs[i]));
    if (best_ms) *best_ms = best_t;
    return SPASM_OK;
}
