// Batched form of the two-stage solve (not in the paper: the throughput form of the hot path
// for many independent problems).  One CUDA graph holds the whole batch: stage 1 of every
// problem not yet placed (each with its own device-side attempt loop, in parallel branches),
// the first stage-2 lift of every problem, one persistent launch of the trajectory kernel
// over the particles of all problems, then per problem (in parallel branches) the
// satisfying selection, its device-side re-lift loop and the FP64 check.  Every particle
// runs the same arithmetic as in the single-problem launches, so each problem's result
// equals its spasm_optimize result.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "problem.h"

using namespace spasm;

namespace {

// Parallel branches of a capture on stream s: fork() makes every branch stream depend on
// s's work so far, join() makes s depend on everything the branches enqueued since.
struct Branches {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ev;
    cudaStream_t s = nullptr;
    ~Branches() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaStream_t b : st) cudaStreamDestroy(b);
    }
    spasm_status init(cudaStream_t main, int n) {
        s = main;
        for (int i = 0; i < n; ++i) {
            cudaStream_t b = nullptr;
            SPASM_CUDA(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
            st.push_back(b);
        }
        return SPASM_OK;
    }
    spasm_status event(cudaEvent_t* e) {
        SPASM_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        ev.push_back(*e);
        return SPASM_OK;
    }
    spasm_status fork() {
        cudaEvent_t e;
        SPASM_TRY(event(&e));
        SPASM_CUDA(cudaEventRecord(e, s));
        for (cudaStream_t b : st) SPASM_CUDA(cudaStreamWaitEvent(b, e, 0));
        return SPASM_OK;
    }
    spasm_status join() {
        for (cudaStream_t b : st) {
            cudaEvent_t e;
            SPASM_TRY(event(&e));
            SPASM_CUDA(cudaEventRecord(e, b));
            SPASM_CUDA(cudaStreamWaitEvent(s, e, 0));
        }
        return SPASM_OK;
    }
    cudaStream_t operator[](size_t i) const { return st[i % st.size()]; }
};

constexpr int kMaxBranches = 16;

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

// Captures `enqueue` (given the capture stream) into a graph, launches it on `launch_on`.
template <typename F>
spasm_status run_graph(cudaStream_t launch_on, F enqueue) {
    cudaStream_t cap = nullptr;
    SPASM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    struct S { cudaStream_t c; ~S() { cudaStreamDestroy(c); } } guard{cap};
    SPASM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    const spasm_status st = enqueue(cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st != SPASM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, launch_on);
    // the executable graph is released only after its launch has finished
    if (e == cudaSuccess) e = cudaStreamSynchronize(launch_on);
    if (x) cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return SPASM_OK;
}

// Stage 1 (with its device-side attempt loop) of the problems `todo`, in parallel branches
// of the capture on s (br: not yet initialised; it must outlive the capture).
spasm_status enqueue_place_all(spasm_problem_t* prs, const std::vector<int>& todo, cudaStream_t s, Branches& br) {
    if (todo.empty()) return SPASM_OK;
    SPASM_TRY(br.init(s, std::min<int>((int)todo.size(), kMaxBranches)));
    SPASM_TRY(br.fork());
    for (size_t k = 0; k < todo.size(); ++k) SPASM_TRY(enqueue_place(prs[todo[k]], br[k]));
    return br.join();
}

void mark_placed(spasm_problem_t* prs, const std::vector<int>& todo) {
    for (int i : todo) {
        prs[i]->placed = true;
        prs[i]->place_pending = true;
        prs[i]->place_timed = false;
    }
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
            j.io.active = &pr->d_ctl->n_place;
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
    const int resident = traj_batch_ctas_per_sm(smem, cfg.sphere_tiling, cfg.particles_per_cta);
    if (resident < 1) return fail(SPASM_ERR_INVALID, "batched trajectory kernel does not fit this shared-memory size");
    const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, resident) : resident;
    *grid = per_sm * sms;
    return SPASM_OK;
}

spasm_status check_config(const spasm_batch_config& c) {
    if (c.per_fetch < 1 || c.per_fetch > 64 || c.ctas_per_sm < 0 || c.ctas_per_sm > 8 || c.order < 0 || c.order > 1 ||
        c.sphere_tiling < 0 || c.sphere_tiling > 1 || c.particles_per_cta < 1 || c.particles_per_cta > 2)
        return fail(SPASM_ERR_INVALID, "batch config outside per_fetch 1..64, ctas_per_sm 0..8, order 0..1, "
                                       "sphere_tiling 0..1, particles_per_cta 1..2");
    return SPASM_OK;
}

}  // namespace

spasm::BatchLaunch::~BatchLaunch() {
    if (jobs) cudaFreeAsync(jobs, s);
    if (next) cudaFreeAsync(next, s);
}

spasm_status spasm::prepare_batch(spasm_problem_t* prs, const std::vector<int>& order, const spasm_batch_config& cfg,
                                  cudaStream_t s, BatchLaunch& bl) {
    SPASM_TRY(check_config(cfg));
    JobList L = make_jobs(prs, order, cfg.per_fetch, kTrajModeDescend, 0, true);
    for (size_t k = 0; k < order.size(); ++k) L.jobs[k].io.k_steps = prs[order[k]]->sc.K_traj;
    SPASM_TRY(batch_grid(cfg, L.smem, &bl.grid));
    bl.host = std::move(L.jobs);
    bl.n_items = L.n_items;
    bl.smem = L.smem;
    bl.per_fetch = cfg.per_fetch;
    bl.tiling = cfg.sphere_tiling;
    bl.ppc = cfg.particles_per_cta;
    bl.s = s;
    SPASM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&bl.jobs), sizeof(TrajJob) * bl.host.size(), s));
    SPASM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&bl.next), sizeof(int), s));
    SPASM_CUDA(cudaMemcpyAsync(bl.jobs, bl.host.data(), sizeof(TrajJob) * bl.host.size(), cudaMemcpyHostToDevice, s));
    return SPASM_OK;
}

spasm_status spasm::enqueue_batch(const BatchLaunch& bl, cudaStream_t s) {
    SPASM_CUDA(cudaMemsetAsync(bl.next, 0, sizeof(int), s));
    SPASM_CUDA(launch_traj_batch(bl.jobs, (int)bl.host.size(), bl.n_items, bl.per_fetch, kTrajModeDescend, bl.next,
                                 bl.smem, bl.grid, s, bl.tiling, bl.ppc));
    return SPASM_OK;
}

extern "C" spasm_status spasm_batch_default_config(spasm_batch_config* cfg) {
    if (!cfg) return fail(SPASM_ERR_INVALID, "null config");
    cfg->per_fetch = 1;
    cfg->ctas_per_sm = 0;
    cfg->order = 0;
    cfg->sphere_tiling = 0;
    cfg->particles_per_cta = 1;
    return SPASM_OK;
}

extern "C" spasm_status spasm_optimize_batch(spasm_problem_t* prs, int n, void* cuda_stream,
                                             const spasm_batch_config* cfg_in) {
    Range r("spasm_optimize_batch");
    SPASM_TRY(check_batch(prs, n, cuda_stream));
    spasm_batch_config cfg;
    spasm_batch_default_config(&cfg);
    if (cfg_in) cfg = *cfg_in;
    SPASM_TRY(check_config(cfg));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<int> todo, all(n);
    for (int i = 0; i < n; ++i) {
        SPASM_TRY(finalize(prs[i]));
        SPASM_CUDA(cudaStreamSynchronize(prs[i]->stream));
        if (!prs[i]->placed) todo.push_back(i);
        all[i] = i;
    }
    const std::vector<int> order = job_order(prs, all, cfg.order);
    BatchLaunch bl;
    SPASM_TRY(prepare_batch(prs, order, cfg, s, bl));
    // one graph: stage 1 of the problems not yet placed, the first lift of every problem, one
    // persistent trajectory launch over all particles, then each problem's selection, re-lift
    // loop and FP64 check; problems whose stage 1 kept nothing skip stage 2 on the device
    Branches br1, br;   // branch streams live until the capture has ended
    SPASM_TRY(run_graph(s, [&](cudaStream_t c) -> spasm_status {
        SPASM_TRY(enqueue_place_all(prs, todo, c, br1));
        SPASM_TRY(br.init(c, std::min(n, kMaxBranches)));
        SPASM_TRY(br.fork());
        for (int i = 0; i < n; ++i) SPASM_TRY(enqueue_traj_lift(prs[i], br[i]));
        SPASM_TRY(br.join());
        SPASM_TRY(enqueue_batch(bl, c));
        SPASM_TRY(br.fork());
        for (int i = 0; i < n; ++i) {
            SPASM_TRY(enqueue_traj_retry(prs[i], br[i]));
            SPASM_TRY(enqueue_finish(prs[i], br[i]));
        }
        return br.join();
    }));
    mark_placed(prs, todo);
    for (int i = 0; i < n; ++i) {
        spasm_problem* pr = prs[i];
        pr->traj_pending = true;
        pr->traj_timed = false;
        pr->traj_batched = true;
    }
    return SPASM_OK;
}

extern "C" spasm_status spasm_batch_autotune(spasm_problem_t* prs, int n, void* cuda_stream, spasm_batch_config* best,
                                             double* best_ms) {
    Range r("spasm_batch_autotune");
    SPASM_TRY(check_batch(prs, n, cuda_stream));
    if (!best) return fail(SPASM_ERR_INVALID, "null config");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<int> todo;
    for (int i = 0; i < n; ++i) {
        SPASM_TRY(finalize(prs[i]));
        SPASM_CUDA(cudaStreamSynchronize(prs[i]->stream));
        if (!prs[i]->placed) todo.push_back(i);
    }
    Branches br;
    SPASM_TRY(run_graph(s, [&](cudaStream_t c) { return enqueue_place_all(prs, todo, c, br); }));
    mark_placed(prs, todo);
    std::vector<int> live;
    for (int i = 0; i < n; ++i) {
        SPASM_TRY(finalize(prs[i]));   // reads the placement counts
        if (prs[i]->n_place > 0) live.push_back(i);
    }
    spasm_batch_default_config(best);
    if (best_ms) *best_ms = 0.0;
    if (live.empty()) return SPASM_OK;
    auto lift_all = [&]() -> spasm_status {
        for (int i : live) {
            spasm_problem* pr = prs[i];
            SPASM_CUDA(launch_lift(pr->sc, pr->sc.Q, pr->d_place, pr->n_place, 0u, pr->d_q, s));
        }
        return SPASM_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPASM_CUDA(cudaEventCreate(&e0));
    SPASM_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    // (1) the trajectory shape (sphere tiling x particles per CTA), each over one full descent of
    // every lifted particle: a descent mostly runs from the cached cull, which one evaluation
    // (every chunk culled) does not show
    double shape_t = 1e300;
    for (int tiling = 0; tiling <= 1; ++tiling)
        for (int ppc = 1; ppc <= 2; ++ppc) {
            JobList L = make_jobs(prs, job_order(prs, live, 0), 1, kTrajModeDescend, 0, true);
            for (size_t k = 0; k < L.jobs.size(); ++k) {
                L.jobs[k].io.k_steps = prs[job_order(prs, live, 0)[k]]->sc.K_traj;
                L.jobs[k].io.tests = nullptr;   // the problems' counters are the solves'
            }
            if (traj_batch_ctas_per_sm(L.smem, tiling, ppc) < 1) continue;   // two particles do not fit
            spasm_batch_config c{1, 0, 0, tiling, ppc};
            int grid = 0;
            SPASM_TRY(batch_grid(c, L.smem, &grid));
            DeviceJobs dj;
            SPASM_TRY(upload_jobs(L, s, dj));
            SPASM_TRY(lift_all());
            SPASM_CUDA(cudaMemsetAsync(dj.next, 0, sizeof(int), s));
            SPASM_CUDA(cudaEventRecord(e0, s));
            SPASM_CUDA(launch_traj_batch(dj.jobs, (int)L.jobs.size(), L.n_items, 1, kTrajModeDescend, dj.next, L.smem,
                                         grid, s, tiling, ppc));
            SPASM_CUDA(cudaEventRecord(e1, s));
            SPASM_CUDA(cudaEventSynchronize(e1));
            const double t = ev_ms(e0, e1);
            if (t < shape_t) { shape_t = t; best->sphere_tiling = tiling; best->particles_per_cta = ppc; }
        }
    // (2) the schedule of the persistent launch under that shape: one evaluation of every lifted
    // particle per candidate (no writes besides q's reads)
    SPASM_TRY(lift_all());
    const int tiling = best->sphere_tiling, ppc = best->particles_per_cta;
    double best_t = 1e300;
    const int fetches[] = {1, 2, 4};
    for (int order = 0; order <= 1; ++order)
        for (int pf : fetches)
            for (int per_sm : {0, 1}) {
                spasm_batch_config c{pf, per_sm, order, tiling, ppc};
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
                                                 L.smem, grid, s, tiling, ppc));
                    SPASM_CUDA(cudaEventRecord(e1, s));
                    SPASM_CUDA(cudaEventSynchronize(e1));
                    if (rep > 0) t = ev_ms(e0, e1);
                }
                if (t < best_t) { best_t = t; *best = c; }
            }
    for (int i : live) SPASM_TRY(check_device_error(prs[i]));
    // the candidates wrote nothing the next solve reads: it lifts q again and starts its descents
    // from fresh multipliers
    if (best_ms) *best_ms = best_t;
    return SPASM_OK;
}
