// The two-stage driver with its attempt loops on the device.
//
// Alg. 1 restarts from a fresh sample until some particle satisfies the constraints
// (Sec. III-A), and the experiments cap the gradient steps at max_steps (Sec. IV-C); stage 2
// re-lifts with the next Philox attempt counter under the same cap.  Each stage is one CUDA
// graph: the first attempt, then a conditional while node whose body repeats the attempt.
// A one-thread control kernel at the end of every attempt advances the attempt counter and
// the step count in device memory (LoopCtl; the next attempt's sampling or lift reads its
// Philox counter there, and the key, so that a new seed needs no new graph), and sets the
// loop condition from the satisfying count.  The host
// enqueues a stage and returns; it reads the counters once, in the first synchronising
// call afterwards (finalize).  A stage-2 run whose stage 1 kept no placement does nothing:
// its kernels read the placement count and return.
#include <string>
#include <vector>

#include "problem.h"

using namespace spasm;

namespace {

// Stage-1 attempt control: the loop condition goes to the while node (kGraph) or to c->more
// for the host to read (the eager mode).
template <bool kGraph>
__global__ void k_place_loop(LoopCtl* __restrict__ c, const int* __restrict__ nsat, int per, int max_steps, int P,
                             cudaGraphConditionalHandle h) {
    const int steps = c->steps + per;
    const int ns = *nsat;
    const bool more = ns == 0 && steps < max_steps;
    c->attempt += 1u;
    c->steps = steps;
    if (!more) c->n_place = ns < P ? ns : P;
    if constexpr (kGraph) cudaGraphSetConditional(h, more ? 1u : 0u);
    else c->more = more ? 1 : 0;
}

__global__ void k_traj_begin(LoopCtl* __restrict__ c, int* __restrict__ tnsat) {
    c->t_attempt = 0u;
    c->t_steps = 0;
    c->found = 0;
    *tnsat = 0;
}

// Satisfying trajectory particles: their rank costs (metrics[.][7]), NaN for the others
// (ranked last by the selection), and their count.
__global__ void __launch_bounds__(1024) k_traj_select(const float* __restrict__ metrics, const int* __restrict__ sat,
                                                      int n, const LoopCtl* __restrict__ c, float* __restrict__ masked,
                                                      int* __restrict__ nsat) {
    if (c->n_place <= 0) return;   // nothing was optimised; the count stays 0
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const bool ok = sat[i] != 0;
        masked[i] = ok ? metrics[8 * (size_t)i + 7] : __int_as_float(0x7fc00000);
        mine += ok;
    }
    mine = __reduce_add_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0) atomicAdd(&cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) *nsat = cnt;
}

__global__ void k_traj_loop(LoopCtl* __restrict__ c, const int* __restrict__ tnsat, int per, int max_steps, int P,
                            cudaGraphConditionalHandle h) {
    const bool active = c->n_place > 0;
    const int ns = active ? *tnsat : 0;
    const int steps = c->t_steps + (active ? per : 0);
    const bool more = active && ns == 0 && steps < max_steps;
    if (active) c->t_attempt += 1u;
    c->t_steps = steps;
    if (!more) c->found = ns < P ? ns : P;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Fault injection of the bounded device wait: one CTA waits, with the bounded wait the table
// staging uses, on an mbarrier whose phase expects 16 bytes that no copy delivers (none is
// issued, so nothing is in flight); after max_polls polls it records kDevTimeout and returns.
__global__ void k_wait_timeout(int max_polls, int* __restrict__ err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    if (!mbar_wait_bounded(&bar, 0, max_polls) && threadIdx.x == 0) set_error(err, kDevTimeout);
    __syncthreads();
}

// Stage-2 attempt control when the attempts are scheduled from the host (the solver service):
// as k_traj_loop, with the decision left in c->t_more for the host to read.
__global__ void k_traj_epoch(LoopCtl* __restrict__ c, const int* __restrict__ tnsat, int per, int max_steps, int P) {
    const bool active = c->n_place > 0;
    const int ns = active ? *tnsat : 0;
    const int steps = c->t_steps + (active ? per : 0);
    const bool more = active && ns == 0 && steps < max_steps;
    if (active) c->t_attempt += 1u;
    c->t_steps = steps;
    if (!more) c->found = ns < P ? ns : P;
    c->t_more = more ? 1 : 0;
}

__global__ void k_gather_solutions(const float* __restrict__ q, const float* __restrict__ metrics,
                                   const int* __restrict__ best, const int* __restrict__ nsat, int P, int C,
                                   float* __restrict__ rq, float* __restrict__ rcost, int* __restrict__ rsucc) {
    const int r = blockIdx.x;
    const int n = min(*nsat, P);
    if (r >= P) return;
    if (r >= n) {
        if (threadIdx.x == 0) { rcost[r] = 0.f; rsucc[r] = 0; }
        return;
    }
    const int src = best[r];
    for (int i = threadIdx.x; i < C * 8; i += blockDim.x) rq[(size_t)r * C * 8 + i] = q[(size_t)src * C * 8 + i];
    if (threadIdx.x == 0) { rcost[r] = metrics[8 * (size_t)src + 7]; rsucc[r] = 1; }
}

// The graph stream s is capturing into, and a conditional handle on it (value 0 at every
// launch until a kernel sets it).
spasm_status new_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    SPASM_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive || !g) return fail(SPASM_ERR_CUDA, "the driver stream is not capturing");
    SPASM_CUDA(cudaGraphConditionalHandleCreate(h, g, 0u, cudaGraphCondAssignDefault));
    return SPASM_OK;
}

// Appends to the capture of s a while node on handle h after s's current work, and captures
// what `body` enqueues on `aux` as the node's body.
template <typename F>
spasm_status add_while(cudaStream_t s, cudaStream_t aux, cudaGraphConditionalHandle h, F body) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t n_deps = 0;
    SPASM_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &n_deps));
    if (cs != cudaStreamCaptureStatusActive) return fail(SPASM_ERR_CUDA, "the driver stream is not capturing");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    SPASM_CUDA(cudaGraphAddNode(&node, g, deps, edges, n_deps, &p));
    SPASM_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t bodyg = p.conditional.phGraph_out[0];
    SPASM_CUDA(cudaStreamBeginCaptureToGraph(aux, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const spasm_status st = body(aux);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(aux, &out);   // out is the node's own body graph
    if (st != SPASM_OK) return st;
    if (e != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("while-body capture: ") + cudaGetErrorString(e));
    return SPASM_OK;
}

// Records `ev` as a node of the graph being captured on s (a timing point of the graph).
spasm_status mark(cudaStream_t s, cudaEvent_t ev) {
    SPASM_CUDA(cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal));
    return SPASM_OK;
}

// One attempt of Alg. 1: sample N with the attempt counter read from the device, initial
// cost, elite top-M, the fused descent, satisfying mask and count (-> d_nsat), best P
// placements (-> d_place).
spasm_status place_attempt(spasm_problem* pr, cudaStream_t s) {
    const Scalars& sc = pr->sc;
    const int N = sc.N, M = sc.M, P = sc.P, B = sc.B;
    SPASM_CUDA(launch_place_sample_cost(sc, pr->tab, N, 0u, pr->d_xs, pr->d_cost, pr->d_err, s, pr->d_ctl));
    SPASM_CUDA(launch_topk(pr->d_cost, N, M, pr->d_idx, nullptr, s));
    SPASM_CUDA(launch_place_descend(sc, pr->tab, M, pr->d_xs, N, pr->d_idx, pr->d_xm, sc.K_lin, sc.K_quad,
                                    pr->d_costm, pr->d_sat, nullptr, pr->d_err, s));
    SPASM_CUDA(launch_mask_costs(pr->d_costm, pr->d_sat, M, pr->d_masked, pr->d_nsat, s));
    SPASM_CUDA(launch_topk(pr->d_masked, M, P, pr->d_best, nullptr, s));
    SPASM_CUDA(launch_gather_soa_to_aos(pr->d_xm, M, 4 * B, pr->d_best, P, pr->d_place, s));
    return SPASM_OK;
}
constexpr int kPlaceAttemptKernels = 7;   // the six above and the loop control

// The loop control after an attempt: into the while node on h, or (eager, h unused) into c->more.
spasm_status place_loop(spasm_problem* pr, cudaStream_t s, cudaGraphConditionalHandle h, bool eager = false) {
    const Scalars& sc = pr->sc;
    if (eager)
        k_place_loop<false><<<1, 1, 0, s>>>(pr->d_ctl, pr->d_nsat, sc.K_lin + sc.K_quad, pr->prm.max_steps, sc.P, h);
    else
        k_place_loop<true><<<1, 1, 0, s>>>(pr->d_ctl, pr->d_nsat, sc.K_lin + sc.K_quad, pr->prm.max_steps, sc.P, h);
    SPASM_CUDA(cudaGetLastError());
    return SPASM_OK;
}

TrajIO descent_io(spasm_problem* pr) {
    TrajIO io{};
    io.q = pr->d_q; io.lam = pr->d_lam; io.mu = pr->d_mu; io.metrics = pr->d_metrics; io.sat = pr->d_tsat;
    io.k_steps = pr->sc.K_traj; io.init_multipliers = 1;
    io.tests = pr->d_tests;
    io.active = &pr->d_ctl->n_place;
    return io;
}

spasm_status traj_lift(spasm_problem* pr, cudaStream_t s) {
    SPASM_CUDA(launch_lift(pr->sc, pr->sc.Q, pr->d_place, 1, 0u, pr->d_q, s, pr->d_ctl));
    return SPASM_OK;
}

spasm_status traj_select_loop(spasm_problem* pr, cudaStream_t s, cudaGraphConditionalHandle h) {
    const Scalars& sc = pr->sc;
    k_traj_select<<<1, 1024, 0, s>>>(pr->d_metrics, pr->d_tsat, sc.Q, pr->d_ctl, pr->d_tmasked, pr->d_tnsat);
    SPASM_CUDA(cudaGetLastError());
    k_traj_loop<<<1, 1, 0, s>>>(pr->d_ctl, pr->d_tnsat, sc.K_traj, pr->prm.max_steps, sc.P, h);
    SPASM_CUDA(cudaGetLastError());
    return SPASM_OK;
}
// begin + finish (3) once; lift (2), descent, select and loop control per attempt
constexpr int kTrajFixedKernels = 4;
constexpr int kTrajAttemptKernels = 5;

// Captures what `enqueue` puts on `cap` into a graph and instantiates it.
template <typename F>
spasm_status build_graph(cudaStream_t cap, cudaGraphExec_t* out, F enqueue) {
    SPASM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    const spasm_status st = enqueue(cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st != SPASM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(SPASM_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ei));
    return SPASM_OK;
}

// The eager mode: the graphs' kernels in the graphs' order, launched one at a time, with the
// loop decision read by the host after every attempt (one wait per attempt).
spasm_status read_more(spasm_problem* pr, const int* d_more, int* more) {
    SPASM_CUDA(cudaMemcpyAsync(more, d_more, sizeof(int), cudaMemcpyDeviceToHost, pr->stream));
    SPASM_TRY(host_wait(pr));
    pr->stats.d2h_bytes += sizeof(int);
    return SPASM_OK;
}

spasm_status record(spasm_problem* pr, int i) {
    SPASM_CUDA(cudaEventRecord(pr->ev[i], pr->stream));
    return SPASM_OK;
}

}  // namespace

spasm_status spasm::run_place_eager(spasm_problem* pr) {
    Range r("spasm stage 1 (eager)");
    cudaStream_t s = pr->stream;
    SPASM_CUDA(cudaMemsetAsync(pr->d_ctl, 0, offsetof(LoopCtl, t_attempt), s));
    for (int more = 1; more;) {
        SPASM_TRY(place_attempt(pr, s));
        SPASM_TRY(place_loop(pr, s, 0, true));
        SPASM_TRY(read_more(pr, &pr->d_ctl->more, &more));
    }
    return SPASM_OK;
}

spasm_status spasm::run_traj_eager(spasm_problem* pr) {
    Range r("spasm stage 2 (eager)");
    cudaStream_t s = pr->stream;
    SPASM_TRY(record(pr, 2));
    SPASM_TRY(enqueue_traj_lift(pr, s));
    SPASM_TRY(record(pr, 3));
    SPASM_TRY(enqueue_traj_descent(pr, s));
    SPASM_TRY(record(pr, 4));
    for (int more = 1;;) {
        SPASM_TRY(enqueue_traj_epoch_end(pr, s));   // the selection and the loop control
        SPASM_TRY(read_more(pr, &pr->d_ctl->t_more, &more));
        if (!more) break;
        SPASM_TRY(enqueue_traj_relift(pr, s));
        SPASM_TRY(enqueue_traj_descent(pr, s));
    }
    SPASM_TRY(record(pr, 5));
    SPASM_TRY(enqueue_finish(pr, s));
    return record(pr, 6);
}

spasm_status spasm::enqueue_place(spasm_problem* pr, cudaStream_t s) {
    cudaGraphConditionalHandle h;
    SPASM_TRY(new_handle(s, &h));
    SPASM_CUDA(cudaMemsetAsync(pr->d_ctl, 0, offsetof(LoopCtl, t_attempt), s));   // stage-1 counters (not the key)
    SPASM_TRY(place_attempt(pr, s));
    SPASM_TRY(place_loop(pr, s, h));
    return add_while(s, pr->cap_body, h, [&](cudaStream_t b) -> spasm_status {
        SPASM_TRY(place_attempt(pr, b));
        return place_loop(pr, b, h);
    });
}

spasm_status spasm::enqueue_traj_lift(spasm_problem* pr, cudaStream_t s) {
    k_traj_begin<<<1, 1, 0, s>>>(pr->d_ctl, pr->d_tnsat);
    SPASM_CUDA(cudaGetLastError());
    SPASM_CUDA(cudaMemsetAsync(pr->d_tests, 0, 3 * sizeof(unsigned long long), s));
    return traj_lift(pr, s);
}

spasm_status spasm::enqueue_traj_descent(spasm_problem* pr, cudaStream_t s) {
    SPASM_CUDA(launch_traj(pr->sc, pr->tab, pr->sc.Q, kTrajModeDescend, descent_io(pr), pr->d_err, s));
    return SPASM_OK;
}

spasm_status spasm::enqueue_traj_retry(spasm_problem* pr, cudaStream_t s) {
    cudaGraphConditionalHandle h;
    SPASM_TRY(new_handle(s, &h));
    SPASM_TRY(traj_select_loop(pr, s, h));
    return add_while(s, pr->cap_body, h, [&](cudaStream_t b) -> spasm_status {
        SPASM_TRY(traj_lift(pr, b));
        SPASM_TRY(enqueue_traj_descent(pr, b));
        return traj_select_loop(pr, b, h);
    });
}

spasm_status spasm::enqueue_traj_relift(spasm_problem* pr, cudaStream_t s) { return traj_lift(pr, s); }

spasm_status spasm::enqueue_traj_epoch_end(spasm_problem* pr, cudaStream_t s) {
    const Scalars& sc = pr->sc;
    k_traj_select<<<1, 1024, 0, s>>>(pr->d_metrics, pr->d_tsat, sc.Q, pr->d_ctl, pr->d_tmasked, pr->d_tnsat);
    SPASM_CUDA(cudaGetLastError());
    k_traj_epoch<<<1, 1, 0, s>>>(pr->d_ctl, pr->d_tnsat, sc.K_traj, pr->prm.max_steps, sc.P);
    SPASM_CUDA(cudaGetLastError());
    return SPASM_OK;
}

spasm_status spasm::enqueue_finish(spasm_problem* pr, cudaStream_t s) {
    const Scalars& sc = pr->sc;
    if (sc.Q > 32768) return fail(SPASM_ERR_INVALID, "Q > 32768 unsupported by the selection kernel");
    SPASM_CUDA(launch_topk(pr->d_tmasked, sc.Q, sc.P, pr->d_tbest, nullptr, s));
    k_gather_solutions<<<sc.P, 256, 0, s>>>(pr->d_q, pr->d_metrics, pr->d_tbest, pr->d_tnsat, sc.P, sc.C, pr->d_rq,
                                             pr->d_rcost, pr->d_rsucc);
    SPASM_CUDA(cudaGetLastError());
    // FP64 re-evaluation of the returned solutions decides their success flags
    SPASM_CUDA(launch_check64(pr->s64, pr->d_cub64, pr->d_osph64, pr->d_rq, pr->d_tnsat, sc.P, pr->d_rmet64,
                              pr->d_rsucc, pr->d_chkacc, s));
    return SPASM_OK;
}

void spasm::drop_graphs(spasm_problem* pr) {
    if (pr->g_place) cudaGraphExecDestroy(pr->g_place);
    if (pr->g_traj) cudaGraphExecDestroy(pr->g_traj);
    pr->g_place = pr->g_traj = nullptr;
}

spasm_status spasm::finalize(spasm_problem* pr) {
    if (!pr->place_pending && !pr->traj_pending) return SPASM_OK;
    Range r("spasm finalize (reads the stage outcome)");
    const bool place = pr->place_pending, traj = pr->traj_pending;
    const int P = pr->sc.P;
    LoopCtl c{};
    int err = 0;
    unsigned long long nt[3] = {0, 0, 0};
    std::vector<int> succ(traj ? P : 0, 0);
    SPASM_CUDA(cudaMemcpyAsync(&c, pr->d_ctl, sizeof c, cudaMemcpyDeviceToHost, pr->stream));
    SPASM_CUDA(cudaMemcpyAsync(&err, pr->d_err, sizeof err, cudaMemcpyDeviceToHost, pr->stream));
    if (traj) {
        SPASM_CUDA(cudaMemcpyAsync(nt, pr->d_tests, sizeof nt, cudaMemcpyDeviceToHost, pr->stream));
        SPASM_CUDA(cudaMemcpyAsync(succ.data(), pr->d_rsucc, P * sizeof(int), cudaMemcpyDeviceToHost, pr->stream));
    }
    SPASM_TRY(host_wait(pr));
    pr->stats.d2h_bytes += sizeof c + sizeof err + (traj ? sizeof nt + P * sizeof(int) : 0);
    pr->place_pending = pr->traj_pending = false;
    if (place) {
        pr->place_attempts = (int)c.attempt;
        pr->place_steps = c.steps;
        pr->n_place = c.n_place;
        pr->stats.place_attempts += (int)c.attempt;
        count_launches(pr, kPlaceAttemptKernels * (int)c.attempt);
        if (pr->place_timed) pr->stats.ms_place += ev_ms(pr->ev[0], pr->ev[1]);
    }
    if (traj) {
        const Scalars& sc = pr->sc;
        const int a = (int)c.t_attempt;
        pr->traj_attempts = a;
        pr->n_found = c.found;
        pr->optimized = true;
        pr->stats.traj_attempts += a;
        pr->stats.traj_launches += a;
        pr->stats.particle_iters += (long long)sc.Q * sc.K_traj * a;
        count_launches(pr, kTrajFixedKernels + kTrajAttemptKernels * (a > 1 ? a : 1) - (pr->traj_batched ? 1 : 0));
        pr->stats.tests_executed += (long long)nt[0];
        pr->stats.cull_configs += (long long)nt[1];
        pr->stats.cand_configs += (long long)nt[2];
        int ns = 0;
        for (int r = 0; r < c.found; ++r) ns += succ[r] != 0;
        pr->stats.n_success = ns;
        pr->stats.n_found = c.found;
        if (pr->traj_timed) {
            pr->stats.ms_lift += ev_ms(pr->ev[2], pr->ev[3]);
            pr->stats.ms_traj += ev_ms(pr->ev[3], pr->ev[4]);
            pr->stats.ms_retry += ev_ms(pr->ev[4], pr->ev[5]);
            pr->stats.ms_finish += ev_ms(pr->ev[5], pr->ev[6]);
        }
    }
    pr->place_timed = pr->traj_timed = pr->traj_batched = false;
    if (err != 0) {
        const char* what = err == kDevTimeout ? "a bounded device wait gave up" : "a kernel rejected its sizes";
        return fail(SPASM_ERR_DEVICE, std::string("device error ") + std::to_string(err) + ": " + what);
    }
    return SPASM_OK;
}

spasm_status spasm::prepare_graphs(spasm_problem* pr) {
    if (pr->sc.kind != kKindP2P && !pr->g_place)
        SPASM_TRY(build_graph(pr->cap, &pr->g_place, [&](cudaStream_t s) { return enqueue_place(pr, s); }));
    if (pr->sc.kind != kKindPack && !pr->g_traj)
        SPASM_TRY(build_graph(pr->cap, &pr->g_traj, [&](cudaStream_t s) -> spasm_status {
            SPASM_TRY(mark(s, pr->ev[2]));
            SPASM_TRY(enqueue_traj_lift(pr, s));
            SPASM_TRY(mark(s, pr->ev[3]));
            SPASM_TRY(enqueue_traj_descent(pr, s));
            SPASM_TRY(mark(s, pr->ev[4]));
            SPASM_TRY(enqueue_traj_retry(pr, s));
            SPASM_TRY(mark(s, pr->ev[5]));
            SPASM_TRY(enqueue_finish(pr, s));
            return mark(s, pr->ev[6]);
        }));
    return SPASM_OK;
}

// ------------------------------------------------------------------------------ the C ABI
extern "C" spasm_status spasm_place(spasm_problem_t pr) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    if (pr->sc.kind == kKindP2P) return fail(SPASM_ERR_INVALID, "a point-to-point problem has no stage 1");
    Range r("spasm_place");
    SPASM_TRY(finalize(pr));   // fold a previous run's counters first
    if (!pr->eager) SPASM_TRY(prepare_graphs(pr));
    if (pr->timing) SPASM_CUDA(cudaEventRecord(pr->ev[0], pr->stream));
    if (pr->eager) SPASM_TRY(run_place_eager(pr));
    else SPASM_CUDA(cudaGraphLaunch(pr->g_place, pr->stream));
    if (pr->timing) SPASM_CUDA(cudaEventRecord(pr->ev[1], pr->stream));
    pr->placed = true;
    pr->place_pending = true;
    pr->place_timed = pr->timing;
    return SPASM_OK;
}

extern "C" spasm_status spasm_optimize(spasm_problem_t pr) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    if (pr->sc.kind == kKindPack)
        return fail(SPASM_ERR_INVALID, "stage 2 is implemented for the tower goal only; packing runs stage 1 (spasm_place)");
    Range r("spasm_optimize");
    if (pr->traj_pending) SPASM_TRY(finalize(pr));
    if (!pr->placed) SPASM_TRY(spasm_place(pr));
    if (pr->eager) {
        SPASM_TRY(run_traj_eager(pr));
    } else {
        SPASM_TRY(prepare_graphs(pr));
        SPASM_CUDA(cudaGraphLaunch(pr->g_traj, pr->stream));
    }
    pr->traj_pending = true;
    pr->traj_timed = pr->timing;
    pr->traj_batched = false;
    return SPASM_OK;
}

extern "C" spasm_status spasm_inject_wait_timeout(spasm_problem_t pr, int max_polls) {
    if (!pr || max_polls < 1 || max_polls > kTablePolls) return fail(SPASM_ERR_INVALID, "need 1 <= max_polls <= 2^22");
    k_wait_timeout<<<1, 32, 0, pr->stream>>>(max_polls, pr->d_err);
    SPASM_CUDA(cudaGetLastError());
    return SPASM_OK;
}

extern "C" spasm_status spasm_set_launch_mode(spasm_problem_t pr, int mode) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    if (mode != SPASM_LAUNCH_GRAPH && mode != SPASM_LAUNCH_EAGER)
        return fail(SPASM_ERR_INVALID, "mode must be SPASM_LAUNCH_GRAPH or SPASM_LAUNCH_EAGER");
    SPASM_TRY(finalize(pr));
    pr->eager = mode == SPASM_LAUNCH_EAGER;
    return SPASM_OK;
}
