// Internal: the problem handle and the host-side helpers shared by the C-ABI files
// (api.cu, batch.cu).  Not part of the public interface.
#pragma once
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "spasm.h"
#include "check64.h"
#include "launch_s2.h"
#include "stage2.cuh"

namespace spasm {
// Records `msg` as this thread's last error and returns `st`.
spasm_status fail(spasm_status st, const std::string& msg);
}  // namespace spasm

#define SPASM_CUDA(call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return spasm::fail(SPASM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

#define SPASM_TRY(x)                      \
    do {                                  \
        spasm_status s_ = (x);            \
        if (s_ != SPASM_OK) return s_;    \
    } while (0)

struct spasm_problem {
    spasm::Scalars sc;
    spasm_params prm;
    cudaStream_t stream = nullptr;
    spasm::DevTables tab{};
    spasm::Scalars* d_sc = nullptr;   // device copy of sc (read by the batched kernels)
    float4* d_cub = nullptr;
    float4* d_osph = nullptr;
    int* d_err = nullptr;
    // stage 1
    float *d_xs = nullptr, *d_cost = nullptr, *d_xm = nullptr, *d_costm = nullptr, *d_masked = nullptr;
    int *d_idx = nullptr, *d_sat = nullptr, *d_nsat = nullptr, *d_best = nullptr;
    float* d_place = nullptr;   // P x B x 4
    bool placed = false;
    int n_place = 0, place_attempts = 0, place_steps = 0;
    // stage 2
    float *d_q = nullptr, *d_lam = nullptr, *d_mu = nullptr, *d_metrics = nullptr, *d_tmasked = nullptr;
    int *d_tsat = nullptr, *d_tnsat = nullptr, *d_tbest = nullptr;
    float *d_rq = nullptr, *d_rcost = nullptr;   // returned solutions
    int* d_rsucc = nullptr;
    unsigned long long* d_tests = nullptr;   // [tests run, configurations culled] by the trajectory kernel
    bool optimized = false;
    int n_found = 0, traj_attempts = 0;
    // device-side attempt loops (driver.cu): counters and the Philox key on the device, each
    // stage's graph (built at creation), streams the graphs are captured on
    spasm::LoopCtl* d_ctl = nullptr;
    cudaGraphExec_t g_place = nullptr, g_traj = nullptr;
    cudaStream_t cap = nullptr, cap_body = nullptr;
    bool place_pending = false;   // a stage-1 run whose outcome the host has not read yet
    bool traj_pending = false;    // likewise stage 2
    bool place_timed = false;     // the pending stage-1 run is bracketed by ev[0], ev[1]
    bool traj_timed = false;      // the pending stage-2 run recorded ev[2..6]
    bool traj_batched = false;    // its first trajectory launch was shared with other problems
    bool eager = false;           // spasm_place / spasm_optimize launch kernel by kernel, the attempt
                                  // loops on the host (the same kernels and order as the graphs)
    std::vector<double> host_cub, host_osph;
    // FP64 final check
    spasm::Scalars64 s64;
    double* d_cub64 = nullptr;
    double* d_osph64 = nullptr;
    double* d_rmet64 = nullptr;
    spasm::CheckAcc* d_chkacc = nullptr;   // accumulators of the split FP64 check (P)
    // statistics and timing
    spasm_stats stats{};
    bool timing = false;
    cudaEvent_t ev[8] = {};
};

namespace spasm {

inline void count_launches(spasm_problem* pr, int n) { pr->stats.kernel_launches += n; }

// A named range on the host timeline of profilers (NVTX push/pop) for the life of the object;
// free when no profiler is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

inline float ev_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
    return ms;
}

inline spasm_status rec(spasm_problem* pr, int i) {
    if (pr->timing) SPASM_CUDA(cudaEventRecord(pr->ev[i], pr->stream));
    return SPASM_OK;
}

// Makes the host wait for the problem's stream (counted in stats.host_waits).
spasm_status host_wait(spasm_problem* pr);
// Reads the problem's device error word (synchronises its stream).
spasm_status check_device_error(spasm_problem* pr);

// ---- the two-stage driver (driver.cu), in pieces shared by spasm_optimize and the batched
// form.  The enqueue_* functions append to a stream that is being captured into a graph
// (they add conditional nodes to it); the attempt loops run on the device.
// Stage 1: the first attempt of Alg. 1, then a while node that repeats attempts until one
// satisfies or max_steps gradient steps are spent; d_ctl->n_place receives the count kept.
spasm_status enqueue_place(spasm_problem* pr, cudaStream_t s);
// Stage 2, first attempt: reset the stage-2 counters and lift (reads d_ctl on the device).
spasm_status enqueue_traj_lift(spasm_problem* pr, cudaStream_t s);
// Stage 2, first attempt: the fused trajectory descent of all Q particles.
spasm_status enqueue_traj_descent(spasm_problem* pr, cudaStream_t s);
// Stage 2 after the first descent: satisfying mask and count, then a while node that
// re-lifts and descends with the next attempt counter while none satisfies within max_steps.
spasm_status enqueue_traj_retry(spasm_problem* pr, cudaStream_t s);
// The final selection of the best P trajectories and their FP64 check.
spasm_status enqueue_finish(spasm_problem* pr, cudaStream_t s);
// Stage 2 attempt by attempt from the host (the solver service; no graph needed): the lift of
// the next attempt (counters on the device), and after a descent the satisfying count and the
// attempt decision (d_ctl->t_more: 1 while another attempt is due; d_ctl->found otherwise).
spasm_status enqueue_traj_relift(spasm_problem* pr, cudaStream_t s);
spasm_status enqueue_traj_epoch_end(spasm_problem* pr, cudaStream_t s);

// A persistent launch of the trajectory kernel in descent mode over the particles of several
// problems (batch.cu): the work list lives on the device until this object is destroyed,
// which must come after the launch has finished.
struct BatchLaunch {
    std::vector<TrajJob> host;   // source of the asynchronous upload
    TrajJob* jobs = nullptr;
    int* next = nullptr;
    cudaStream_t s = nullptr;
    int n_items = 0, grid = 0, per_fetch = 1, tiling = 0, ppc = 1;
    size_t smem = 0;
    BatchLaunch() = default;
    BatchLaunch(const BatchLaunch&) = delete;
    BatchLaunch& operator=(const BatchLaunch&) = delete;
    ~BatchLaunch();
};
// Builds and uploads (on s, asynchronously) the work list of problems prs[order[k]], each with
// its own K_traj steps and its placement count as the gate.
spasm_status prepare_batch(spasm_problem_t* prs, const std::vector<int>& order, const spasm_batch_config& cfg,
                           cudaStream_t s, BatchLaunch& bl);
// Enqueues the launch (resetting its work counter first).
spasm_status enqueue_batch(const BatchLaunch& bl, cudaStream_t s);
// Reads what the device loops left (attempts, counts, counters, success flags, the error
// word) after the pending stages, once; synchronises the problem's stream.
spasm_status finalize(spasm_problem* pr);
// Builds the stage graphs the problem's kind uses (stage 1 unless point to point, stage 2
// unless packing), once.
spasm_status prepare_graphs(spasm_problem* pr);
// Destroys the stage graphs.
void drop_graphs(spasm_problem* pr);
// The eager mode's stage runs on the problem's stream: the graphs' kernels in the same order,
// the attempt loops on the host (one wait per attempt).
spasm_status run_place_eager(spasm_problem* pr);
spasm_status run_traj_eager(spasm_problem* pr);

}  // namespace spasm
