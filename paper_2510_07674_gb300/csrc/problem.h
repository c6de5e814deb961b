// Internal: the problem handle and the host-side helpers shared by the C-ABI files
// (api.cu, batch.cu).  Not part of the public interface.
#pragma once
#include <string>
#include <vector>

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

inline float ev_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
    return ms;
}

inline spasm_status rec(spasm_problem* pr, int i) {
    if (pr->timing) SPASM_CUDA(cudaEventRecord(pr->ev[i], pr->stream));
    return SPASM_OK;
}

// Reads the problem's device error word (synchronises its stream).
spasm_status check_device_error(spasm_problem* pr);

// ---- the two-stage driver, in pieces shared by spasm_optimize and the batched form
// Enqueue one attempt of Alg. 1 on stream s (count of satisfying particles -> d_nsat,
// best placements -> d_place).
spasm_status place_attempt(spasm_problem* pr, uint32_t attempt, cudaStream_t s);
// Continue stage 1 after `attempt` attempts and `steps` gradient steps, whose last attempt
// left `nsat` satisfying particles (0: none, or no attempt yet), until an attempt
// satisfies or the step budget is spent; then record the placements.
spasm_status place_continue(spasm_problem* pr, int attempt, int steps, int nsat);
// Enqueue the rank costs and the satisfying mask of the trajectory particles (count -> d_tnsat).
spasm_status traj_select(spasm_problem* pr, cudaStream_t s);
// Enqueue the final selection of the best P trajectories and their FP64 check.
spasm_status finish_enqueue(spasm_problem* pr, cudaStream_t s);
// Continue stage 2 like place_continue; returns the number of solutions in *found.
spasm_status traj_continue(spasm_problem* pr, int attempt, int steps, int nsat, int* found);
// Record the outcome of stage 2 (enqueueing the finish first unless `finish_done`).
spasm_status finish_record(spasm_problem* pr, int found, bool finish_done);

}  // namespace spasm
