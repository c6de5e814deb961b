// Stage-1 sampling and elite selection that allocates no device memory.
//
// Some callers cannot allocate device memory when they ask for work: a planner inside a
// real-time control loop must not stall on cudaMalloc (it can block and implicitly
// synchronise the device), and a plug-in hosted by a framework that owns all of the GPU's
// memory through its own pool may not be allowed to allocate behind the framework's back.
// For them this entry point keeps its intermediate buffers (the n sampled particles, their
// costs and the selected indices) in one file-scope device array of fixed size instead of
// allocating them.  The caller still provides the outputs.
//
// Set-up: the device address of the array is looked up once per device, with that device
// current, by the first call made on it (cudaGetSymbolAddress); make that first call before
// any stream capture begins.  With lazy module loading (the CUDA default) that lookup may be
// what loads the library's device code and creates the array, so the first call can allocate
// and synchronise; the calls after it allocate nothing.  The array is shared by every call on a device and keeps the
// contents of the last call; nothing in it needs to start at zero because every call
// overwrites what it reads.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the caller.
#include <mutex>
#include <string>

#include "launch.h"
#include "spasm.h"

namespace spasm {

// 2^20 floats (4 MiB): 4B x n particle values + n costs + m indices must fit.
constexpr size_t kStaticScratchFloats = size_t(1) << 20;
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

// x_out[v][r] = x[v][idx[r]] for SoA arrays (ld n in, ld m out)
__global__ void k_gather_soa(const float* __restrict__ x, int n, int nv, const int* __restrict__ idx, int m,
                             float* __restrict__ x_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv * m) return;
    const int v = i / m, r = i % m;
    x_out[(size_t)v * m + r] = x[(size_t)v * n + idx[r]];
}

static std::mutex g_scratch_mutex;
static void* g_scratch_ptr[64] = {};

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t static_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<float*>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

}  // namespace spasm

// Problem internals shared with api.cu
struct spasm_problem;
namespace spasm {
const Scalars& problem_scalars(const spasm_problem* pr);
DevTables problem_tables(const spasm_problem* pr);
cudaStream_t problem_stream(const spasm_problem* pr);
int* problem_error_word(spasm_problem* pr);
spasm_status set_last_error(spasm_status st, const std::string& msg);
}  // namespace spasm

extern "C" spasm_status spasm_place_select_static(spasm_problem_t pr, int n, uint32_t attempt, int m, float* x_elite,
                                                  float* cost_elite) {
    using namespace spasm;
    if (!pr) return set_last_error(SPASM_ERR_INVALID, "null problem");
    const Scalars& sc = problem_scalars(pr);
    const int nv = 4 * sc.B;
    if (n < 1 || m < 1 || m > n || !x_elite || !cost_elite)
        return set_last_error(SPASM_ERR_INVALID, "need 1 <= m <= n and output buffers");
    if (n > 32768 || m > 8192)
        return set_last_error(SPASM_ERR_INVALID, "n <= 32768 and m <= 8192 required by the selection kernel");
    const size_t need = (size_t)nv * n + (size_t)n + (size_t)m;
    if (need > kStaticScratchFloats)
        return set_last_error(SPASM_ERR_INVALID,
                              "4B*n + n + m = " + std::to_string(need) + " exceeds the static scratch of " +
                                  std::to_string(kStaticScratchFloats) + " floats (4 MiB)");
    float* scr = nullptr;
    cudaError_t e = static_scratch(&scr);
    if (e != cudaSuccess) return set_last_error(SPASM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    float* xs = scr;                                   // 4B x n sampled particles
    float* cost = scr + (size_t)nv * n;                // n costs
    int* idx = reinterpret_cast<int*>(cost + n);       // m selected indices
    cudaStream_t st = problem_stream(pr);
    e = launch_place_sample_cost(sc, problem_tables(pr), n, attempt, xs, cost, problem_error_word(pr), st);
    if (e == cudaSuccess) e = launch_topk(cost, n, m, idx, cost_elite, st);
    if (e == cudaSuccess) {
        k_gather_soa<<<(nv * m + 255) / 256, 256, 0, st>>>(xs, n, nv, idx, m, x_elite);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_last_error(SPASM_ERR_CUDA, std::string("place_select_static: ") + cudaGetErrorString(e));
    return SPASM_OK;
}
