// Stage-1 kernels (Alg. 1): sampling + initial cost, evaluation, fused descent, and the
// selection kernel.
#include "launch.h"
#include "select.cuh"
#include "stage1.cuh"
#include "stage1_pack.cuh"

namespace spasm {

constexpr int kS1Warps = 8;
constexpr int kS1Threads = 32 * kS1Warps;

struct S1Warp {
    float x[4 * kMaxB];
    float g[4 * kMaxB];
    PlaceScratch ps;
    float4 gcell[kMaxCells];   // per-cube sphere-side gradients of the packing goal
    uint32_t cand[kMaxCub / 32 + kMaxOSph / 32];   // candidate obstacles of the particle (tower goal)
};

// dynamic shared memory: mbarrier | env cuboids | env spheres | per-warp scratch
__host__ __device__ inline size_t s1_env_offset() { return 16; }
__host__ __device__ inline size_t s1_warp_offset(int n_cub, int n_osph) {
    size_t off = 16 + (size_t)n_cub * 64 + (size_t)n_osph * 16;
    return (off + 15) & ~(size_t)15;
}
static size_t s1_smem_bytes(const Scalars& sc) {
    return s1_warp_offset(sc.n_cub, sc.n_osph) + sizeof(S1Warp) * kS1Warps;
}

struct S1Smem {
    uint64_t* bar;
    float4* cub;
    float4* osph;
    S1Warp* warp;
};

__device__ __forceinline__ bool s1_setup(const Scalars& sc, DevTables t, S1Smem& s, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    s.bar = reinterpret_cast<uint64_t*>(smem_raw);
    s.cub = reinterpret_cast<float4*>(smem_raw + s1_env_offset());
    s.osph = s.cub + 4 * sc.n_cub;
    s.warp = reinterpret_cast<S1Warp*>(smem_raw + s1_warp_offset(sc.n_cub, sc.n_osph));
    return stage_tables(s.cub, t.cub, (uint32_t)sc.n_cub * 64u, s.osph, t.osph, (uint32_t)sc.n_osph * 16u, s.bar, err);
}

__global__ void __launch_bounds__(kS1Threads) k_place_sample_cost(const __grid_constant__ Scalars sc, DevTables t, int n,
                                                                   uint32_t attempt, float* __restrict__ x_out,
                                                                   float* __restrict__ cost_out, int* err,
                                                                   const LoopCtl* __restrict__ ctl) {
    uint64_t key = sc.seed;   // the Philox key
    if (ctl) { attempt = ctl->attempt; key = ctl->seed; }
    S1Smem s;
    if (!s1_setup(sc, t, s, err)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * kS1Warps + w;
    if (p >= n) return;
    S1Warp& W = s.warp[w];
    if (lane < sc.B) {
        const int i = lane;
        const U4 u = philox4x32_10((uint32_t)i, (uint32_t)p, kTagSample, attempt, key);
        const float zlo = sc.zlo[i];
        W.x[4 * i + 0] = sc.box_lo[0] + u01(u.x) * (sc.box_hi[0] - sc.box_lo[0]);
        W.x[4 * i + 1] = sc.box_lo[1] + u01(u.y) * (sc.box_hi[1] - sc.box_lo[1]);
        W.x[4 * i + 2] = zlo + u01(u.z) * (sc.box_hi[2] - zlo);
        W.x[4 * i + 3] = -kPi + u01(u.w) * (2.f * kPi);
    }
    __syncwarp();
    PlaceOut o;
    place_eval(sc, s.cub, sc.n_cub, s.osph, sc.n_osph, W.x, false, kPlaceForward, nullptr, W.ps,
               W.gcell, W.cand, o);
    for (int v = lane; v < 4 * sc.B; v += 32) x_out[(size_t)v * n + p] = W.x[v];
    if (lane == 0) cost_out[p] = place_cost_value(sc, o);
}

__global__ void __launch_bounds__(kS1Threads) k_place_eval(const __grid_constant__ Scalars sc, DevTables t, int n,
                                                            const float* __restrict__ x, int quad,
                                                            float* __restrict__ cost, float* __restrict__ grad,
                                                            float* __restrict__ metrics, float* __restrict__ terms,
                                                            int* err) {
    S1Smem s;
    if (!s1_setup(sc, t, s, err)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * kS1Warps + w;
    if (p >= n) return;
    S1Warp& W = s.warp[w];
    for (int v = lane; v < 4 * sc.B; v += 32) W.x[v] = x[(size_t)v * n + p];
    __syncwarp();
    PlaceOut o;
    place_eval(sc, s.cub, sc.n_cub, s.osph, sc.n_osph, W.x, quad != 0, grad ? kPlaceStage1 : kPlaceForward, W.g, W.ps,
               W.gcell, W.cand, o);
    if (grad)
        for (int v = lane; v < 4 * sc.B; v += 32) grad[(size_t)v * n + p] = W.g[v];
    if (lane == 0) {
        if (cost) cost[p] = place_cost_value(sc, o);
        if (metrics) { metrics[3 * p] = o.maxpen; metrics[3 * p + 1] = o.maxD; metrics[3 * p + 2] = o.maxdz; }
        if (terms) { terms[3 * p] = o.c_stable; terms[3 * p + 1] = o.c_height; terms[3 * p + 2] = o.c_coll; }
    }
}

// Alg. 1, linear cost descent (eta = eta_init (1 - k/K_lin)) then quadratic refinement
// (fixed alpha), each followed by the box projection; then GetSatisfyingParticles and
// the final (quadratic-form) cost.  The whole loop runs inside one launch.
__global__ void __launch_bounds__(kS1Threads) k_place_descend(const __grid_constant__ Scalars sc, DevTables t, int m,
                                                               const float* __restrict__ x_src, int ld_src,
                                                               const int* __restrict__ idx, float* __restrict__ x_dst,
                                                               int k_lin, int k_quad, float* __restrict__ cost,
                                                               int* __restrict__ sat, float* __restrict__ metrics,
                                                               int* err) {
    S1Smem s;
    if (!s1_setup(sc, t, s, err)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * kS1Warps + w;
    if (p >= m) return;
    S1Warp& W = s.warp[w];
    const int nv = 4 * sc.B;
    const int src = idx ? idx[p] : p;
    for (int v = lane; v < nv; v += 32) W.x[v] = x_src[(size_t)v * ld_src + src];
    __syncwarp();
    PlaceOut o;
    for (int k = 1; k <= k_lin; ++k) {
        const float eta = sc.eta_init * (1.f - (float)k / (float)k_lin);
        place_eval(sc, s.cub, sc.n_cub, s.osph, sc.n_osph, W.x, false, kPlaceStage1, W.g, W.ps,
               W.gcell, W.cand, o);
        for (int v = lane; v < nv; v += 32) W.x[v] = place_clamp(sc, v, W.x[v] - eta * W.g[v]);
        __syncwarp();
    }
    for (int k = 1; k <= k_quad; ++k) {
        place_eval(sc, s.cub, sc.n_cub, s.osph, sc.n_osph, W.x, true, kPlaceStage1, W.g, W.ps,
               W.gcell, W.cand, o);
        for (int v = lane; v < nv; v += 32) W.x[v] = place_clamp(sc, v, W.x[v] - sc.alpha * W.g[v]);
        __syncwarp();
    }
    place_eval(sc, s.cub, sc.n_cub, s.osph, sc.n_osph, W.x, true, kPlaceForward, nullptr, W.ps,
               W.gcell, W.cand, o);
    for (int v = lane; v < nv; v += 32) x_dst[(size_t)v * m + p] = W.x[v];
    if (lane == 0) {
        if (cost) cost[p] = place_cost_value(sc, o);
        if (sat) sat[p] = (o.maxpen <= sc.eps && o.maxD <= sc.eps && o.maxdz <= sc.eps) ? 1 : 0;
        if (metrics) { metrics[3 * p] = o.maxpen; metrics[3 * p + 1] = o.maxD; metrics[3 * p + 2] = o.maxdz; }
    }
}

__global__ void k_mask_costs(const float* __restrict__ cost, const int* __restrict__ sat, int n,
                             float* __restrict__ out, int* __restrict__ n_sat) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const bool ok = sat[i] != 0;
        out[i] = ok ? cost[i] : __int_as_float(0x7fc00000);
        mine += ok;
    }
    mine = __reduce_add_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0) atomicAdd(&cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) *n_sat = cnt;
}

__global__ void k_gather_soa_to_aos(const float* __restrict__ src, int ld_src, int nv, const int* __restrict__ idx,
                                    int k, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k * nv) return;
    const int r = i / nv, v = i % nv;
    out[i] = src[(size_t)v * ld_src + idx[r]];
}

// ------------------------------------------------------------------------------ launchers
static cudaError_t s1_prepare(const Scalars& sc) {
    size_t bytes = s1_smem_bytes(sc);
    cudaError_t e = allow_max_dynamic_smem(k_place_sample_cost, bytes);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem(k_place_eval, bytes);
    if (e != cudaSuccess) return e;
    return allow_max_dynamic_smem(k_place_descend, bytes);
}

cudaError_t launch_place_sample_cost(const Scalars& sc, DevTables t, int n, uint32_t attempt, float* x, float* cost,
                                     int* err, cudaStream_t st, const LoopCtl* ctl) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = s1_prepare(sc);
    if (e != cudaSuccess) return e;
    k_place_sample_cost<<<(n + kS1Warps - 1) / kS1Warps, kS1Threads, s1_smem_bytes(sc), st>>>(sc, t, n, attempt, x,
                                                                                               cost, err, ctl);
    return cudaGetLastError();
}

cudaError_t launch_place_eval(const Scalars& sc, DevTables t, int n, const float* x, int quad, float* cost, float* grad,
                              float* metrics, float* terms, int* err, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = s1_prepare(sc);
    if (e != cudaSuccess) return e;
    k_place_eval<<<(n + kS1Warps - 1) / kS1Warps, kS1Threads, s1_smem_bytes(sc), st>>>(sc, t, n, x, quad, cost, grad,
                                                                                        metrics, terms, err);
    return cudaGetLastError();
}

cudaError_t launch_place_descend(const Scalars& sc, DevTables t, int m, const float* x_src, int ld_src, const int* idx,
                                 float* x_dst, int k_lin, int k_quad, float* cost, int* sat, float* metrics, int* err,
                                 cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    cudaError_t e = s1_prepare(sc);
    if (e != cudaSuccess) return e;
    k_place_descend<<<(m + kS1Warps - 1) / kS1Warps, kS1Threads, s1_smem_bytes(sc), st>>>(
        sc, t, m, x_src, ld_src, idx, x_dst, k_lin, k_quad, cost, sat, metrics, err);
    return cudaGetLastError();
}

static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

size_t topk_smem_bytes(int n, int k) {
    return (size_t)next_pow2(k < 1 ? 1 : k) * 8 + (size_t)n * 4;
}

cudaError_t launch_topk(const float* cost, int n, int k, int* idx, float* cost_out, cudaStream_t st) {
    if (n <= 0 || k <= 0) return cudaSuccess;
    if (k > n) k = n;
    const int kp2 = next_pow2(k);
    const size_t bytes = topk_smem_bytes(n, k);
    cudaError_t e = allow_max_dynamic_smem(k_topk, bytes);
    if (e != cudaSuccess) return e;
    k_topk<<<1, kSelectThreads, bytes, st>>>(cost, n, k, idx, cost_out, kp2);
    return cudaGetLastError();
}

cudaError_t launch_mask_costs(const float* cost, const int* sat, int n, float* cost_masked, int* n_sat,
                              cudaStream_t st) {
    k_mask_costs<<<1, 1024, 0, st>>>(cost, sat, n, cost_masked, n_sat);
    return cudaGetLastError();
}

cudaError_t launch_gather_soa_to_aos(const float* src, int ld_src, int nv, const int* idx, int k, float* out,
                                     cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    const int total = k * nv;
    k_gather_soa_to_aos<<<(total + 255) / 256, 256, 0, st>>>(src, ld_src, nv, idx, k, out);
    return cudaGetLastError();
}

}  // namespace spasm
