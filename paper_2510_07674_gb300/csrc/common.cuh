// Device building blocks of the SPaSM hot path for sm_103a.
//
// Everything here is FP32 unless templated on the scalar type (the final feasibility
// check instantiates the geometry in FP64).  Layouts:
//   cuboid  : 4 x float4 = centre (xyz, w = bounding radius), then the three columns of
//             its rotation R with the half extent along that column in w.
//   sphere  : float4 (x, y, z, r).
//   stage-1 particle state: SoA float[4B][n] (variable-major, block i uses rows 4i..4i+3:
//             x, y, z, yaw), so a warp's loads of one variable are coalesced.
//   stage-2 particle state: float[n][C][8] (configuration-major, 7 joints padded to 8),
//             one contiguous 32-byte record per configuration.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spasm {

constexpr int kMaxB = 16;          // blocks per problem
constexpr int kMaxRobotSpheres = 56;   // + 8 held-block spheres = 2 per lane
constexpr int kMaxCub = 256;       // environment cuboids (incl. table)
constexpr int kMaxOSph = 64;       // environment spheres
constexpr int kMaxC = 1024;        // configurations per trajectory particle
constexpr int kMaxNR = 9 * kMaxB + 3;
constexpr int kMaxCells = 64;      // unit cells over all blocks of a packing problem
enum GoalKind { kKindTower = 0, kKindPack = 1, kKindP2P = 2 };
constexpr float kPi = 3.14159265358979323846f;

// Scalars, robot tables and block tables: passed by value as a __grid_constant__ kernel
// parameter (about 3 KB, well inside the 32 KB parameter space of CUDA 12.1+).
struct Scalars {
    int B, S, C, NR;                 // blocks, steps per segment (W-1), configurations, residuals
    int n_rsph, n_cub, n_osph;       // robot spheres, env cuboids, env spheres
    int K_lin, K_quad, K_traj, K_al, K_ik;
    int N, M, P, Q;
    // robot: modified DH rows as (cos alpha, sin alpha, a, d), joint offsets, limits, tool
    float ca[7], sa[7], a[7], d[7], th0[7];
    float qlo[7], qhi[7];
    float ee_R[9], ee_p[3];
    float q_home[7];
    float4 rsph[kMaxRobotSpheres];   // x, y, z, r in the link frame
    int rlink[kMaxRobotSpheres];     // 0 = base
    float4 lbox_c[8], lbox_h[8];     // per link: box of its spheres in the link frame (centre, half
                                     // extents, slightly padded); half.x < 0 when the link has none
    float sweep[7];                  // per joint: bound on the distance from its axis to any robot or
                                     // held-block sphere centre it moves, so a step dq moves every
                                     // such centre by at most sum_j |dq_j| sweep[j]
    // blocks in stack order
    float4 half[kMaxB];              // hx, hy, hz, sphere radius min(h)/2
    float4 init[kMaxB];              // x, y, z, yaw
    float box_lo[3], box_hi[3];
    float z_table, grasp_off;
    float zt[kMaxB];                 // resting centre height of the block at stack position i
    float zlo[kMaxB];                // lower clamp of z for stack position i
    // optimiser parameters
    float eta_init, alpha, eta_traj, eps, eps_start;
    float w_stable, w_height, w_coll, w_start, w_arm, w_block, w_path, w_jl;
    float sqw[6];                    // sqrt of w_start, w_height, w_stable, w_coll, w_arm, w_block (float sqrt)
    float mu0, mu_max, ik_damp;
    int ik_mode;                     // lift IK: 0 damped least squares, 1 analytic (Franka joint layout)
    int sphere_tiling;               // trajectory kernels: sphere items per lane, 0 strided (lane + 32 k),
                                     // 1 blocked (2 lane + k); the same terms, summed in another order
    int particles_per_cta;           // trajectory kernels: particles a CTA runs at once, 1 or 2 (0 = 1)
    unsigned long long seed;
    // packing goal (the appendix's Tetris problem), kind = kKindPack: block i is a polyomino
    // of unit cubes of edge cell_size centred at cell[cell_start[i] .. cell_start[i+1]) in
    // its frame; the walls are the environment cuboids; z_star is the resting height
    int kind;
    int n_cells;
    int cell_start[kMaxB + 1];
    signed char cell_block[kMaxCells];   // block of each cell
    float2 cell[kMaxCells];
    float cell_size, z_star;
    float cell_reach[kMaxB];             // largest distance from a block's origin to a point of its cubes
};

// ------------------------------------------------------------------------------ launches
// Raise a kernel's dynamic shared-memory cap to the device's opt-in maximum (minus its
// static shared memory), once per (kernel, device) under a lock: host threads launching
// the kernel for problems of different sizes never change the attribute while another
// thread launches it.
// Runs `set` once per (kernel, device) while holding a process-wide lock.
cudaError_t configure_once_impl(const void* kernel, int dev, cudaError_t (*fn)(void*), void* ctx);
template <typename F>
inline cudaError_t configure_once(const void* kernel, int dev, F set) {
    return configure_once_impl(kernel, dev, [](void* c) { return (*static_cast<F*>(c))(); }, &set);
}

template <typename K>
inline cudaError_t allow_max_dynamic_smem(K kernel, size_t need) {
    int dev = 0, max_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int cap = max_optin - (int)fa.sharedSizeBytes;   // static + dynamic <= opt-in maximum
    if ((long long)need > (long long)cap) return cudaErrorInvalidValue;
    return configure_once(reinterpret_cast<const void*>(kernel), dev, [&] {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    });
}

// ------------------------------------------------------------------------------ errors
// Device error word (per problem): kernels record the first problem they see here and
// return early instead of trapping; the host reads it after the stream syncs.
enum DeviceError : int {
    kDevOk = 0,
    kDevTimeout = 1,       // a bounded wait (mbarrier / bulk copy) gave up
    kDevBadSize = 2,       // a size outside the compiled limits reached a kernel
};

__device__ __forceinline__ void set_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): key = (seed low, seed high), 4-word counter.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            unsigned long long seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// top 24 bits -> [0, 1): exact in binary32
__device__ __forceinline__ float u01(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }

enum PhiloxTag : uint32_t { kTagSample = 0, kTagGrasp = 1, kTagIkSeed = 2, kTagVia = 3, kTagQ6 = 4 };

// ------------------------------------------------------------------------------ warp helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------------------ geometry
// Penetration of sphere (c, r) into a cuboid, pen = max(0, -sd) with
//   p = R^T (c - centre), q = |p| - h,  sd = ||max(q,0)|| + min(max_k q_k, 0) - r.
// Split in two: cub_local gives p, q and max_k q_k; pen_finish turns them into pen and
// dpen/dc (zero when pen == 0).  The test max_k q_k >= r rejects separated pairs exactly
// (then sd >= 0) before any square root is taken.
template <typename T, typename V4>
__device__ __forceinline__ T cub_local(T cx, T cy, T cz, const V4& o, const V4& c0, const V4& c1, const V4& c2,
                                       T& p0, T& p1, T& p2, T& q0, T& q1, T& q2) {
    const T dx = cx - (T)o.x, dy = cy - (T)o.y, dz = cz - (T)o.z;
    p0 = (T)c0.x * dx + (T)c0.y * dy + (T)c0.z * dz;
    p1 = (T)c1.x * dx + (T)c1.y * dy + (T)c1.z * dz;
    p2 = (T)c2.x * dx + (T)c2.y * dy + (T)c2.z * dz;
    q0 = fabs(p0) - (T)c0.w; q1 = fabs(p1) - (T)c1.w; q2 = fabs(p2) - (T)c2.w;
    return q0 > q1 ? (q0 > q2 ? q0 : q2) : (q1 > q2 ? q1 : q2);
}

template <typename T, typename V4>
__device__ __forceinline__ T pen_finish(T p0, T p1, T p2, T q0, T q1, T q2, T qm, T r, const V4& c0, const V4& c1,
                                        const V4& c2, T& gx, T& gy, T& gz) {
    gx = gy = gz = (T)0;
    if (!(qm < r)) return (T)0;
    const T s0 = p0 >= (T)0 ? (T)1 : (T)-1, s1 = p1 >= (T)0 ? (T)1 : (T)-1, s2 = p2 >= (T)0 ? (T)1 : (T)-1;
    T pen, d0, d1, d2;   // dsd/dp
    if (qm > (T)0) {
        const T m0 = q0 > (T)0 ? q0 : (T)0, m1 = q1 > (T)0 ? q1 : (T)0, m2 = q2 > (T)0 ? q2 : (T)0;
        const T n2 = m0 * m0 + m1 * m1 + m2 * m2;
        if (!(n2 < r * r)) return (T)0;
        const T n = sqrt(n2);
        pen = r - n;
        const T inv = (T)1 / n;
        d0 = s0 * m0 * inv; d1 = s1 * m1 * inv; d2 = s2 * m2 * inv;
    } else {
        pen = r - qm;
        // argmax with the lowest index on ties
        int ax = 0;
        T best = q0;
        if (q1 > best) { ax = 1; best = q1; }
        if (q2 > best) { ax = 2; }
        d0 = ax == 0 ? s0 : (T)0; d1 = ax == 1 ? s1 : (T)0; d2 = ax == 2 ? s2 : (T)0;
        if (!(pen > (T)0)) return (T)0;
    }
    // dpen/dc = -R dsd/dp
    gx = -((T)c0.x * d0 + (T)c1.x * d1 + (T)c2.x * d2);
    gy = -((T)c0.y * d0 + (T)c1.y * d1 + (T)c2.y * d2);
    gz = -((T)c0.z * d0 + (T)c1.z * d1 + (T)c2.z * d2);
    return pen;
}

template <typename T, typename V4>
__device__ __forceinline__ T pen_cuboid(T cx, T cy, T cz, T r, const V4& o, const V4& c0, const V4& c1,
                                        const V4& c2, T& gx, T& gy, T& gz) {
    T p0, p1, p2, q0, q1, q2;
    const T qm = cub_local<T, V4>(cx, cy, cz, o, c0, c1, c2, p0, p1, p2, q0, q1, q2);
    return pen_finish<T, V4>(p0, p1, p2, q0, q1, q2, qm, r, c0, c1, c2, gx, gy, gz);
}

template <typename T, typename V4>
__device__ __forceinline__ T pen_sphere(T cx, T cy, T cz, T r, const V4& s, T& gx, T& gy, T& gz) {
    T dx = cx - (T)s.x, dy = cy - (T)s.y, dz = cz - (T)s.z;
    T rr = r + (T)s.w;
    T n2 = dx * dx + dy * dy + dz * dz;
    gx = gy = gz = (T)0;
    if (!(n2 < rr * rr)) return (T)0;
    T n = sqrt(n2);
    T pen = rr - n;
    if (n > (T)0) { T inv = (T)1 / n; gx = -dx * inv; gy = -dy * inv; gz = -dz * inv; }
    return pen;
}

// Cuboid of an upright block pose (x, y, z, yaw): columns of Rz(yaw).
__device__ __forceinline__ void block_cuboid(float x, float y, float z, float yaw, const float4& h, float4* out) {
    float s, c;
    sincosf(yaw, &s, &c);
    out[0] = make_float4(x, y, z, 0.f);
    out[1] = make_float4(c, s, 0.f, h.x);
    out[2] = make_float4(-s, c, 0.f, h.y);
    out[3] = make_float4(0.f, 0.f, 1.f, h.z);
}

// Sphere m of a block (objects as sphere sets): (+-hx/2, +-hy/2, +-hz/2), bit 0/1/2 of m
// selects the sign along x/y/z.
__device__ __forceinline__ void block_sphere_local(const float4& h, int m, float& lx, float& ly, float& lz) {
    lx = ((m & 1) ? 0.5f : -0.5f) * h.x;
    ly = ((m & 2) ? 0.5f : -0.5f) * h.y;
    lz = ((m & 4) ? 0.5f : -0.5f) * h.z;
}

// ------------------------------------------------------------------------------ kinematics
// One modified-DH link transform T = Rx(alpha) Tx(a) Rz(theta) Tz(d) applied to the running
// frame (R row-major, o):  R <- R * Rk,  o <- o + R * tk, with
//   Rk = [[ct, -st, 0], [ca st, ca ct, -sa], [sa st, sa ct, ca]],  tk = (a, -sa d, ca d).
template <typename T>
__device__ __forceinline__ void dh_step(T R[9], T o[3], T ca, T sa, T a, T d, T ct, T st) {
    T tk0 = a, tk1 = -sa * d, tk2 = ca * d;
    T n[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
        o[i] += r0 * tk0 + r1 * tk1 + r2 * tk2;
        n[3 * i + 0] = r0 * ct + r1 * (ca * st) + r2 * (sa * st);
        n[3 * i + 1] = -r0 * st + r1 * (ca * ct) + r2 * (sa * ct);
        n[3 * i + 2] = -r1 * sa + r2 * ca;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = n[i];
}

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }

// Tool frame from frame 7: R_tool = R7 ee_R, p_tool = o7 + R7 ee_p.
template <typename T>
__device__ __forceinline__ void tool_frame(const Scalars& sc, const T R7[9], const T o7[3], T Rt[9], T pt[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Rt[3 * i + j] = R7[3 * i] * (T)sc.ee_R[j] + R7[3 * i + 1] * (T)sc.ee_R[3 + j] + R7[3 * i + 2] * (T)sc.ee_R[6 + j];
        pt[i] = o7[i] + R7[3 * i] * (T)sc.ee_p[0] + R7[3 * i + 1] * (T)sc.ee_p[1] + R7[3 * i + 2] * (T)sc.ee_p[2];
    }
}

// Full FK of one configuration: frames 1..7 as (R, o), and the tool frame.
template <typename T>
__device__ __forceinline__ void fk_full(const Scalars& sc, const T q[7], T R[8][9], T o[8][3], T Rt[9], T pt[3]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) R[0][i] = (i % 4 == 0) ? (T)1 : (T)0;
    o[0][0] = o[0][1] = o[0][2] = (T)0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        T s, c;
        sincos_t((T)sc.th0[k] + q[k], &s, &c);
#pragma unroll
        for (int i = 0; i < 9; ++i) R[k + 1][i] = R[k][i];
        o[k + 1][0] = o[k][0]; o[k + 1][1] = o[k][1]; o[k + 1][2] = o[k][2];
        dh_step<T>(R[k + 1], o[k + 1], (T)sc.ca[k], (T)sc.sa[k], (T)sc.a[k], (T)sc.d[k], c, s);
    }
    tool_frame<T>(sc, R[7], o[7], Rt, pt);
}

// Block frame held by the tool (top-down grasp): R_blk = R_tool diag(1,-1,-1),
// p_blk = p_tool + (hz + grasp_off) z_tool.
template <typename T>
__device__ __forceinline__ void held_block(const Scalars& sc, int b, const T Rt[9], const T pt[3], T Rb[9], T pb[3]) {
    T off = (T)sc.half[b].z + (T)sc.grasp_off;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Rb[3 * i] = Rt[3 * i];
        Rb[3 * i + 1] = -Rt[3 * i + 1];
        Rb[3 * i + 2] = -Rt[3 * i + 2];
        pb[i] = pt[i] + off * Rt[3 * i + 2];
    }
}

// ------------------------------------------------------------------------------ TMA bulk copy
// Stage a contiguous global table into shared memory with the bulk-copy engine
// (cp.async.bulk, completion on an mbarrier).  Addresses and size must be multiples of
// 16 bytes.  The wait is bounded: after `max_polls` unsuccessful polls the error word
// is set and the function returns false (the caller then falls back to nothing: it
// skips its work and exits).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Polls phase `phase` of an mbarrier at most max_polls times; true once it has completed.
constexpr int kTablePolls = 1 << 22;   // about a second of polling
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int max_polls) {
    for (int polls = 0; polls < max_polls; ++polls)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// Copies up to two tables; every thread of the CTA calls it; returns false on timeout.
// `init`: initialise the barrier first (its first use in the CTA); `phase`: parity of the
// barrier phase this copy completes (0 for the first use, then alternating).
__device__ __forceinline__ bool stage_tables(void* dst0, const void* src0, uint32_t bytes0, void* dst1, const void* src1,
                                             uint32_t bytes1, uint64_t* bar, int* err, bool init = true,
                                             uint32_t phase = 0) {
    if (init && threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes0 + bytes1);
        if (bytes0) bulk_g2s(dst0, src0, bytes0, bar);
        if (bytes1) bulk_g2s(dst1, src1, bytes1, bar);
    }
    const bool done = mbar_wait_bounded(bar, phase, kTablePolls);
    if (!done) {
        set_error(err, kDevTimeout);
        // the copies this CTA issued may still be landing in its shared memory: give them a
        // second bounded wait before the CTA exits
        mbar_wait_bounded(bar, phase, kTablePolls);
    }
    int all = __syncthreads_and(done ? 1 : 0);
    return all != 0;
}

}  // namespace spasm
