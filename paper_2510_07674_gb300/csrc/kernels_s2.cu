// Stage-2 kernels: the fused trajectory optimisation (one CTA per particle, every
// iteration inside one launch).  The lift that initialises it is in kernels_lift.cu.
#include <cuda_fp16.h>

#include "launch_s2.h"
#include "stage1.cuh"
#include "stage2.cuh"

namespace spasm {

// ================================================================================== trajopt
constexpr int kTWarps = 8;
constexpr int kTThreads = 32 * kTWarps;
constexpr int kSlots = 2;   // sphere items per lane: up to 56 robot + 8 held-block spheres

constexpr int kChunk = 4;   // configurations whose kinematics one warp evaluates together

// A trajectory CTA runs 1 or 2 particles at once (particles per CTA, a launch option): each on
// its own group of kTThreads threads, with its own region of dynamic shared memory and its own
// named barrier 1 + group.  With one particle the group is the whole CTA.
template <int kPpc>
__device__ __forceinline__ int grp_tid() { return kPpc == 1 ? (int)threadIdx.x : (int)(threadIdx.x & (kTThreads - 1)); }
template <int kPpc>
__device__ __forceinline__ int grp_index() { return kPpc == 1 ? 0 : (int)(threadIdx.x / kTThreads); }
template <int kPpc>
__device__ __forceinline__ void grp_sync() {
    if (kPpc == 1) __syncthreads();
    else if (threadIdx.x < kTThreads) asm volatile("bar.sync 1, %0;" ::"n"(kTThreads) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"n"(kTThreads) : "memory");
}

// Cached cull.  When a chunk's cull finds no candidate for any of its configurations, it
// also returns the chunk's clearances: the smallest separation (largest per-axis gap) between
// any of its link boxes and any static box that could touch it (the environment, blocks at
// their initial poses), and the same for the placed blocks, which move: the top one (the
// highest block placed before the chunk's last block) on its own, the ones below it together.
// Later iterations skip the chunk (kinematics, cull and tests: its terms are zero) while the
// bound on how far its spheres moved since stays below the static clearance, plus the top
// block's own motion since below the clearance to it, and plus a bound on how far any one of
// the blocks below the top one moved below the clearance to those, so the skipped work is
// exactly the work whose result is zero.  A chunk whose configurations have
// candidates but whose spheres all miss them (no penetration anywhere: its terms are zero as
// well) is kept the same way; for the obstacles its spheres were tested against, its
// clearance is the smallest sphere-level gap those tests found.
constexpr float kClearSlack = 1e-5f;   // FP32 rounding of the boxes, metres

// Work queue of an evaluation: its items (the chunks, the residual jobs, the slices of the
// placed tower's collisions) go to the warps in list order from a shared counter, the larger
// items first, so that the warps finish together.  What the items add up goes into fixed-point
// accumulators (integer sums are exact, hence independent of which warp took which item and
// when): a value v becomes round(v 2^40), |v| < 8e6.
constexpr float kFix = 1099511627776.f;   // 2^40
__device__ __forceinline__ void fx_add(long long* acc, float v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)__float2ll_rn(v * kFix));
}
__device__ __forceinline__ float fx_value(long long a) { return __ll2float_rn(a) * (1.f / kFix); }
constexpr int kPlaceUnits = (8 * kMaxB + 31) / 32;   // slices of 32 block spheres of the placed tower
constexpr int kResidualJobs = 2;                      // placement residuals; start residuals

struct TWarp {
    float4 F[kChunk][8][3];  // frames 0..7 of each configuration of the chunk: rows (R_i0, R_i1, R_i2, o_i)
    float4 H[kChunk][3];     // held-block frame of each configuration (same row layout)
    float part[4];           // this warp's path length and joint-limit sums [0, 1], maximum penetration [2]
    uint32_t cmask[kChunk][kMaxCub / 32];    // environment cuboids that may touch configuration c of the chunk
    uint32_t smask[kChunk][kMaxOSph / 32];   // environment spheres that may touch configuration c
    uint32_t bmask[2][kChunk];               // placed / not-yet-moved blocks that may touch configuration c
    uint32_t envany[kChunk];                 // configuration c has an environment candidate
};

// Frames of one configuration kept for the epilogue (grasp and place configurations).
struct SpecialFrames {
    float4 F[8][3];
    float4 H[3];
};

struct TShared {
    float4 bcub[kMaxB][4];   // placed-block cuboids of this iteration
    float4 icub[kMaxB][4];   // initial-pose cuboids
    float4 baabb[kMaxB][2];  // their axis-aligned boxes (lo, hi)
    float4 iaabb[kMaxB][2];
    float pose[4 * kMaxB];   // placed poses (x, y, z, yaw)
    float g4[4 * kMaxB];     // dL/d(placed pose)
    float h[kMaxNR], lam[kMaxNR], s[kMaxNR];
    // gradient rows of the grasp (b) and place (B + b) configurations; until the gradient pass
    // overwrites them, their first 6 floats hold the residual pass's (w_roll, w_pitch) of that block frame
    float extra[2 * kMaxB][8];
    float pg[kMaxB][4];                // dC_coll/d(placed pose j), sphere side (from the slice holding block j)
    float pgc[kPlaceUnits][kMaxB][4];  // dC_coll/d(placed pose i), cuboid side of block pairs, per slice
    float pcu[kPlaceUnits][2];         // per slice: sum and maximum of the tower's penetrations
    long long fx_wr[2][kMaxB][4];      // d/d(placed pose k) of the arm and block groups (fixed point)
    long long fx_arm, fx_blk;          // C_arm, C_block (fixed point)
    int next;                          // the work queue's counter
    PlaceScratch ps;
    float4 dh[8];            // joint j: cos alpha, sin alpha, a, d (per-lane reads in the kinematics)
    float th0[8];            // joint offsets
    float4 lbc[8], lbh[8];   // link-frame boxes of each link's spheres (centre, half extents)
    float s_arm, s_blk, mu, L;
    float pose_prev[4 * kMaxB];   // placed poses of the previous evaluation
    // chunks to evaluate by tier (kChunk .. 1 configurations with candidates at the last cull, then the
    // candidate-free ones to cull again): active[tier][32g + i] for group g
    unsigned char active[kChunk + 1][(kMaxC + kChunk - 1) / kChunk];
    short n_group[kChunk + 1][kTWarps];
    unsigned skip[kTWarps];       // bit i of word g: chunk 32g + i kept its cached cull this evaluation
    float blk_cum[kMaxB];         // [k]: sum over the evaluations of the largest motion among the placed blocks 0..k
    float bown[kMaxB];            // [k]: sum over the evaluations of placed block k's own motion
    int pose_prev_ok;
    float c_arm, c_blk, maxpen, c_coll, c_stable, c_height, c_start;
    float max_start, max_tilt, pm_pen, pm_D, pm_dz, path, jl;
    TWarp warp[kTWarps];
};

__host__ __device__ inline size_t t_env_offset() { return 16; }
__host__ __device__ inline size_t t_aabb_offset(int n_cub, int n_osph) {
    return (16 + (size_t)n_cub * 64 + (size_t)n_osph * 16 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t t_shared_offset(int n_cub, int n_osph) {
    return t_aabb_offset(n_cub, n_osph) + (size_t)(n_cub + n_osph) * 32;
}
__host__ __device__ inline size_t t_q_offset(int n_cub, int n_osph) {
    return (t_shared_offset(n_cub, n_osph) + sizeof(TShared) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t t_sp_offset(int n_cub, int n_osph, int C) {
    return t_q_offset(n_cub, n_osph) + (size_t)3 * C * 8 * sizeof(float);
}
__host__ __device__ inline int t_n_chunks(int C) { return (C - 1 + kChunk - 1) / kChunk; }
// cached cull state: per configuration the motion bound since its chunk's last cull; per
// chunk, at that cull, the motion bound of the placed blocks below its top block and the top
// block's own motion, its (static, moving) clearances as an fp16 pair, how many of its
// configurations had a candidate (0: none, the chunk's cull is cacheable) and its fp16
// clearance to the top block
__host__ __device__ inline size_t t_cache_offset(int n_cub, int n_osph, int C, int B) {
    return (t_sp_offset(n_cub, n_osph, C) + (size_t)2 * B * sizeof(SpecialFrames) + 15) & ~(size_t)15;
}
size_t traj_smem_bytes(const Scalars& sc) {
    return t_cache_offset(sc.n_cub, sc.n_osph, sc.C, sc.B) + (size_t)sc.C * sizeof(float) +
           (size_t)t_n_chunks(sc.C) * (3 * sizeof(float) + sizeof(int) + sizeof(__half));
}

// Sphere item held in slot k by a lane: strided tiling, item lane + 32 k (the spheres of a link
// spread over neighbouring lanes), or blocked tiling, item kSlots lane + k (a lane's spheres are
// neighbours, mostly on one link).  Either covers 64 items; the choice reorders the per-lane
// sums only.
template <int kTile>
__device__ __forceinline__ int slot_item(int lane, int k) {
    return kTile ? kSlots * lane + k : lane + 32 * k;
}

// The robot spheres a lane owns (slot_item), loaded once per kernel launch: link-frame centre,
// radius, link index.  Items beyond the robot spheres are the held block's.
struct LaneSpheres {
    float lx[kSlots], ly[kSlots], lz[kSlots], r[kSlots];
    int link[kSlots];
};

template <int kTile>
__device__ __forceinline__ LaneSpheres lane_spheres(const Scalars& sc) {
    const int lane = threadIdx.x & 31;
    LaneSpheres ls;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
        const int it = slot_item<kTile>(lane, k);
        if (it < sc.n_rsph) {
            const float4 v = sc.rsph[it];
            ls.lx[k] = v.x; ls.ly[k] = v.y; ls.lz[k] = v.z; ls.r[k] = v.w;
            ls.link[k] = sc.rlink[it];
        } else {
            ls.lx[k] = ls.ly[k] = ls.lz[k] = ls.r[k] = 0.f;
            ls.link[k] = 7;
        }
    }
    return ls;
}

// Forward kinematics of four configurations by one warp: lane 8c + k holds link transform
// k of configuration t_c (k = 0: identity), and a 3-level inclusive scan of affine products
// inside each group of 8 lanes gives frame_k = T_1 ... T_k.  Group c writes its frames (rows
// (R_i0, R_i1, R_i2, o_i)) to F_c, unless `write` is false for that group, and, when
// `want_h`, the frame of the block the tool would hold in t_c's segment to H_c.  With `box`,
// the lane also returns a world box (lo xyz, hi xyz) that holds every sphere of link k (and of
// the held block, at k = 7 with `want_h`): the link-frame box of those spheres carried by the
// frame, i.e. centre R c + o and half extents |R| h.
__device__ __forceinline__ void chunk_fk(const Scalars& sc, const TShared& sh, const float* __restrict__ q, int t_c,
                                         bool write, bool want_h, float4 (*F_c)[3], float4* H_c, float* box) {
    const int lane = threadIdx.x & 31;
    const int k = lane & 7;
    const int t = min(max(t_c, 1), sc.C - 1);
    float A[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, bv[3] = {0, 0, 0};
    if (k > 0) {
        const int j = k - 1;
        float st, ct;
        sincosf(sh.th0[j] + q[t * 8 + j], &st, &ct);
        const float4 row = sh.dh[j];
        const float ca = row.x, sa = row.y;
        A[0] = ct;      A[1] = -st;     A[2] = 0.f;
        A[3] = ca * st; A[4] = ca * ct; A[5] = -sa;
        A[6] = sa * st; A[7] = sa * ct; A[8] = ca;
        bv[0] = row.z; bv[1] = -sa * row.w; bv[2] = ca * row.w;
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
        float L[9], lb[3];
#pragma unroll
        for (int i = 0; i < 9; ++i) L[i] = __shfl_up_sync(0xffffffffu, A[i], off, 8);
#pragma unroll
        for (int i = 0; i < 3; ++i) lb[i] = __shfl_up_sync(0xffffffffu, bv[i], off, 8);
        if (k >= off) {
            float nA[9], nb[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    nA[3 * r + cc] = L[3 * r] * A[cc] + L[3 * r + 1] * A[3 + cc] + L[3 * r + 2] * A[6 + cc];
                nb[r] = L[3 * r] * bv[0] + L[3 * r + 1] * bv[1] + L[3 * r + 2] * bv[2] + lb[r];
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) A[i] = nA[i];
#pragma unroll
            for (int i = 0; i < 3; ++i) bv[i] = nb[i];
        }
    }
    if (box) {
        const float4 lc = sh.lbc[k], lh = sh.lbh[k];
        const bool has = lh.x >= 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float w = A[3 * r] * lc.x + A[3 * r + 1] * lc.y + A[3 * r + 2] * lc.z + bv[r];
            const float e = fabsf(A[3 * r]) * lh.x + fabsf(A[3 * r + 1]) * lh.y + fabsf(A[3 * r + 2]) * lh.z;
            box[r] = has ? w - e : 3.4e38f;
            box[3 + r] = has ? w + e : -3.4e38f;
        }
    }
    if (!write) return;
#pragma unroll
    for (int r = 0; r < 3; ++r) F_c[k][r] = make_float4(A[3 * r], A[3 * r + 1], A[3 * r + 2], bv[r]);
    if (k == 7 && want_h) {
        const int seg = (t - 1) / sc.S, b = seg >> 1;
        float Rt[9], pt[3], Rb[9], pb[3];
        tool_frame<float>(sc, A, bv, Rt, pt);
        held_block<float>(sc, b, Rt, pt, Rb, pb);
#pragma unroll
        for (int r = 0; r < 3; ++r) H_c[r] = make_float4(Rb[3 * r], Rb[3 * r + 1], Rb[3 * r + 2], pb[r]);
        if (box) {
            // held-block spheres sit at (+-hx/2, +-hy/2, +-hz/2) with radius r_b in the block frame
            const float4 hb = sc.half[b];
            const float ex = 0.5f * hb.x + hb.w + 1e-5f, ey = 0.5f * hb.y + hb.w + 1e-5f, ez = 0.5f * hb.z + hb.w + 1e-5f;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float e = fabsf(Rb[3 * r]) * ex + fabsf(Rb[3 * r + 1]) * ey + fabsf(Rb[3 * r + 2]) * ez;
                box[r] = fminf(box[r], pb[r] - e);
                box[3 + r] = fmaxf(box[3 + r], pb[r] + e);
            }
        }
    }
}

// World centres of the lane's sphere items for one configuration (frames F, held-block
// frame H); items beyond the robot spheres are the held block's (transfer interior only).
template <int kTile>
__device__ __forceinline__ void sphere_centres(const Scalars& sc, const LaneSpheres& ls, const float4 (*F)[3],
                                               const float4* H, int n_items, int b, float* cx, float* cy, float* cz,
                                               float* rr, bool* act, bool* isblk) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
        const int it = slot_item<kTile>(lane, k);
        act[k] = it < n_items;
        isblk[k] = act[k] && it >= sc.n_rsph;
        float x = ls.lx[k], y = ls.ly[k], z = ls.lz[k];
        float4 r0, r1, r2;
        if (isblk[k]) {
            block_sphere_local(sc.half[b], it - sc.n_rsph, x, y, z);
            r0 = H[0]; r1 = H[1]; r2 = H[2];
            rr[k] = sc.half[b].w;
        } else {
            const int l = ls.link[k];
            r0 = F[l][0]; r1 = F[l][1]; r2 = F[l][2];
            rr[k] = act[k] ? ls.r[k] : 0.f;
        }
        cx[k] = r0.x * x + r0.y * y + r0.z * z + r0.w;
        cy[k] = r1.x * x + r1.y * y + r1.z * z + r1.w;
        cz[k] = r2.x * x + r2.y * y + r2.z * z + r2.w;
    }
}

// Collision terms of the configurations t0 .. t0+nc-1 (kinematics in the warp's frames),
// evaluated by one warp: arm spheres and, on the transfer interior, the held block's spheres
// against the environment and the context blocks.  An exact cull first keeps the obstacles
// whose boxes overlap the box of all spheres of the chunk (consecutive waypoints are close);
// per configuration lanes own sphere items, screen both slots branch-free and evaluate the
// penetration only where the separation test fails.  With `grad`, writes the unscaled group
// gradients G_arm[t], G_blk[t] and accumulates placed-pose derivatives in the warp scratch.
// Returns whether the chunk's collision terms are zero (no candidate, or candidates that no
// sphere penetrates); then `clearance` / `clearance_top` / `clearance_moving` bound from below
// how far any of its spheres is from a static box / the top placed block it could touch (the
// block below the chunk's last block) / the other placed blocks: the gaps between link boxes
// and the boxes apart from them, and the sphere-level gaps of the tests that ran.
template <int kTile>
__device__ __forceinline__ bool chunk_collisions(const Scalars& sc, const LaneSpheres& ls,
                                                 const float4* __restrict__ cub, const float4* __restrict__ osph,
                                                 const float4* __restrict__ aabb, TShared& sh, TWarp& tw, float* G_arm,
                                                 float* G_blk, int t0, int nc, bool grad, const float* lane_box,
                                                 float& acc_arm, float& acc_blk, float& acc_max,
                                                 unsigned long long& n_tests, unsigned long long& n_cand,
                                                 float& clearance, float& clearance_moving, float& clearance_top) {
    const int lane = threadIdx.x & 31;
    const int S = sc.S, B = sc.B;
    float cx[kSlots], cy[kSlots], cz[kSlots], rr[kSlots];
    bool act[kSlots], isblk[kSlots];

    // pass 1: box of every sphere of the chunk (union of the lanes' link boxes), candidate
    // obstacles by warp ballots
    float lo_x = lane_box[0], lo_y = lane_box[1], lo_z = lane_box[2];
    float hi_x = lane_box[3], hi_y = lane_box[4], hi_z = lane_box[5];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, off));
        lo_y = fminf(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, off));
        lo_z = fminf(lo_z, __shfl_xor_sync(0xffffffffu, lo_z, off));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, off));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, off));
        hi_z = fmaxf(hi_z, __shfl_xor_sync(0xffffffffu, hi_z, off));
    }
    // separation of a box from the chunk box: the largest per-axis gap, > 0 iff they are apart
    auto sep_chunk = [&](const float4& blo, const float4& bhi) {
        return fmaxf(fmaxf(fmaxf(blo.x - hi_x, lo_x - bhi.x), fmaxf(blo.y - hi_y, lo_y - bhi.y)),
                     fmaxf(blo.z - hi_z, lo_z - bhi.z));
    };
    // second level: each candidate of the chunk box against the lanes' own link boxes (lane
    // 8c + k: link k of configuration c); configuration c keeps the candidate when one of its
    // link boxes overlaps the candidate's box.  Both levels are exact: no sphere inside the
    // boxes is dropped.  Every box apart from the chunk box, or from a lane's link box, that
    // the lane's configuration could touch lowers the lane's clearance to that separation.
    const float* lb = lane_box;
    float clear = 3.4e38f;
    auto refine = [&](unsigned m, int base, const float4* boxes, int stride, uint32_t out[kChunk], auto relevant) {
#pragma unroll
        for (int c = 0; c < kChunk; ++c) out[c] = 0u;
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            const float4 blo = boxes[stride * (base + bit)], bhi = boxes[stride * (base + bit) + 1];
            const float s2 = fmaxf(fmaxf(fmaxf(blo.x - lb[3], lb[0] - bhi.x), fmaxf(blo.y - lb[4], lb[1] - bhi.y)),
                                   fmaxf(blo.z - lb[5], lb[2] - bhi.z));
            // a box that overlaps this link's box is tested against the spheres, which give the gap
            if (relevant(bit) && s2 > 0.f) clear = fminf(clear, s2);
            const unsigned bal = __ballot_sync(0xffffffffu, s2 <= 0.f);
#pragma unroll
            for (int c = 0; c < kChunk; ++c)
                if ((bal >> (8 * c)) & 0xffu) out[c] |= 1u << bit;
        }
    };
    // link 0 (lane k = 0) is the fixed base: its gaps to static boxes (the environment, blocks
    // at their initial poses) never shrink and do not bound the clearance
    const bool moving_link = (lane & 7) != 0;
    auto moving = [&](int) { return moving_link; };
    const int n_cw = (sc.n_cub + 31) >> 5, n_sw = (sc.n_osph + 31) >> 5;
    uint32_t per[kChunk], any[kChunk] = {0u, 0u, 0u, 0u};
    for (int wd = 0; wd < n_cw; ++wd) {
        const int oi = 32 * wd + lane;
        const float s1 = oi < sc.n_cub ? sep_chunk(aabb[2 * oi], aabb[2 * oi + 1]) : 3.4e38f;
        clear = fminf(clear, s1 > 0.f ? s1 : 3.4e38f);
        const unsigned m = __ballot_sync(0xffffffffu, s1 <= 0.f);
        refine(m, 32 * wd, aabb, 2, per, moving);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < kChunk; ++c) tw.cmask[c][wd] = per[c];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) any[c] |= per[c];
    }
    for (int wd = 0; wd < n_sw; ++wd) {
        const int oi = 32 * wd + lane;
        const int ai = sc.n_cub + oi;
        const float s1 = oi < sc.n_osph ? sep_chunk(aabb[2 * ai], aabb[2 * ai + 1]) : 3.4e38f;
        clear = fminf(clear, s1 > 0.f ? s1 : 3.4e38f);
        const unsigned m = __ballot_sync(0xffffffffu, s1 <= 0.f);
        refine(m, sc.n_cub + 32 * wd, aabb, 2, per, moving);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < kChunk; ++c) tw.smask[c][wd] = per[c];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) any[c] |= per[c];
    }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < kChunk; ++c) tw.envany[c] = any[c];
    // the highest placed block a configuration of the chunk can touch: it moves by its own motion,
    // the blocks below it by at most the largest motion among them
    const int top = ((min(t0 + nc - 1, sc.C - 1) - 1) / S >> 1) - 1;
    {
        // a configuration of block b's segments can touch the placed blocks k < b and the
        // blocks k > b still at their initial poses (the chunk: any of its configurations)
        const int b_lane = (min(t0 + (lane >> 3), sc.C - 1) - 1) / S >> 1;
        const int b_first = (t0 - 1) / S >> 1, b_last = (min(t0 + nc - 1, sc.C - 1) - 1) / S >> 1;
        // blocks at their initial poses (static), then the placed blocks (moving): the clearance
        // so far is the static one, and the placed blocks' gaps form the moving one
        const float si = lane < B ? sep_chunk(sh.iaabb[lane][0], sh.iaabb[lane][1]) : 3.4e38f;
        if (lane < B && lane > b_first && si > 0.f) clear = fminf(clear, si);
        const unsigned bm_init = __ballot_sync(0xffffffffu, si <= 0.f);
        refine(bm_init, 0, &sh.iaabb[0][0], 2, per, [&](int k) { return k > b_lane && moving_link; });
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < kChunk; ++c) tw.bmask[1][c] = per[c];
        clearance = warp_min(clear);
        clear = 3.4e38f;
        const float sp = lane < B ? sep_chunk(sh.baabb[lane][0], sh.baabb[lane][1]) : 3.4e38f;
        if (lane < b_last && lane != top && sp > 0.f) clear = fminf(clear, sp);
        const unsigned bm_placed = __ballot_sync(0xffffffffu, sp <= 0.f);
        refine(bm_placed, 0, &sh.baabb[0][0], 2, per, [&](int k) { return k < b_lane && k != top; });
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < kChunk; ++c) tw.bmask[0][c] = per[c];
        clearance_moving = warp_min(clear);
        // the top block: the gap from each link box of the configurations it concerns
        float ct = 3.4e38f;
        if (top >= 0 && top < b_lane) {
            const float4 blo = sh.baabb[top][0], bhi = sh.baabb[top][1];
            const float g = fmaxf(fmaxf(fmaxf(blo.x - lb[3], lb[0] - bhi.x), fmaxf(blo.y - lb[4], lb[1] - bhi.y)),
                                  fmaxf(blo.z - lb[5], lb[2] - bhi.z));
            if (g > 0.f) ct = g;   // an overlapping box is tested against the spheres, which give the gap
        }
        clearance_top = warp_min(ct);
    }
    __syncwarp();

    // pass 2: every configuration against the candidates.  gap_s / gap_m / gap_t: the lane's smallest
    // sphere-level gap (lower bound) to a tested static box / placed block below the top one / the
    // top placed block; the fixed base's
    // spheres do not move relative to static boxes and are left out of gap_s.
    const int seg0 = (t0 - 1) / S, r0 = (t0 - 1) - seg0 * S;
    bool none = true, chunk_hit = false;
    float gap_s = 3.4e38f, gap_m = 3.4e38f, gap_t = 3.4e38f;
    for (int ci = 0; ci < nc; ++ci) {
        const int t = t0 + ci;
        int seg = seg0, r = r0 + ci;
        while (r >= S) { r -= S; ++seg; }
        const int b = seg >> 1, jj = r + 1;
        const bool held = (seg & 1) && jj < S;
        const int n_items = sc.n_rsph + (held ? 8 : 0);
        // candidates of this configuration: environment (any mask bit), context blocks placed
        // (k < b, movable) and not yet moved (k > b).  Without any, its collision terms and
        // their gradient are zero and the sphere centres are not needed.
        const bool env_c = tw.envany[ci] != 0u;
        const unsigned below = (1u << b) - 1u;
        const unsigned ctx = (tw.bmask[0][ci] & below) | (tw.bmask[1][ci] & ~below & ~(1u << b));
        if (!env_c && ctx == 0u) {
            if (grad && lane < 16 && (lane & 7) != 7) (lane < 8 ? G_arm : G_blk)[t * 8 + (lane & 7)] = 0.f;
            continue;
        }
        none = false;
        ++n_cand;
        sphere_centres<kTile>(sc, ls, tw.F[ci], tw.H[ci], n_items, b, cx, cy, cz, rr, act, isblk);
        bool fixed[kSlots];
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) fixed[sl] = !isblk[sl] && ls.link[sl] == 0;
        float gx[kSlots], gy[kSlots], gz[kSlots], pen_sum[kSlots];
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) gx[sl] = gy[sl] = gz[sl] = pen_sum[sl] = 0.f;
        bool any_hit = false;
        int visits = 0;

        for (int wd = 0; wd < (env_c ? n_cw : 0); ++wd) {
            unsigned m = tw.cmask[ci][wd];
            visits += __popc(m);
            while (m) {
                const int ob = 32 * wd + __ffs(m) - 1;
                m &= m - 1;
                const float4 o0 = cub[4 * ob], o1 = cub[4 * ob + 1], o2 = cub[4 * ob + 2], o3 = cub[4 * ob + 3];
                float p0[kSlots], p1[kSlots], p2[kSlots], q0[kSlots], q1[kSlots], q2[kSlots], qm[kSlots];
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl)
                    qm[sl] = cub_local<float>(cx[sl], cy[sl], cz[sl], o0, o1, o2, o3, p0[sl], p1[sl], p2[sl], q0[sl],
                                              q1[sl], q2[sl]);
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl) {
                    // separated along a box axis by qm: the sphere is at least qm - r from the box
                    if (act[sl] && !fixed[sl]) gap_s = fminf(gap_s, fmaxf(qm[sl] - rr[sl], 0.f));
                    if (!act[sl] || !(qm[sl] < rr[sl])) continue;
                    float ax, ay, az;
                    const float pen = pen_finish<float>(p0[sl], p1[sl], p2[sl], q0[sl], q1[sl], q2[sl], qm[sl], rr[sl],
                                                        o1, o2, o3, ax, ay, az);
                    if (pen > 0.f) {
                        any_hit = true;
                        pen_sum[sl] += pen;
                        acc_max = fmaxf(acc_max, pen);
                        gx[sl] += ax; gy[sl] += ay; gz[sl] += az;
                    }
                }
            }
        }
        for (int wd = 0; wd < (env_c ? n_sw : 0); ++wd) {
            unsigned m = tw.smask[ci][wd];
            visits += __popc(m);
            while (m) {
                const int ob = 32 * wd + __ffs(m) - 1;
                m &= m - 1;
                const float4 os = osph[ob];
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl) {
                    if (!act[sl]) continue;
                    if (!fixed[sl]) {
                        // the largest per-axis offset bounds the centre distance from below
                        const float dm = fmaxf(fmaxf(fabsf(cx[sl] - os.x), fabsf(cy[sl] - os.y)), fabsf(cz[sl] - os.z));
                        gap_s = fminf(gap_s, fmaxf(dm - rr[sl] - os.w, 0.f));
                    }
                    float ax, ay, az;
                    const float pen = pen_sphere<float>(cx[sl], cy[sl], cz[sl], rr[sl], os, ax, ay, az);
                    if (pen > 0.f) {
                        any_hit = true;
                        pen_sum[sl] += pen;
                        acc_max = fmaxf(acc_max, pen);
                        gx[sl] += ax; gy[sl] += ay; gz[sl] += az;
                    }
                }
            }
        }
        // context blocks
        {
            unsigned m = ctx;
            visits += __popc(m);
            while (m) {
                const int kb = __ffs(m) - 1;
                m &= m - 1;
                const bool placed = kb < b;
                const float4* cb = placed ? sh.bcub[kb] : sh.icub[kb];
                const float4 o0 = cb[0], o1 = cb[1], o2 = cb[2], o3 = cb[3];
                float dax = 0.f, day = 0.f, daz = 0.f, dayaw = 0.f, dbx = 0.f, dby = 0.f, dbz = 0.f, dbyaw = 0.f;
                bool hit = false;
                float p0[kSlots], p1[kSlots], p2[kSlots], q0[kSlots], q1[kSlots], q2[kSlots], qm[kSlots];
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl)
                    qm[sl] = cub_local<float>(cx[sl], cy[sl], cz[sl], o0, o1, o2, o3, p0[sl], p1[sl], p2[sl], q0[sl],
                                              q1[sl], q2[sl]);
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl) {
                    if (act[sl]) {
                        const float g = fmaxf(qm[sl] - rr[sl], 0.f);
                        if (placed) {
                            if (kb == top) gap_t = fminf(gap_t, g);
                            else gap_m = fminf(gap_m, g);
                        }
                        else if (!fixed[sl]) gap_s = fminf(gap_s, g);
                    }
                    if (!act[sl] || !(qm[sl] < rr[sl])) continue;
                    float ax, ay, az;
                    const float pen = pen_finish<float>(p0[sl], p1[sl], p2[sl], q0[sl], q1[sl], q2[sl], qm[sl], rr[sl],
                                                        o1, o2, o3, ax, ay, az);
                    if (pen > 0.f) {
                        any_hit = true;
                        hit = true;
                        pen_sum[sl] += pen;
                        acc_max = fmaxf(acc_max, pen);
                        gx[sl] += ax; gy[sl] += ay; gz[sl] += az;
                        // rigid motion of the cuboid: d/dP = -g, d/dyaw = -((c - P) x g)_z
                        const float dyaw = -((cx[sl] - o0.x) * ay - (cy[sl] - o0.y) * ax);
                        if (isblk[sl]) { dbx -= ax; dby -= ay; dbz -= az; dbyaw += dyaw; }
                        else { dax -= ax; day -= ay; daz -= az; dayaw += dyaw; }
                    }
                }
                if (grad && placed && __any_sync(0xffffffffu, hit)) {
                    dax = warp_sum(dax); day = warp_sum(day); daz = warp_sum(daz); dayaw = warp_sum(dayaw);
                    dbx = warp_sum(dbx); dby = warp_sum(dby); dbz = warp_sum(dbz); dbyaw = warp_sum(dbyaw);
                    if (lane == 0) {
                        fx_add(&sh.fx_wr[0][kb][0], dax); fx_add(&sh.fx_wr[0][kb][1], day);
                        fx_add(&sh.fx_wr[0][kb][2], daz); fx_add(&sh.fx_wr[0][kb][3], dayaw);
                        fx_add(&sh.fx_wr[1][kb][0], dbx); fx_add(&sh.fx_wr[1][kb][1], dby);
                        fx_add(&sh.fx_wr[1][kb][2], dbz); fx_add(&sh.fx_wr[1][kb][3], dbyaw);
                    }
                }
            }
        }
        n_tests += (unsigned long long)visits * (unsigned)n_items;
        chunk_hit |= any_hit;
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
            if (isblk[sl]) acc_blk += pen_sum[sl];
            else acc_arm += pen_sum[sl];
        }
        if (!grad) continue;

        // backward: dC/dq_k = sum_s z_k . ((c_s - o_k) x g_s) over spheres on links >= k
        // v[k] = arm-group torque of joint k, v[8 + k] = block-group torque (v[7], v[15] unused)
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
        const bool warp_hit = __any_sync(0xffffffffu, any_hit);
        if (warp_hit) {
            const float4(*F)[3] = tw.F[ci];
            if (any_hit) {
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    const float4 f0 = F[k + 1][0], f1 = F[k + 1][1], f2 = F[k + 1][2];
                    const float ox = f0.w, oy = f1.w, oz = f2.w;
                    const float zx = f0.z, zy = f1.z, zz = f2.z;
#pragma unroll
                    for (int sl = 0; sl < kSlots; ++sl) {
                        const int lk = isblk[sl] ? 7 : ls.link[sl];
                        if (!act[sl] || lk < k + 1) continue;
                        const float vx = cx[sl] - ox, vy = cy[sl] - oy, vz = cz[sl] - oz;
                        const float mm = zx * (vy * gz[sl] - vz * gy[sl]) + zy * (vz * gx[sl] - vx * gz[sl]) +
                                         zz * (vx * gy[sl] - vy * gx[sl]);
                        if (isblk[sl]) v[8 + k] += mm; else v[k] += mm;
                    }
                }
            }
            // warp reduce-scatter by recursive halving: at the step of lane bit `off` a lane keeps
            // the half of its values selected by that bit and adds the partner's copy of it; after
            // bits 16, 8, 4, 2 lane L holds value 8 b4 + 4 b3 + 2 b2 + b1 summed over 16 lanes, and
            // the last exchange (bit 1) completes the sum over the warp
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const bool up = lane & 16;
                const float send = up ? v[i] : v[i + 8], keep = up ? v[i + 8] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool up = lane & 8;
                const float send = up ? v[i] : v[i + 4], keep = up ? v[i + 4] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const bool up = lane & 4;
                const float send = up ? v[i] : v[i + 2], keep = up ? v[i + 2] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            {
                const bool up = lane & 2;
                const float send = up ? v[0] : v[1], keep = up ? v[1] : v[0];
                v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
            }
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
        }
        {
            const int j = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
            if ((lane & 1) == 0 && (j & 7) != 7) (j < 8 ? G_arm : G_blk)[t * 8 + (j & 7)] = v[0];
        }
    }
    if (none) return true;
    // candidates, but no sphere penetrates any of them: the chunk's terms are zero, and the
    // tests' gaps join the clearances
    if (__any_sync(0xffffffffu, chunk_hit)) return false;
    clearance = fminf(clearance, warp_min(gap_s));
    clearance_moving = fminf(clearance_moving, warp_min(gap_m));
    clearance_top = fminf(clearance_top, warp_min(gap_t));
    return true;
}

// Residuals of the start group at the grasp (which = 0) or place (which = 1) configuration
// of block b from that configuration's frames (s_r == nullptr; the roll and pitch torques go
// to rpt), or, with s_r, their weighted joint gradient sum_r s_r dh_r/dq (plus the placed-pose
// gradient g4 at a place config) from the torques the residual pass left in rpt.
__device__ __forceinline__ void start_terms(const Scalars& sc, int b, int which, const SpecialFrames& sf, float* h_out,
                                            const float* s_r, float grad_out[7], const float* g4 /*4 or null*/,
                                            float rpt[6]) {
    float Rb[9], pb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        Rb[3 * r] = sf.H[r].x; Rb[3 * r + 1] = sf.H[r].y; Rb[3 * r + 2] = sf.H[r].z; pb[r] = sf.H[r].w;
    }
    if (!s_r) {
        float roll, pitch;
        roll_pitch_torque<float>(Rb, roll, pitch, rpt, rpt + 3);
        if (which == 0) {
            h_out[0] = pb[0] - sc.init[b].x;
            h_out[1] = pb[1] - sc.init[b].y;
            h_out[2] = pb[2] - sc.init[b].z;
            h_out[3] = roll;
            h_out[4] = pitch;
        } else {
            h_out[0] = roll;
            h_out[1] = pitch;
        }
        return;
    }
    const float wr[3] = {rpt[0], rpt[1], rpt[2]}, wp[3] = {rpt[3], rpt[4], rpt[5]};
    // wrench at the block frame: force F (on p_blk), torque M (about the world origin)
    float F[3] = {0, 0, 0}, M[3] = {0, 0, 0};
    if (which == 0) {
        F[0] = s_r[0]; F[1] = s_r[1]; F[2] = s_r[2];
        for (int i = 0; i < 3; ++i) M[i] = s_r[3] * wr[i] + s_r[4] * wp[i];
    } else {
        for (int i = 0; i < 3; ++i) M[i] = s_r[0] * wr[i] + s_r[1] * wp[i];
    }
    if (g4) {
        // placed-pose gradient (x, y, z, yaw) of the same configuration
        const float e[3] = {Rb[0], Rb[3], Rb[6]};
        float wy[3];
        yaw_torque(e, wy);
        F[0] += g4[0]; F[1] += g4[1]; F[2] += g4[2];
        for (int i = 0; i < 3; ++i) M[i] += g4[3] * wy[i];
    }
    // moment of F about the origin: p x F
    M[0] += pb[1] * F[2] - pb[2] * F[1];
    M[1] += pb[2] * F[0] - pb[0] * F[2];
    M[2] += pb[0] * F[1] - pb[1] * F[0];
    for (int k = 0; k < 7; ++k) {
        const float4 f0 = sf.F[k + 1][0], f1 = sf.F[k + 1][1], f2 = sf.F[k + 1][2];
        const float ok[3] = {f0.w, f1.w, f2.w};
        // z . (M - o x F)
        const float tx = M[0] - (ok[1] * F[2] - ok[2] * F[1]);
        const float ty = M[1] - (ok[2] * F[0] - ok[0] * F[2]);
        const float tz = M[2] - (ok[0] * F[1] - ok[1] * F[0]);
        grad_out[k] = f0.z * tx + f1.z * ty + f2.z * tz;
    }
}

// Collisions of the placed tower (the C_coll residual of the placement terms), slice u of its
// block spheres (items 32u .. 32u+31, item 8j + m: sphere m of block j) by one warp.  An exact
// cull first keeps the environment obstacles whose boxes overlap the tower's box (every block
// sphere lies inside its block's cuboid box); a box test screens each pair before the exact
// one; each sphere of block j is also tested against the cuboids of the blocks i < j below it.
// Writes the slice's sum and maximum of the penetrations (sh.pcu[u]); with `grad`, the
// unscaled pose gradient dC_coll/dx, sphere side in sh.pg[j] for the slice's blocks and
// cuboid side in sh.pgc[u][i] for every i < B - 1.
__device__ __forceinline__ void placed_slice(const Scalars& sc, const float4* __restrict__ cub,
                                             const float4* __restrict__ osph, const float4* __restrict__ aabb,
                                             TShared& sh, bool grad, int u) {
    const int lane = threadIdx.x & 31;
    const int B = sc.B, n_items = 8 * B;
    const int it = 32 * u + lane;
    const bool valid = it < n_items;
    const int j = valid ? it >> 3 : 0, m = it & 7;
    const float4 h = sc.half[j];
    float lx, ly, lz;
    block_sphere_local(h, m, lx, ly, lz);
    const float c = sh.bcub[j][1].x, s = sh.bcub[j][1].y;
    const float cx = sh.pose[4 * j] + c * lx - s * ly;
    const float cy = sh.pose[4 * j + 1] + s * lx + c * ly;
    const float cz = sh.pose[4 * j + 2] + lz;
    const float r = h.w;
    auto apart = [&](const float4& lo, const float4& hi) {
        return lo.x > cx + r || hi.x < cx - r || lo.y > cy + r || hi.y < cy - r || lo.z > cz + r || hi.z < cz - r;
    };
    // the tower's box
    float tlx = lane < B ? sh.baabb[lane][0].x : 3.4e38f, tly = lane < B ? sh.baabb[lane][0].y : 3.4e38f;
    float tlz = lane < B ? sh.baabb[lane][0].z : 3.4e38f, thx = lane < B ? sh.baabb[lane][1].x : -3.4e38f;
    float thy = lane < B ? sh.baabb[lane][1].y : -3.4e38f, thz = lane < B ? sh.baabb[lane][1].z : -3.4e38f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        tlx = fminf(tlx, __shfl_xor_sync(0xffffffffu, tlx, off));
        tly = fminf(tly, __shfl_xor_sync(0xffffffffu, tly, off));
        tlz = fminf(tlz, __shfl_xor_sync(0xffffffffu, tlz, off));
        thx = fmaxf(thx, __shfl_xor_sync(0xffffffffu, thx, off));
        thy = fmaxf(thy, __shfl_xor_sync(0xffffffffu, thy, off));
        thz = fmaxf(thz, __shfl_xor_sync(0xffffffffu, thz, off));
    }
    float coll = 0.f, maxpen = 0.f;
    float ax = 0.f, ay = 0.f, az = 0.f;   // dC/dc of this item
    const int n_env = sc.n_cub + sc.n_osph;
    for (int wd = 0; 32 * wd < n_env; ++wd) {
        const int a_l = 32 * wd + lane;
        bool near = false;
        if (a_l < n_env) {
            const float4 lo = aabb[2 * a_l], hi = aabb[2 * a_l + 1];
            near = !(lo.x > thx || hi.x < tlx || lo.y > thy || hi.y < tly || lo.z > thz || hi.z < tlz);
        }
        unsigned mk = __ballot_sync(0xffffffffu, near);
        if (!valid) continue;
        while (mk) {
            const int a = 32 * wd + __ffs(mk) - 1;
            mk &= mk - 1;
            float gx, gy, gz, pen;
            if (a < sc.n_cub) {
                if (apart(aabb[2 * a], aabb[2 * a + 1])) continue;
                pen = pen_cuboid<float>(cx, cy, cz, r, cub[4 * a], cub[4 * a + 1], cub[4 * a + 2], cub[4 * a + 3], gx,
                                        gy, gz);
            } else {
                pen = pen_sphere<float>(cx, cy, cz, r, osph[a - sc.n_cub], gx, gy, gz);
            }
            if (pen > 0.f) {
                coll += pen; maxpen = fmaxf(maxpen, pen);
                ax += gx; ay += gy; az += gz;
            }
        }
    }
    // blocks below in the stack: sphere of j against the cuboid of i < j (the slice's highest
    // block bounds i)
    const int i_end = min(B - 1, (min(32 * u + 31, n_items - 1) >> 3));
    for (int i = 0; i < B - 1; ++i) {
        float bx = 0.f, by = 0.f, bz = 0.f, byaw = 0.f;   // dC/d(pose i) from this item
        bool hit = false;
        if (i < i_end && valid && i < j && !apart(sh.baabb[i][0], sh.baabb[i][1])) {
            float gx, gy, gz;
            const float pen = pen_cuboid<float>(cx, cy, cz, r, sh.bcub[i][0], sh.bcub[i][1], sh.bcub[i][2],
                                                sh.bcub[i][3], gx, gy, gz);
            if (pen > 0.f) {
                hit = true;
                coll += pen; maxpen = fmaxf(maxpen, pen);
                ax += gx; ay += gy; az += gz;
                // the cuboid moves rigidly: d/dP_i = -g, d/dyaw_i = -((c - P_i) x g)_z
                bx = -gx; by = -gy; bz = -gz;
                byaw = -((cx - sh.pose[4 * i]) * gy - (cy - sh.pose[4 * i + 1]) * gx);
            }
        }
        if (!grad) continue;
        if (__any_sync(0xffffffffu, hit)) {
            bx = warp_sum(bx); by = warp_sum(by); bz = warp_sum(bz); byaw = warp_sum(byaw);
        }
        if (lane == 0) { sh.pgc[u][i][0] = bx; sh.pgc[u][i][1] = by; sh.pgc[u][i][2] = bz; sh.pgc[u][i][3] = byaw; }
    }
    if (grad) {
        float gyaw = ax * (-s * lx - c * ly) + ay * (c * lx - s * ly);   // dc/dyaw_j
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, off);
            ay += __shfl_xor_sync(0xffffffffu, ay, off);
            az += __shfl_xor_sync(0xffffffffu, az, off);
            gyaw += __shfl_xor_sync(0xffffffffu, gyaw, off);
        }
        // one writer per block j: the lane with m == 0
        if (valid && m == 0) { sh.pg[j][0] = ax; sh.pg[j][1] = ay; sh.pg[j][2] = az; sh.pg[j][3] = gyaw; }
    }
    coll = warp_sum(coll);
    maxpen = warp_max(maxpen);
    if (lane == 0) { sh.pcu[u][0] = coll; sh.pcu[u][1] = maxpen; }
}

// Modes of the trajectory kernel
enum TrajMode { kTrajEval = 0, kTrajDescend = 1, kTrajCheck = 2 };

// Axis-aligned box of a cuboid record (centre, then R columns with half extents).
__device__ __forceinline__ void cuboid_aabb(const float4* c, float4* box) {
    const float ex = fabsf(c[1].x) * c[1].w + fabsf(c[2].x) * c[2].w + fabsf(c[3].x) * c[3].w;
    const float ey = fabsf(c[1].y) * c[1].w + fabsf(c[2].y) * c[2].w + fabsf(c[3].y) * c[3].w;
    const float ez = fabsf(c[1].z) * c[1].w + fabsf(c[2].z) * c[2].w + fabsf(c[3].z) * c[3].w;
    box[0] = make_float4(c[0].x - ex, c[0].y - ey, c[0].z - ez, 0.f);
    box[1] = make_float4(c[0].x + ex, c[0].y + ey, c[0].z + ez, 0.f);
}

// Evaluate the whole particle: kinematics of the grasp/place configurations and the placed
// poses, the configuration loop, residuals and objective; with `grad`, the assembled dL/dq
// ends up in G_blk (G_arm holds the unscaled arm-group gradient).
template <bool kP2P, int kTile, int kPpc>
__device__ void traj_evaluate(const Scalars& sc, const LaneSpheres& ls, const float4* cub, const float4* osph,
                              const float4* aabb, TShared& sh, SpecialFrames* sp, float* q, float* G_arm,
                              float* G_blk, float* disp, float* cblk, __half2* cgap, int* ccand, float* ctopm,
                              __half* ctop, bool grad,
                              unsigned long long& n_tests, unsigned long long& n_cull,
                              unsigned long long& n_cand) {
    const int tid = grp_tid<kPpc>(), lane = tid & 31, w = tid >> 5;
    const int B = sc.B, S = sc.S, C = sc.C, NR = sc.NR;
    // point to point (kP2P): one segment ending at the target's grasp configuration; no placement
    constexpr bool p2p = kP2P;

    // (1) frames of the 2B grasp/place configurations (4 per warp), kept for the epilogue
    const int n_sp = p2p ? 1 : 2 * B;
    for (int gi = w; gi * 4 < n_sp; gi += kTWarps) {
        const int si = 4 * gi + (lane >> 3);
        const bool ok = si < n_sp;
        chunk_fk(sc, sh, q, ok ? (si + 1) * S : 1, ok, true, sp[ok ? si : 0].F, sp[ok ? si : 0].H, nullptr);
    }
    for (int i = tid; i < 2 * kMaxB * 4; i += kTThreads) (&sh.fx_wr[0][0][0])[i] = 0;
    if (tid == 0) { sh.fx_arm = 0; sh.fx_blk = 0; sh.next = 0; }
    grp_sync<kPpc>();
    // placed poses: the block frame at each place configuration, (x, y, z, yaw)
    if (w == 0) {
        float moved = 0.f;
        if (lane < B && !p2p) {
            const float4* H = sp[2 * lane + 1].H;
            const float pose[4] = {H[0].w, H[1].w, H[2].w, atan2f(H[1].x, H[0].x)};
            // how far any point of the placed cuboid moved since the previous evaluation:
            // |d position| + |d yaw| times its horizontal half diagonal
            if (sh.pose_prev_ok) {
                const float* pp = &sh.pose_prev[4 * lane];
                const float dx = pose[0] - pp[0], dy = pose[1] - pp[1], dz = pose[2] - pp[2];
                float dyaw = fabsf(pose[3] - pp[3]);
                dyaw = fminf(dyaw, 2.f * kPi - dyaw);
                const float4 h = sc.half[lane];
                moved = (sqrtf(dx * dx + dy * dy + dz * dz) + dyaw * sqrtf(h.x * h.x + h.y * h.y)) * 1.0001f + 1e-6f;
            }
            for (int i = 0; i < 4; ++i) sh.pose[4 * lane + i] = sh.pose_prev[4 * lane + i] = pose[i];
            block_cuboid(pose[0], pose[1], pose[2], pose[3], sc.half[lane], sh.bcub[lane]);
            cuboid_aabb(sh.bcub[lane], sh.baabb[lane]);
        } else if (lane < B) {
            for (int i = 0; i < 4; ++i) sh.pose[4 * lane + i] = 0.f;
            sh.baabb[lane][0] = make_float4(3.4e38f, 3.4e38f, 3.4e38f, 0.f);   // an empty box: never a candidate
            sh.baabb[lane][1] = make_float4(-3.4e38f, -3.4e38f, -3.4e38f, 0.f);
        }
        if (lane < B) sh.bown[lane] += moved;   // the block's own motion, before the scan
        // inclusive max-scan over the blocks: blk_cum[k] accumulates, evaluation by evaluation, the
        // largest motion among blocks 0..k.  Summed over the evaluations since a chunk's cull it
        // bounds the motion of each of those blocks since then, which is all that a gap to any
        // one of them needs (a sum over the blocks would bound their total motion instead)
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float up = __shfl_up_sync(0xffffffffu, moved, off);
            if (lane >= off) moved = fmaxf(moved, up);
        }
        if (lane < B) sh.blk_cum[lane] += moved;
        if (lane == 0) sh.pose_prev_ok = 1;
    }
    grp_sync<kPpc>();

    // (2) the evaluation's work queue: chunks of kChunk consecutive configurations, the slices of
    // the placed tower's collisions and the residual jobs
    float acc_max = 0.f;
    const int n_chunks = (C - 1 + kChunk - 1) / kChunk;
    // Chunks to evaluate: those without a valid cached cull (terms zero at its last cull, and
    // the motion since below its clearances).  Warp g lists those of chunks 32g .. 32g+31 in
    // chunk order, by tier: the chunks with 4, 3, 2, 1 configurations with candidates at the
    // last cull (tests and the gradient chain), then the chunks to cull again; it marks the
    // skipped ones in sh.skip, whose block-group gradient rows the assembly reads as zero
    // (their arm-group rows are still zero from their last cull).
    static_assert((kMaxC + kChunk - 1) / kChunk <= 256, "chunk indices fit the byte lists");
    static_assert((kMaxC + kChunk - 1) / kChunk <= 32 * kTWarps && (kTWarps & (kTWarps - 1)) == 0,
                  "one 32-chunk group per warp");
    static_assert(kChunk * kTWarps == 32, "a lane per (tier, group) of the candidate tiers");
    // bound on the motion of each block placed before block b (the only placed blocks the
    // configurations of a chunk whose last configuration belongs to block b's segments can
    // touch): its difference between two evaluations bounds any one block's motion between them
    auto blk_before = [&](int b) { return b > 0 ? sh.blk_cum[b - 1] : 0.f; };
    auto chunk_block = [&](int t0c) { return (min(t0c + kChunk - 1, C - 1) - 1) / S >> 1; };
    // own motion of block k (the top block of a chunk of block k + 1's segments), 0 for none
    auto own_motion = [&](int k) { return k >= 0 ? sh.bown[k] : 0.f; };
    {
        const int chk = 32 * w + lane;
        const int t0 = 1 + kChunk * chk, nc = min(kChunk, C - t0);
        bool active = chk < n_chunks;
        if (active && ccand[chk] == 0) {
            float d = 0.f;
            for (int i = 0; i < nc; ++i) d = fmaxf(d, disp[t0 + i]);
            const __half2 cg = cgap[chk];
            const int top = chunk_block(t0) - 1;
            active = !(d < __low2float(cg) && d + (blk_before(top) - cblk[chk]) < __high2float(cg) &&
                       d + (own_motion(top) - ctopm[chk]) < __half2float(ctop[chk]));
        }
        // tier: kChunk - (configurations with candidates), kChunk for a chunk to cull again
        const int tier = active ? (ccand[chk] == 0 ? kChunk : kChunk - ccand[chk]) : -1;
#pragma unroll
        for (int tr = 0; tr <= kChunk; ++tr) {
            const unsigned bal = __ballot_sync(0xffffffffu, tier == tr);
            if (tier == tr) sh.active[tr][32 * w + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)chk;
            if (lane == 0) sh.n_group[tr][w] = (short)__popc(bal);
        }
        // skipped chunks: their block-group rows count as zero in the assembly (step 5)
        const unsigned skipped = __ballot_sync(0xffffffffu, chk < n_chunks && !active);
        if (lane == 0) sh.skip[w] = skipped;
    }
    grp_sync<kPpc>();
    // The queue, in order: the chunks of the candidate tiers (tier by tier, group by group), the
    // chunks to cull again, the residual jobs (they need only the placed poses and the special
    // frames), the slices of the placed tower: the smaller items come last, so that the warps
    // finish together.  Lane l holds the list of (tier l / 8, group l % 8): its count and first
    // position in the candidate part of the queue; lane l < 8 also that of (kChunk, group l).
    const int n_cnt = sh.n_group[lane >> 3][lane & (kTWarps - 1)];
    int c_end = n_cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int up = __shfl_up_sync(0xffffffffu, c_end, off);
        if (lane >= off) c_end += up;
    }
    const int c_first = c_end - n_cnt, n_heavy = __shfl_sync(0xffffffffu, c_end, 31);
    const int n_rc = lane < kTWarps ? sh.n_group[kChunk][lane] : 0;
    int r_end = n_rc;
#pragma unroll
    for (int off = 1; off < kTWarps; off <<= 1) {
        const int up = __shfl_up_sync(0xffffffffu, r_end, off);
        if (lane >= off) r_end += up;
    }
    const int r_first = r_end - n_rc, n_light = __shfl_sync(0xffffffffu, r_end, kTWarps - 1);
    const int n_pu = p2p ? 0 : (8 * B + 31) / 32;
    const int n_chunk_items = n_heavy + n_light, total = n_chunk_items + kResidualJobs + n_pu;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(&sh.next, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        if (idx >= n_chunk_items + kResidualJobs) {
            placed_slice(sc, cub, osph, aabb, sh, grad, idx - n_chunk_items - kResidualJobs);
            continue;
        }
        if (idx == n_chunk_items) {
            // placement residuals (tower terms) with their unit-coefficient support factors
            float my_D = 0.f, my_e = 0.f;
            if (!p2p) place_stack_warp(sc, sh.pose, kPlaceUnit, nullptr, nullptr, nullptr, sh.ps, my_D, my_e);
            const float c_stable = warp_sum(lane < B ? my_D : 0.f);
            const float c_height = warp_sum(lane < B ? my_e * my_e : 0.f);
            const float max_D = warp_max(lane < B ? my_D : 0.f);
            const float max_dz = warp_max(lane < B ? fabsf(my_e) : 0.f);
            if (lane < B) {
                sh.h[7 * B + lane] = my_e;
                sh.h[8 * B + lane] = my_D;
            }
            if (lane == 0) { sh.c_stable = c_stable; sh.c_height = c_height; sh.pm_D = max_D; sh.pm_dz = max_dz; }
            continue;
        }
        if (idx == n_chunk_items + 1) {
            // start residuals: grasp configurations on lanes 0..15, place configurations on 16..31
            const int which = lane >> 4, b = lane & 15;
            if (b < B) {
                if (which == 0)
                    start_terms(sc, b, 0, sp[2 * b], &sh.h[5 * b], nullptr, nullptr, nullptr, sh.extra[b]);
                else if (!p2p)
                    start_terms(sc, b, 1, sp[2 * b + 1], &sh.h[5 * B + 2 * b], nullptr, nullptr, nullptr,
                                sh.extra[B + b]);
                else
                    sh.h[5 * B + 2 * b] = sh.h[5 * B + 2 * b + 1] = 0.f;
            }
            continue;
        }
        int chk;
        if (idx < n_heavy) {
            const int src = __ffs(__ballot_sync(0xffffffffu, c_first <= idx && idx < c_end)) - 1;
            chk = sh.active[src >> 3][32 * (src & (kTWarps - 1)) + idx - __shfl_sync(0xffffffffu, c_first, src)];
        } else {
            idx -= n_heavy;
            const int src = __ffs(__ballot_sync(0xffffffffu, r_first <= idx && idx < r_end)) - 1;
            chk = sh.active[kChunk][32 * src + idx - __shfl_sync(0xffffffffu, r_first, src)];
        }
        {
            const int t0 = 1 + kChunk * chk;
            const int nc = min(kChunk, C - t0);
            const int c = lane >> 3;
            // the held block's frame matters on transfer-segment interiors only
            const int tc = min(t0 + c, C - 1), seg_c = (tc - 1) / S;
            const bool held_c = (seg_c & 1) && tc - seg_c * S < S;
            float box[6];
            chunk_fk(sc, sh, q, t0 + c, true, held_c, sh.warp[w].F[c], sh.warp[w].H[c], box);
            __syncwarp();
            float clearance, clearance_moving, clearance_top, c_arm = 0.f, c_blk = 0.f;
            const unsigned long long cand0 = n_cand;
            const bool zero = chunk_collisions<kTile>(sc, ls, cub, osph, aabb, sh, sh.warp[w], G_arm, G_blk, t0, nc,
                                                      grad, box, c_arm, c_blk, acc_max, n_tests, n_cand, clearance,
                                                      clearance_moving, clearance_top);
            n_cull += (unsigned)nc;
            if (!zero) {
                c_arm = warp_sum(c_arm);
                c_blk = warp_sum(c_blk);
            }
            if (lane == 0) {
                if (!zero) { fx_add(&sh.fx_arm, c_arm); fx_add(&sh.fx_blk, c_blk); }
                ccand[chk] = zero ? 0 : (int)(n_cand - cand0);   // 0: a chunk whose terms are zero (cacheable)
                const int top = chunk_block(t0) - 1;
                cblk[chk] = blk_before(top);
                ctopm[chk] = own_motion(top);
                // fp16, rounded down: still lower bounds on the clearances
                cgap[chk] = __halves2half2(__float2half_rd(clearance - kClearSlack),
                                           __float2half_rd(clearance_moving - kClearSlack));
                ctop[chk] = __float2half_rd(clearance_top - kClearSlack);
            }
            if (lane < nc) disp[t0 + lane] = 0.f;
            __syncwarp();
        }
    }
    acc_max = warp_max(acc_max);
    if (lane == 0) sh.warp[w].part[2] = acc_max;
    grp_sync<kPpc>();

    // (3) warp 0: the group sums, then the objective and dL/dh
    if (w == 0) {
        const float tot_a = fx_value(sh.fx_arm), tot_b = fx_value(sh.fx_blk);
        const float cm = warp_max(lane < kTWarps ? sh.warp[lane].part[2] : 0.f);
        const float pm = warp_max(lane < n_pu ? sh.pcu[lane][1] : 0.f);
        float c_coll = 0.f;   // fixed-order sum over the slices
        for (int u = 0; u < n_pu; ++u) c_coll += sh.pcu[u][0];
        if (lane == 0) {
            sh.h[9 * B] = c_coll;
            sh.h[9 * B + 1] = tot_a;
            sh.h[9 * B + 2] = tot_b;
            sh.c_arm = tot_a; sh.c_blk = tot_b; sh.maxpen = cm;
            sh.c_coll = c_coll; sh.pm_pen = pm;
        }
        __syncwarp();   // the group residuals before every lane reads sh.h[]
        float v_start = 0.f, v_tilt = 0.f;
        if (lane < B) {
            const float* hg = &sh.h[5 * lane];
            const float* hp = &sh.h[5 * B + 2 * lane];
            v_start = hg[0] * hg[0] + hg[1] * hg[1] + hg[2] * hg[2] + hg[3] * hg[3] + hg[4] * hg[4];
            v_tilt = hp[0] * hp[0] + hp[1] * hp[1];
        }
        const float c_start = warp_sum(v_start + v_tilt);
        const float m_start = warp_max(v_start), m_tilt = warp_max(v_tilt);
        float Lp = 0.f;
        for (int r = lane; r < NR; r += 32) {
            const float sw = residual_sqrt_weight(sc, r), hw = sw * sh.h[r];
            Lp += sh.lam[r] * hw + 0.5f * sh.mu * hw * hw;
            sh.s[r] = (sh.lam[r] + sh.mu * hw) * sw;
        }
        Lp = warp_sum(Lp);
        __syncwarp();   // sh.s[] was written by other lanes: order those stores before lane 0 reads them
        if (lane == 0) {
            sh.L = Lp; sh.c_start = c_start; sh.max_start = m_start; sh.max_tilt = m_tilt;
            sh.s_arm = sh.s[9 * B + 1]; sh.s_blk = sh.s[9 * B + 2];
        }
    }
    grp_sync<kPpc>();
    if (grad) {
        // (4) warp 0: placement gradient w.r.t. the placed poses, then the place configurations'
        // gradient rows; warp 1: grasp gradients
        if (w == 0 && !p2p) {
            place_stack_grad(sc, sh.ps, &sh.s[8 * B], &sh.s[7 * B], sh.g4);
            const float s_arm = sh.s_arm, s_blk = sh.s_blk, s_coll = sh.s[9 * B];
            const int n_pu = (8 * B + 31) / 32;
            for (int i = lane; i < 4 * B; i += 32) {
                const int kb = i >> 2, c = i & 3;
                const float wa = fx_value(sh.fx_wr[0][kb][c]), wb = fx_value(sh.fx_wr[1][kb][c]);
                float gc = sh.pg[kb][c];
                if (kb + 1 < B)
                    for (int u = 0; u < n_pu; ++u) gc += sh.pgc[u][kb][c];
                sh.g4[i] += s_coll * gc + s_arm * wa + s_blk * wb;
            }
            __syncwarp();
            // place configurations: tilt residuals and the placed-pose gradient through fk
            if (lane < B) {
                start_terms(sc, lane, 1, sp[2 * lane + 1], nullptr, &sh.s[5 * B + 2 * lane], sh.extra[B + lane],
                            &sh.g4[4 * lane], sh.extra[B + lane]);
            }
        } else if (w == 1 && lane < B) {
            start_terms(sc, lane, 0, sp[2 * lane], nullptr, &sh.s[5 * lane], sh.extra[lane], nullptr, sh.extra[lane]);
        }
        grp_sync<kPpc>();
    }

    // (5) path length, joint limits; assemble the gradient into G_blk: a configuration per
    // thread (its own, previous and next rows as float4 pairs)
    float path = 0.f, jl = 0.f;
    for (int t = tid; t < C; t += kTThreads) {
        const float4* qv = reinterpret_cast<const float4*>(q + t * 8);
        const float4 a0 = qv[0], a1 = qv[1];
        const float v[7] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z};
        float nx[7] = {0, 0, 0, 0, 0, 0, 0}, pv[7] = {0, 0, 0, 0, 0, 0, 0};
        if (t + 1 < C) {
            const float4 b0 = qv[2], b1 = qv[3];
            nx[0] = b0.x; nx[1] = b0.y; nx[2] = b0.z; nx[3] = b0.w; nx[4] = b1.x; nx[5] = b1.y; nx[6] = b1.z;
        }
        if (t > 0) {
            const float4 c0 = qv[-2], c1 = qv[-1];
            pv[0] = c0.x; pv[1] = c0.y; pv[2] = c0.z; pv[3] = c0.w; pv[4] = c1.x; pv[5] = c1.y; pv[6] = c1.z;
        }
        float g[8];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            float gsum = 0.f;
            if (t + 1 < C) {
                const float d = nx[j] - v[j];
                path += d * d;
                gsum -= 2.f * sc.w_path * d;
            }
            if (t > 0) {
                const float d = v[j] - pv[j];
                gsum += 2.f * sc.w_path * d;
                const float over = fmaxf(v[j] - sc.qhi[j], 0.f), under = fmaxf(sc.qlo[j] - v[j], 0.f);
                jl += over * over + under * under;
                gsum += sc.w_jl * (2.f * over - 2.f * under);
            }
            g[j] = gsum;
        }
        if (grad) {
            float4* gv = reinterpret_cast<float4*>(G_blk + t * 8);
            if (t == 0) {
                gv[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                gv[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const float4* av = reinterpret_cast<const float4*>(G_arm + t * 8);
                const int chk = (t - 1) / kChunk;
                const bool kept = (sh.skip[chk >> 5] >> (chk & 31)) & 1u;   // cached cull: no block-group rows
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 p0 = av[0], p1 = av[1], r0 = kept ? z : gv[0], r1 = kept ? z : gv[1];
                const float ga[7] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z};
                const float gb[7] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
                const float* ex = nullptr;
                if (t % S == 0) {
                    const int e = t / S - 1;   // t = (e+1) S: grasp of block e/2 (e even) or place (e odd)
                    ex = (e & 1) ? sh.extra[B + (e >> 1)] : sh.extra[e >> 1];
                }
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    g[j] += sh.s_arm * ga[j] + sh.s_blk * gb[j];
                    if (ex) g[j] += ex[j];
                }
                gv[0] = make_float4(g[0], g[1], g[2], g[3]);   // G_blk becomes the assembled gradient
                gv[1] = make_float4(g[4], g[5], g[6], 0.f);
            }
        }
    }
    path = warp_sum(path);
    jl = warp_sum(jl);
    if (lane == 0) { sh.warp[w].part[0] = path; sh.warp[w].part[1] = jl; }
    grp_sync<kPpc>();
    if (tid == 0) {
        float p = 0.f, l = 0.f;
        for (int i = 0; i < kTWarps; ++i) { p += sh.warp[i].part[0]; l += sh.warp[i].part[1]; }
        sh.path = p;
        sh.jl = l;
        sh.L += sc.w_path * p + sc.w_jl * l;
    }
    // no barrier: the assembled gradient was complete at the one above, and only thread 0
    // reads sh.path, sh.jl and sh.L before the next one
}

// One particle of the trajectory stage by the whole CTA: load its state, run the descent (or
// the single evaluation), write the outputs.  The environment tables are already in shared
// memory (smem_raw, laid out by the t_*_offset functions of this problem).
template <bool kP2P, int kTile, int kPpc>
__device__ __forceinline__ void traj_particle(const Scalars& sc, int p, int mode, const TrajIO& io,
                                              unsigned char* smem_raw) {
    float4* cub = reinterpret_cast<float4*>(smem_raw + t_env_offset());
    float4* osph = cub + 4 * sc.n_cub;
    float4* aabb = reinterpret_cast<float4*>(smem_raw + t_aabb_offset(sc.n_cub, sc.n_osph));
    TShared& sh = *reinterpret_cast<TShared*>(smem_raw + t_shared_offset(sc.n_cub, sc.n_osph));
    float* q = reinterpret_cast<float*>(smem_raw + t_q_offset(sc.n_cub, sc.n_osph));
    float* G_arm = q + sc.C * 8;
    float* G_blk = G_arm + sc.C * 8;
    SpecialFrames* sp = reinterpret_cast<SpecialFrames*>(smem_raw + t_sp_offset(sc.n_cub, sc.n_osph, sc.C));
    float* disp = reinterpret_cast<float*>(smem_raw + t_cache_offset(sc.n_cub, sc.n_osph, sc.C, sc.B));
    const int n_chunks = t_n_chunks(sc.C);
    float* cblk = disp + sc.C;
    __half2* cgap = reinterpret_cast<__half2*>(cblk + n_chunks);   // (static, moving) clearances
    int* ccand = reinterpret_cast<int*>(cgap + n_chunks);
    float* ctopm = reinterpret_cast<float*>(ccand + n_chunks);   // the top block's own motion at the cull
    __half* ctop = reinterpret_cast<__half*>(ctopm + n_chunks);  // clearance to the top block
    const int tid = grp_tid<kPpc>();
    const int C = sc.C, NR = sc.NR, B = sc.B;
    for (int i = tid; i < C; i += kTThreads) disp[i] = 0.f;
    for (int i = tid; i < n_chunks; i += kTThreads) {
        cblk[i] = 0.f; cgap[i] = __float2half2_rn(0.f); ccand[i] = kChunk; ctopm[i] = 0.f; ctop[i] = __float2half_rn(0.f);
    }
    if (tid < kMaxB) { sh.blk_cum[tid] = 0.f; sh.bown[tid] = 0.f; }
    if (tid == 0) sh.pose_prev_ok = 0;

    // particle state -> shared memory (coalesced float4)
    const float4* qg = reinterpret_cast<const float4*>(io.q + (size_t)p * C * 8);
    float4* qs = reinterpret_cast<float4*>(q);
    for (int i = tid; i < C * 2; i += kTThreads) qs[i] = qg[i];
    if (tid < B) {
        block_cuboid(sc.init[tid].x, sc.init[tid].y, sc.init[tid].z, sc.init[tid].w, sc.half[tid], sh.icub[tid]);
        cuboid_aabb(sh.icub[tid], sh.iaabb[tid]);
    }
    if (tid < 8) {
        sh.dh[tid] = tid < 7 ? make_float4(sc.ca[tid], sc.sa[tid], sc.a[tid], sc.d[tid]) : make_float4(1.f, 0.f, 0.f, 0.f);
        sh.th0[tid] = tid < 7 ? sc.th0[tid] : 0.f;
        sh.lbc[tid] = sc.lbox_c[tid];
        sh.lbh[tid] = sc.lbox_h[tid];
    }
    for (int o = tid; o < sc.n_cub; o += kTThreads) cuboid_aabb(&cub[4 * o], &aabb[2 * o]);
    for (int o = tid; o < sc.n_osph; o += kTThreads) {
        const float4 sp = osph[o];
        aabb[2 * (sc.n_cub + o)] = make_float4(sp.x - sp.w, sp.y - sp.w, sp.z - sp.w, 0.f);
        aabb[2 * (sc.n_cub + o) + 1] = make_float4(sp.x + sp.w, sp.y + sp.w, sp.z + sp.w, 0.f);
    }
    unsigned long long n_tests = 0, n_cull = 0, n_cand = 0;
    const LaneSpheres ls = lane_spheres<kTile>(sc);
    const bool fresh = mode == kTrajDescend && io.init_multipliers;
    for (int r = tid; r < NR; r += kTThreads) {
        sh.lam[r] = (fresh || !io.lam) ? 0.f : io.lam[(size_t)p * NR + r];
    }
    if (tid == 0) sh.mu = (fresh || !io.mu) ? sc.mu0 : io.mu[p];
    grp_sync<kPpc>();

    // K descent iterations (evaluation with gradient, update), then the final evaluation: one
    // call site of traj_evaluate, so that its code is inlined once
    const bool want_grad = mode == kTrajEval && io.grad != nullptr;
    const int K = mode == kTrajDescend ? io.k_steps : 0;
    for (int k = 1;; ++k) {
        const bool last = k > K;
        traj_evaluate<kP2P, kTile, kPpc>(sc, ls, cub, osph, aabb, sh, sp, q, G_arm, G_blk, disp, cblk, cgap, ccand, ctopm, ctop,
                                         last ? want_grad : true, n_tests, n_cull, n_cand);
        if (last) break;
        const float eta = sc.eta_traj * (1.f - (float)k / (float)K);
        // q <- clamp(q - eta g) per configuration, and the bound on how far its spheres moved
        for (int t = 1 + tid; t < C; t += kTThreads) {
            float4* qv = reinterpret_cast<float4*>(q + t * 8);
            const float4* gv = reinterpret_cast<const float4*>(G_blk + t * 8);
            const float4 qa = qv[0], qb = qv[1], ga = gv[0], gb = gv[1];
            const float old[7] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z};
            const float g[7] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z};
            float nw[7], moved = 0.f;
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const float v = old[j] - eta * g[j];
                nw[j] = fminf(fmaxf(v, sc.qlo[j]), sc.qhi[j]);
                moved += fabsf(nw[j] - old[j]) * sc.sweep[j];
            }
            qv[0] = make_float4(nw[0], nw[1], nw[2], nw[3]);
            qv[1] = make_float4(nw[4], nw[5], nw[6], qb.w);
            disp[t] += moved * 1.0001f + 1e-7f;
        }
        if (sc.K_al > 0 && k % sc.K_al == 0) {
            for (int r = tid; r < NR; r += kTThreads) sh.lam[r] += sh.mu * residual_sqrt_weight(sc, r) * sh.h[r];
            grp_sync<kPpc>();
            if (tid == 0) sh.mu = fminf(sh.mu * 2.f, sc.mu_max);
        }
        grp_sync<kPpc>();
    }
    if (io.tests && (threadIdx.x & 31) == 0) {
        atomicAdd(io.tests, n_tests);
        atomicAdd(io.tests + 1, n_cull);
        atomicAdd(io.tests + 2, n_cand);
    }

    // outputs
    if (mode == kTrajDescend) {
        float4* qo = reinterpret_cast<float4*>(io.q + (size_t)p * C * 8);
        for (int i = tid; i < C * 2; i += kTThreads) qo[i] = qs[i];
        if (io.lam)
            for (int r = tid; r < NR; r += kTThreads) io.lam[(size_t)p * NR + r] = sh.lam[r];
        if (io.mu && tid == 0) io.mu[p] = sh.mu;
    }
    if (want_grad)
        for (int i = tid; i < C * 8; i += kTThreads) io.grad[(size_t)p * C * 8 + i] = (i & 7) == 7 ? 0.f : G_blk[i];
    if (io.h)
        for (int r = tid; r < NR; r += kTThreads) io.h[(size_t)p * NR + r] = sh.h[r];
    if (tid == 0) {
        if (io.L) io.L[p] = sh.L;
        if (io.groups) {
            float* g = io.groups + (size_t)p * 6;
            g[0] = sh.c_start; g[1] = sh.c_arm; g[2] = sh.c_blk; g[3] = sh.c_coll; g[4] = sh.c_stable; g[5] = sh.c_height;
        }
        const float rank = sc.w_path * sh.path + sc.w_stable * sh.c_stable + sc.w_height * sh.c_height +
                           sc.w_coll * sh.c_coll + sc.w_start * sh.c_start + sc.w_arm * sh.c_arm + sc.w_block * sh.c_blk;
        if (io.metrics) {
            float* m = io.metrics + (size_t)p * 8;
            m[0] = sh.maxpen; m[1] = sh.max_start; m[2] = sh.max_tilt; m[3] = sh.pm_pen; m[4] = sh.pm_D;
            m[5] = sh.pm_dz; m[6] = sh.path; m[7] = rank;
        }
        if (io.sat) {
            const bool ok = sh.maxpen <= sc.eps && sh.max_start <= sc.eps_start && sh.max_tilt <= sc.eps_start &&
                            sh.pm_pen <= sc.eps && sh.pm_D <= sc.eps && sh.pm_dz <= sc.eps && sh.jl == 0.f;
            io.sat[p] = ok ? 1 : 0;
        }
    }
}

// Bulk-copy staging of the environment tables into one group's region, with the group's own
// barrier: stage_tables for a group of kTThreads threads (the bounded wait, the error word, a
// second bounded wait for copies in flight after a timeout).  `init`: first use of the
// group's mbarrier; `phase`: the parity this copy completes.
template <int kPpc>
__device__ __forceinline__ bool stage_tables_grp(void* dst0, const void* src0, uint32_t bytes0, void* dst1,
                                                 const void* src1, uint32_t bytes1, uint64_t* bar, int* err,
                                                 bool init = true, uint32_t phase = 0) {
    volatile uint32_t* okw = reinterpret_cast<volatile uint32_t*>(bar + 1);   // the region header's second word
    if (grp_tid<kPpc>() == 0) {
        if (init) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        *okw = 1u;
    }
    grp_sync<kPpc>();
    if (grp_tid<kPpc>() == 0) {
        mbar_expect_tx(bar, bytes0 + bytes1);
        if (bytes0) bulk_g2s(dst0, src0, bytes0, bar);
        if (bytes1) bulk_g2s(dst1, src1, bytes1, bar);
    }
    const bool done = mbar_wait_bounded(bar, phase, kTablePolls);
    if (!done) {
        set_error(err, kDevTimeout);
        mbar_wait_bounded(bar, phase, kTablePolls);
        *okw = 0u;
    }
    grp_sync<kPpc>();
    const bool all = *okw != 0u;
    grp_sync<kPpc>();   // every thread has read the flag before a later call resets it
    return all;
}

// kPpc particles per CTA (one CTA per particle, or two): group g of CTA i takes particle
// kPpc i + g in its own shared-memory region of `region` bytes (kP2P: the point-to-point
// instantiation; kTile: the sphere tiling).
template <bool kP2P, int kTile, int kPpc>
__global__ void __launch_bounds__(kTThreads * kPpc, 3 - kPpc) k_traj(const __grid_constant__ Scalars sc, DevTables tab,
                                                                    int n, int mode, TrajIO io, int* err, int region) {
    extern __shared__ __align__(16) unsigned char smem_all[];
    if (io.active && *io.active <= 0) return;   // stage 1 of this problem found no placement
    unsigned char* smem_raw = smem_all + (size_t)grp_index<kPpc>() * region;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float4* cub = reinterpret_cast<float4*>(smem_raw + t_env_offset());
    float4* osph = cub + 4 * sc.n_cub;
    if (!stage_tables_grp<kPpc>(cub, tab.cub, (uint32_t)sc.n_cub * 64u, osph, tab.osph, (uint32_t)sc.n_osph * 16u, bar, err))
        return;
    const int p = blockIdx.x * kPpc + grp_index<kPpc>();
    if (p >= n) return;
    traj_particle<kP2P, kTile, kPpc>(sc, p, mode, io, smem_raw);
}

static_assert(sizeof(Scalars) % 16 == 0, "the batched kernel copies Scalars in 16-byte words");

// Batched form: a persistent grid over the particles of several problems.  Work items are
// runs of `per_fetch` consecutive particles of one problem, numbered problem after problem
// (jobs[j].first is the first item of problem j); each group (kPpc per CTA) takes the next
// item from *next until none is left.  On a change of problem the group stages that
// problem's constants and tables into its shared memory.  Every particle runs exactly the
// code of k_traj, so results equal the single-problem launches bit for bit, whatever the
// schedule.
template <int kTile, int kPpc>
__global__ void __launch_bounds__(kTThreads * kPpc, 3 - kPpc) k_traj_batch(const TrajJob* __restrict__ jobs, int n_jobs,
                                                                          int n_items, int per_fetch, int mode, int* next,
                                                                          int region) {
    extern __shared__ __align__(16) unsigned char smem_all[];
    __shared__ __align__(16) Scalars sc_arr[kPpc];
    __shared__ TrajIO io_arr[kPpc];
    __shared__ int s_item[kPpc], s_job[kPpc];
    const int g = grp_index<kPpc>(), tid = grp_tid<kPpc>();
    unsigned char* smem_raw = smem_all + (size_t)g * region;
    Scalars& sc_s = sc_arr[g];
    TrajIO& io_s = io_arr[g];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    int cur = -1;
    uint32_t uses = 0;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(next, 1);
            int j = -1;
            if (it < n_items) {   // last job whose first item is <= it
                int lo = 0, hi = n_jobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (jobs[mid].first <= it) lo = mid; else hi = mid - 1;
                }
                j = lo;
            }
            s_item[g] = it;
            s_job[g] = j;
        }
        grp_sync<kPpc>();
        const int it = s_item[g], j = s_job[g];
        if (j < 0) break;
        const TrajJob& job = jobs[j];
        if (j != cur) {
            // stage the problem's constants (int4 words) and its tables
            const int4* src = reinterpret_cast<const int4*>(job.sc);
            int4* dst = reinterpret_cast<int4*>(&sc_s);
            for (int i = tid; i < (int)(sizeof(Scalars) / 16); i += kTThreads) dst[i] = src[i];
            if (tid == 0) io_s = job.io;
            grp_sync<kPpc>();
            float4* cub = reinterpret_cast<float4*>(smem_raw + t_env_offset());
            float4* osph = cub + 4 * sc_s.n_cub;
            if (!stage_tables_grp<kPpc>(cub, job.tab.cub, (uint32_t)sc_s.n_cub * 64u, osph, job.tab.osph,
                                  (uint32_t)sc_s.n_osph * 16u, bar, job.err, uses == 0, uses & 1u))
                return;
            ++uses;
            cur = j;
        }
        const int p0 = (it - job.first) * per_fetch;
        // a problem whose stage 1 found no placement has nothing to optimise
        const int p1 = (io_s.active && *io_s.active <= 0) ? p0 : min(p0 + per_fetch, job.n);
        for (int p = p0; p < p1; ++p) {
            if (sc_s.kind == kKindP2P) traj_particle<true, kTile, kPpc>(sc_s, p, mode, io_s, smem_raw);
            else traj_particle<false, kTile, kPpc>(sc_s, p, mode, io_s, smem_raw);
            grp_sync<kPpc>();
        }
    }
}

// ================================================================================== launchers
// Shared memory of one group: the problem's layout, rounded to 128 bytes.
static int t_region(size_t bytes) { return (int)((bytes + 127) & ~(size_t)127); }

template <int kTile, int kPpc>
static cudaError_t batch_kernel(const TrajJob* jobs, int n_jobs, int n_items, int per_fetch, int mode, int* next,
                                size_t smem_bytes, int grid, cudaStream_t st) {
    const int region = t_region(smem_bytes);
    const size_t dyn = (size_t)region * kPpc;
    cudaError_t e = allow_max_dynamic_smem(k_traj_batch<kTile, kPpc>, dyn);
    if (e != cudaSuccess) return e;
    k_traj_batch<kTile, kPpc><<<grid, kTThreads * kPpc, dyn, st>>>(jobs, n_jobs, n_items, per_fetch, mode, next, region);
    return cudaGetLastError();
}

cudaError_t launch_traj_batch(const TrajJob* jobs, int n_jobs, int n_items, int per_fetch, int mode, int* next,
                              size_t smem_bytes, int grid, cudaStream_t st, int tiling, int ppc) {
    if (n_items <= 0) return cudaSuccess;
    if (ppc == 2)
        return tiling ? batch_kernel<1, 2>(jobs, n_jobs, n_items, per_fetch, mode, next, smem_bytes, grid, st)
                      : batch_kernel<0, 2>(jobs, n_jobs, n_items, per_fetch, mode, next, smem_bytes, grid, st);
    return tiling ? batch_kernel<1, 1>(jobs, n_jobs, n_items, per_fetch, mode, next, smem_bytes, grid, st)
                  : batch_kernel<0, 1>(jobs, n_jobs, n_items, per_fetch, mode, next, smem_bytes, grid, st);
}

template <int kTile, int kPpc>
static int batch_occupancy(size_t smem_bytes) {
    int n = 0;
    const size_t dyn = (size_t)t_region(smem_bytes) * kPpc;
    if (allow_max_dynamic_smem(k_traj_batch<kTile, kPpc>, dyn) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_traj_batch<kTile, kPpc>, kTThreads * kPpc, dyn) !=
        cudaSuccess)
        return 0;
    return n;
}

int traj_batch_ctas_per_sm(size_t smem_bytes, int tiling, int ppc) {
    if (ppc == 2) return tiling ? batch_occupancy<1, 2>(smem_bytes) : batch_occupancy<0, 2>(smem_bytes);
    return tiling ? batch_occupancy<1, 1>(smem_bytes) : batch_occupancy<0, 1>(smem_bytes);
}

template <bool kP2P, int kTile, int kPpc>
static int single_occupancy(size_t smem_bytes) {
    int n = 0;
    const size_t dyn = (size_t)t_region(smem_bytes) * kPpc;
    if (allow_max_dynamic_smem(k_traj<kP2P, kTile, kPpc>, dyn) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_traj<kP2P, kTile, kPpc>, kTThreads * kPpc, dyn) !=
        cudaSuccess)
        return 0;
    return n;
}

template <bool kP2P>
static int single_ctas(size_t smem, int tiling, int ppc) {
    if (ppc == 2) return tiling ? single_occupancy<kP2P, 1, 2>(smem) : single_occupancy<kP2P, 0, 2>(smem);
    return tiling ? single_occupancy<kP2P, 1, 1>(smem) : single_occupancy<kP2P, 0, 1>(smem);
}

int traj_ctas_per_sm(const Scalars& sc) {
    const size_t smem = traj_smem_bytes(sc);
    const int ppc = sc.particles_per_cta == 2 ? 2 : 1;
    return sc.kind == kKindP2P ? single_ctas<true>(smem, sc.sphere_tiling, ppc)
                               : single_ctas<false>(smem, sc.sphere_tiling, ppc);
}

template <bool kP2P, int kTile, int kPpc>
static cudaError_t traj_kernel(const Scalars& sc, DevTables t, int n, int mode, const TrajIO& io, int* err,
                               cudaStream_t st) {
    const int region = t_region(traj_smem_bytes(sc));
    const size_t dyn = (size_t)region * kPpc;
    cudaError_t e = allow_max_dynamic_smem(k_traj<kP2P, kTile, kPpc>, dyn);
    if (e != cudaSuccess) return e;
    k_traj<kP2P, kTile, kPpc><<<(n + kPpc - 1) / kPpc, kTThreads * kPpc, dyn, st>>>(sc, t, n, mode, io, err, region);
    return cudaGetLastError();
}

template <bool kP2P>
static cudaError_t traj_dispatch(const Scalars& sc, DevTables t, int n, int mode, const TrajIO& io, int* err,
                                 cudaStream_t st) {
    if (sc.particles_per_cta == 2)
        return sc.sphere_tiling ? traj_kernel<kP2P, 1, 2>(sc, t, n, mode, io, err, st)
                                : traj_kernel<kP2P, 0, 2>(sc, t, n, mode, io, err, st);
    return sc.sphere_tiling ? traj_kernel<kP2P, 1, 1>(sc, t, n, mode, io, err, st)
                            : traj_kernel<kP2P, 0, 1>(sc, t, n, mode, io, err, st);
}

cudaError_t launch_traj(const Scalars& sc, DevTables t, int n, int mode, const TrajIO& io, int* err,
                        cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    return sc.kind == kKindP2P ? traj_dispatch<true>(sc, t, n, mode, io, err, st)
                               : traj_dispatch<false>(sc, t, n, mode, io, err, st);
}

size_t traj_cta_smem_bytes(const Scalars& sc, int ppc) { return (size_t)t_region(traj_smem_bytes(sc)) * ppc; }

}  // namespace spasm
