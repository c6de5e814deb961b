// Stage 1 of SPaSM (Alg. 1): tower placement cost and gradient, one warp per particle.
//
// Per particle the warp holds the B x 4 pose vector in shared memory.  Lanes own
// (block j, sphere m) items of the block sphere sets and test them against the
// environment tables (staged once per CTA in shared memory, read as broadcasts) and the
// cuboids of the blocks below j.  Gradients are reduced deterministically: groups of 8
// lanes (the 8 spheres of one block) by xor-shuffles, block-pair terms by whole-warp
// reductions taken only when a lane of the warp penetrates.
#pragma once
#include "common.cuh"

namespace spasm {

struct PlaceOut {
    float c_stable, c_height, c_coll;    // sum D, sum e^2, sum pen (or pen^2)
    float maxpen, maxD, maxdz;           // satisfying metrics
};

// Per-warp shared scratch of the placement evaluation.
struct PlaceScratch {
    float4 bc[kMaxB][4];     // block cuboids
    float stab[kMaxB][4];    // a_i dD_i/dv (x, y), a_i dD_i/dyaw, D_i
    float e[kMaxB];          // height residuals
    float D[kMaxB];
};

// Coefficient modes of the gradient: stage-1 cost (a = w_stable, b = 2 w_height e,
// s_coll = w_coll), explicit per-residual coefficients (stage 2), or the residuals with the
// unit-coefficient support factors (a = 1) left in ps.stab and no gradient written (stage 2
// scales them by its multipliers once those are known).
enum PlaceMode { kPlaceForward = 0, kPlaceStage1 = 1, kPlaceExplicit = 2, kPlaceUnit = 3 };

// Per-block terms of the tower (lane i < B owns block i): height residual e_i, support
// distance D_i and the block cuboids in ps.  With mode kPlaceStage1 or kPlaceExplicit, sets
//   g = sum_i a_i dD_i/dx + sum_i b_i de_i/dx   (the collision part is added by the caller);
// with kPlaceUnit, leaves dD_i/d(centre of mass, yaw) in ps.stab for place_stack_grad and
// writes no block cuboids.
// x, g: per-warp shared arrays of 4B floats.  Must be called by all 32 lanes of the warp.
__device__ __forceinline__ void place_stack_warp(const Scalars& sc, const float* x, int mode, const float* a_in,
                                                 const float* b_in, float* g, PlaceScratch& ps, float& my_D,
                                                 float& my_e) {
    const int lane = threadIdx.x & 31;
    const int B = sc.B;
    const bool want_grad = mode != kPlaceForward;
    my_D = 0.f; my_e = 0.f;
    if (lane < B) {
        const int i = lane;
        my_e = x[4 * i + 2] - sc.zt[i];
        ps.e[i] = my_e;
        if (mode != kPlaceUnit)   // the stage-2 caller keeps its own placed cuboids
            block_cuboid(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3], sc.half[i], ps.bc[i]);
        float sx = 0.f, sy = 0.f, dvx = 0.f, dvy = 0.f, dyaw = 0.f;
        if (i + 1 < B) {
            const int n_above = B - 1 - i;
            for (int j = i + 1; j < B; ++j) { sx += x[4 * j]; sy += x[4 * j + 1]; }
            const float mx = sx / (float)n_above, my = sy / (float)n_above;
            float s, c;
            sincosf(x[4 * i + 3], &s, &c);
            const float vx = mx - x[4 * i], vy = my - x[4 * i + 1];
            const float ux = c * vx + s * vy, uy = -s * vx + c * vy;       // Rz(-yaw) v
            const float ex = fmaxf(fabsf(ux) - sc.half[i].x, 0.f), ey = fmaxf(fabsf(uy) - sc.half[i].y, 0.f);
            my_D = sqrtf(ex * ex + ey * ey);
            if (want_grad && my_D > 0.f) {
                const float a = mode == kPlaceStage1 ? sc.w_stable : mode == kPlaceUnit ? 1.f : a_in[i];
                const float du_x = (ux >= 0.f ? ex : -ex) / my_D, du_y = (uy >= 0.f ? ey : -ey) / my_D;
                dvx = a * (c * du_x - s * du_y);
                dvy = a * (s * du_x + c * du_y);
                dyaw = a * (du_x * uy - du_y * ux);
            }
        }
        ps.stab[i][0] = dvx; ps.stab[i][1] = dvy; ps.stab[i][2] = dyaw; ps.stab[i][3] = my_D;
        ps.D[i] = my_D;
    }
    __syncwarp();
    if (want_grad && mode != kPlaceUnit && lane < B) {
        const int i = lane;
        float gx = -ps.stab[i][0], gy = -ps.stab[i][1];
        for (int k = 0; k < i; ++k) {
            const float inv = 1.f / (float)(B - 1 - k);
            gx += ps.stab[k][0] * inv;
            gy += ps.stab[k][1] * inv;
        }
        const float b = mode == kPlaceStage1 ? 2.f * sc.w_height * my_e : b_in[i];
        g[4 * i] = gx; g[4 * i + 1] = gy; g[4 * i + 2] = b; g[4 * i + 3] = ps.stab[i][2];
    }
    __syncwarp();
}

// The gradient place_stack_warp writes in mode kPlaceExplicit, from the factors its kPlaceUnit
// pass left in ps (a_i dD_i/d... = a_i times the unit factor, in the same order of operations).
__device__ __forceinline__ void place_stack_grad(const Scalars& sc, const PlaceScratch& ps, const float* a_in,
                                                 const float* b_in, float* g) {
    const int lane = threadIdx.x & 31;
    const int B = sc.B;
    if (lane < B) {
        const int i = lane;
        float gx = -(a_in[i] * ps.stab[i][0]), gy = -(a_in[i] * ps.stab[i][1]);
        for (int k = 0; k < i; ++k) {
            const float inv = 1.f / (float)(B - 1 - k);
            gx += (a_in[k] * ps.stab[k][0]) * inv;
            gy += (a_in[k] * ps.stab[k][1]) * inv;
        }
        g[4 * i] = gx; g[4 * i + 1] = gy; g[4 * i + 2] = b_in[i]; g[4 * i + 3] = a_in[i] * ps.stab[i][2];
    }
    __syncwarp();
}

// x, g: per-warp shared arrays of 4B floats.  With mode != kPlaceForward, writes
//   g = sum_i a_i dD_i/dx + sum_i b_i de_i/dx + s_coll dC_coll/dx.
// Must be called by all 32 lanes of the warp.
// cand: per-warp scratch of kMaxCub/32 + kMaxOSph/32 words (the candidate obstacles of the particle).
__device__ __forceinline__ void place_eval_warp(const Scalars& sc, const float4* __restrict__ cub, int n_cub,
                                                const float4* __restrict__ osph, int n_osph, const float* x,
                                                bool quad, int mode, const float* a_in, const float* b_in,
                                                float s_coll_in, float* g, PlaceScratch& ps, uint32_t* cand,
                                                PlaceOut& out) {
    const int lane = threadIdx.x & 31;
    const int B = sc.B;
    const bool want_grad = mode != kPlaceForward;
    float my_D, my_e;
    place_stack_warp(sc, x, mode, a_in, b_in, g, ps, my_D, my_e);

    // -- collisions: items (block j, sphere m)
    const float s_coll = mode == kPlaceStage1 ? sc.w_coll : s_coll_in;
    float coll = 0.f, maxpen = 0.f;
    const int n_items = 8 * B;
    // exact cull: the box of every block sphere of the particle (padded by 1e-5 against the
    // rounding of the boxes) against each obstacle's box; only the obstacles that overlap it
    // can touch a sphere, and they are visited in the same order as without the cull
    const int n_cw = (n_cub + 31) >> 5, n_sw = (n_osph + 31) >> 5;
    {
        float lo_x = 3.4e38f, lo_y = 3.4e38f, lo_z = 3.4e38f, hi_x = -3.4e38f, hi_y = -3.4e38f, hi_z = -3.4e38f;
        for (int base = 0; base < n_items; base += 32) {
            const int it = base + lane;
            if (it < n_items) {
                const int j = it >> 3, m = it & 7;
                const float4 h = sc.half[j];
                float lx, ly, lz;
                block_sphere_local(h, m, lx, ly, lz);
                const float c = ps.bc[j][1].x, s = ps.bc[j][1].y;
                const float cx = x[4 * j] + c * lx - s * ly, cy = x[4 * j + 1] + s * lx + c * ly, cz = x[4 * j + 2] + lz;
                const float r = h.w + 1e-5f;
                lo_x = fminf(lo_x, cx - r); lo_y = fminf(lo_y, cy - r); lo_z = fminf(lo_z, cz - r);
                hi_x = fmaxf(hi_x, cx + r); hi_y = fmaxf(hi_y, cy + r); hi_z = fmaxf(hi_z, cz + r);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            lo_x = fminf(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, off));
            lo_y = fminf(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, off));
            lo_z = fminf(lo_z, __shfl_xor_sync(0xffffffffu, lo_z, off));
            hi_x = fmaxf(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, off));
            hi_y = fmaxf(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, off));
            hi_z = fmaxf(hi_z, __shfl_xor_sync(0xffffffffu, hi_z, off));
        }
        for (int wd = 0; wd < n_cw; ++wd) {
            const int o = 32 * wd + lane;
            bool near = false;
            if (o < n_cub) {
                const float4 c0 = cub[4 * o], c1 = cub[4 * o + 1], c2 = cub[4 * o + 2], c3 = cub[4 * o + 3];
                const float ex = fabsf(c1.x) * c1.w + fabsf(c2.x) * c2.w + fabsf(c3.x) * c3.w;
                const float ey = fabsf(c1.y) * c1.w + fabsf(c2.y) * c2.w + fabsf(c3.y) * c3.w;
                const float ez = fabsf(c1.z) * c1.w + fabsf(c2.z) * c2.w + fabsf(c3.z) * c3.w;
                near = c0.x - ex <= hi_x && c0.x + ex >= lo_x && c0.y - ey <= hi_y && c0.y + ey >= lo_y &&
                       c0.z - ez <= hi_z && c0.z + ez >= lo_z;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, near);
            if (lane == 0) cand[wd] = mk;
        }
        for (int wd = 0; wd < n_sw; ++wd) {
            const int o = 32 * wd + lane;
            bool near = false;
            if (o < n_osph) {
                const float4 sp = osph[o];
                near = sp.x - sp.w <= hi_x && sp.x + sp.w >= lo_x && sp.y - sp.w <= hi_y && sp.y + sp.w >= lo_y &&
                       sp.z - sp.w <= hi_z && sp.z + sp.w >= lo_z;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, near);
            if (lane == 0) cand[kMaxCub / 32 + wd] = mk;
        }
        __syncwarp();
    }
    for (int base = 0; base < n_items; base += 32) {
        const int it = base + lane;
        const bool valid = it < n_items;
        const int j = valid ? it >> 3 : 0, m = it & 7;
        float cx = 0.f, cy = 0.f, cz = 0.f, r = 0.f, dcx = 0.f, dcy = 0.f;
        float pj0 = 0.f, pj1 = 0.f;
        if (valid) {
            const float4 h = sc.half[j];
            float lx, ly, lz;
            block_sphere_local(h, m, lx, ly, lz);
            const float c = ps.bc[j][1].x, s = ps.bc[j][1].y;
            pj0 = x[4 * j]; pj1 = x[4 * j + 1];
            cx = pj0 + c * lx - s * ly;
            cy = pj1 + s * lx + c * ly;
            cz = x[4 * j + 2] + lz;
            dcx = -s * lx - c * ly;   // dc/dyaw_j
            dcy = c * lx - s * ly;
            r = h.w;
        }
        float ax = 0.f, ay = 0.f, az = 0.f;   // dC/dc of this item (scaled by 2 pen in quad form)
        if (valid) {
            for (int wd = 0; wd < n_cw; ++wd) {
                unsigned mk = cand[wd];
                while (mk) {
                    const int o = 32 * wd + __ffs(mk) - 1;
                    mk &= mk - 1;
                    float gx, gy, gz;
                    const float pen = pen_cuboid<float>(cx, cy, cz, r, cub[4 * o], cub[4 * o + 1], cub[4 * o + 2],
                                                        cub[4 * o + 3], gx, gy, gz);
                    if (pen > 0.f) {
                        maxpen = fmaxf(maxpen, pen);
                        coll += quad ? pen * pen : pen;
                        const float sgrad = quad ? 2.f * pen : 1.f;
                        ax += sgrad * gx; ay += sgrad * gy; az += sgrad * gz;
                    }
                }
            }
            for (int wd = 0; wd < n_sw; ++wd) {
                unsigned mk = cand[kMaxCub / 32 + wd];
                while (mk) {
                    const int o = 32 * wd + __ffs(mk) - 1;
                    mk &= mk - 1;
                    float gx, gy, gz;
                    const float pen = pen_sphere<float>(cx, cy, cz, r, osph[o], gx, gy, gz);
                    if (pen > 0.f) {
                        maxpen = fmaxf(maxpen, pen);
                        coll += quad ? pen * pen : pen;
                        const float sgrad = quad ? 2.f * pen : 1.f;
                        ax += sgrad * gx; ay += sgrad * gy; az += sgrad * gz;
                    }
                }
            }
        }
        // blocks below in the stack: sphere of j vs cuboid of i < j
        for (int i = 0; i + 1 < B; ++i) {
            float bx = 0.f, by = 0.f, bz = 0.f, byaw = 0.f;   // dC/d pose_i from this item
            bool hit = false;
            if (valid && i < j) {
                float gx, gy, gz;
                const float pen = pen_cuboid<float>(cx, cy, cz, r, ps.bc[i][0], ps.bc[i][1], ps.bc[i][2], ps.bc[i][3],
                                                    gx, gy, gz);
                if (pen > 0.f) {
                    hit = true;
                    maxpen = fmaxf(maxpen, pen);
                    coll += quad ? pen * pen : pen;
                    const float sgrad = quad ? 2.f * pen : 1.f;
                    gx *= sgrad; gy *= sgrad; gz *= sgrad;
                    ax += gx; ay += gy; az += gz;
                    // the cuboid moves rigidly: d/dP_i = -g, d/dyaw_i = -((c - P_i) x g)_z
                    bx = -gx; by = -gy; bz = -gz;
                    byaw = -((cx - x[4 * i]) * gy - (cy - x[4 * i + 1]) * gx);
                }
            }
            if (want_grad && __any_sync(0xffffffffu, hit)) {
                bx = warp_sum(bx); by = warp_sum(by); bz = warp_sum(bz); byaw = warp_sum(byaw);
                if (lane == 0) {
                    g[4 * i] += s_coll * bx; g[4 * i + 1] += s_coll * by;
                    g[4 * i + 2] += s_coll * bz; g[4 * i + 3] += s_coll * byaw;
                }
                __syncwarp();
            }
        }
        if (want_grad) {
            float gyaw = ax * dcx + ay * dcy;
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, off);
                ay += __shfl_xor_sync(0xffffffffu, ay, off);
                az += __shfl_xor_sync(0xffffffffu, az, off);
                gyaw += __shfl_xor_sync(0xffffffffu, gyaw, off);
            }
            // one writer per block j (lane with m == 0); groups of 8 lanes never share j
            if (valid && m == 0) {
                g[4 * j] += s_coll * ax; g[4 * j + 1] += s_coll * ay;
                g[4 * j + 2] += s_coll * az; g[4 * j + 3] += s_coll * gyaw;
            }
            __syncwarp();
        }
    }
    out.c_coll = warp_sum(coll);
    out.maxpen = warp_max(maxpen);
    out.c_stable = warp_sum(lane < B ? my_D : 0.f);
    out.c_height = warp_sum(lane < B ? my_e * my_e : 0.f);
    out.maxD = warp_max(lane < B ? my_D : 0.f);
    out.maxdz = warp_max(lane < B ? fabsf(my_e) : 0.f);
    __syncwarp();
}

__device__ __forceinline__ float place_cost_value(const Scalars& sc, const PlaceOut& o) {
    return sc.w_stable * o.c_stable + sc.w_height * o.c_height + sc.w_coll * o.c_coll;
}

// Projection onto the problem box (x, y in the goal box; z above the block's resting
// height; yaw wrapped to [-pi, pi)) of variable v = 4 i + k.
__device__ __forceinline__ float place_clamp(const Scalars& sc, int v, float val) {
    const int i = v >> 2, k = v & 3;
    if (k == 0) return fminf(fmaxf(val, sc.box_lo[0]), sc.box_hi[0]);
    if (k == 1) return fminf(fmaxf(val, sc.box_lo[1]), sc.box_hi[1]);
    if (k == 2) return fminf(fmaxf(val, sc.zlo[i]), sc.box_hi[2]);
    const float two_pi = 2.f * kPi;
    return val - two_pi * floorf((val + kPi) / two_pi);
}

}  // namespace spasm
