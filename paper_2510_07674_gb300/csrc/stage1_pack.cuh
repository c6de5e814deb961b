// Stage 1 (Alg. 1) for the packing goal: the placement cost of the appendix's Tetris
// problem, one warp per particle.
//
//   C = w_coll (sum_{i<j} P(i, j) + sum_i sum_{w in walls} P(i, w)) + w_height sum_i |z_i - z*|
//
// Block i is a polyomino of unit cubes; each cube (edge u) carries 8 spheres of radius u/4
// at (+-u/4, +-u/4, +-u/4) from its centre (objects as sphere sets, Sec. III).  P(i, j) sums
// the penetration of every sphere of block j into every cube of block i < j, P(i, w) every
// sphere of block i into wall w (the environment cuboids).  Penetrations turn quadratic in
// the refinement phase; |z - z*| keeps its form.
//
// Lanes own (cell, sphere) items: the 8 spheres of a cube are 8 consecutive lanes, so a
// cube's sphere-side gradient is reduced inside its lane group and stored once per
// evaluation (gcell); lanes < B then add their cubes in order, so sums are deterministic.
// The cube side of a block pair is reduced over the warp once per lower block.
#pragma once
#include "stage1.cuh"

namespace spasm {

__device__ __forceinline__ void place_eval_pack_warp(const Scalars& sc, const float4* __restrict__ cub, int n_cub,
                                                     const float4* __restrict__ osph, int n_osph, const float* x,
                                                     bool quad, int mode, const float* b_in, float s_coll_in,
                                                     float* g, PlaceScratch& ps, float4* gcell, PlaceOut& out) {
    const int lane = threadIdx.x & 31;
    const int B = sc.B;
    const bool want_grad = mode != kPlaceForward;
    const float u = sc.cell_size, r = 0.25f * u;
    const float4 half = make_float4(0.5f * u, 0.5f * u, 0.5f * u, r);

    // -- per-block terms (lane i owns block i): height residual, the cube frame (cos, sin)
    float my_e = 0.f;
    if (lane < B) {
        const int i = lane;
        my_e = x[4 * i + 2] - sc.z_star;
        ps.e[i] = my_e;
        block_cuboid(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3], half, ps.bc[i]);
        if (want_grad) {
            const float b = mode == kPlaceStage1 ? sc.w_height * (my_e > 0.f ? 1.f : (my_e < 0.f ? -1.f : 0.f)) : b_in[i];
            g[4 * i] = 0.f; g[4 * i + 1] = 0.f; g[4 * i + 2] = b; g[4 * i + 3] = 0.f;
        }
    }
    __syncwarp();

    const float s_coll = mode == kPlaceStage1 ? sc.w_coll : s_coll_in;
    float coll = 0.f, maxpen = 0.f;
    const int n_items = 8 * sc.n_cells;
    for (int base = 0; base < n_items; base += 32) {
        const int it = base + lane;
        const bool valid = it < n_items;
        const int k = valid ? it >> 3 : 0, m = it & 7;
        const int j = sc.cell_block[k];
        const float c = ps.bc[j][1].x, s = ps.bc[j][1].y;
        const float lx = sc.cell[k].x + ((m & 1) ? 0.25f : -0.25f) * u;
        const float ly = sc.cell[k].y + ((m & 2) ? 0.25f : -0.25f) * u;
        const float lz = ((m & 4) ? 0.25f : -0.25f) * u;
        const float cx = x[4 * j] + c * lx - s * ly, cy = x[4 * j + 1] + s * lx + c * ly, cz = x[4 * j + 2] + lz;
        float ax = 0.f, ay = 0.f, az = 0.f;   // dC/dc of this sphere (scaled by 2 pen in the quadratic form)
        if (valid) {
            for (int o = 0; o < n_cub; ++o) {
                float gx, gy, gz;
                const float pen = pen_cuboid<float>(cx, cy, cz, r, cub[4 * o], cub[4 * o + 1], cub[4 * o + 2],
                                                    cub[4 * o + 3], gx, gy, gz);
                if (pen > 0.f) {
                    maxpen = fmaxf(maxpen, pen);
                    coll += quad ? pen * pen : pen;
                    const float sg = quad ? 2.f * pen : 1.f;
                    ax += sg * gx; ay += sg * gy; az += sg * gz;
                }
            }
            for (int o = 0; o < n_osph; ++o) {
                float gx, gy, gz;
                const float pen = pen_sphere<float>(cx, cy, cz, r, osph[o], gx, gy, gz);
                if (pen > 0.f) {
                    maxpen = fmaxf(maxpen, pen);
                    coll += quad ? pen * pen : pen;
                    const float sg = quad ? 2.f * pen : 1.f;
                    ax += sg * gx; ay += sg * gy; az += sg * gz;
                }
            }
        }
        // cubes of the blocks below j in the skeleton order
        for (int i = 0; i + 1 < B; ++i) {
            float bx = 0.f, by = 0.f, bz = 0.f, byaw = 0.f;   // dC/d(pose i) from this sphere
            bool hit = false;
            const float oxi = x[4 * i], oyi = x[4 * i + 1], ozi = x[4 * i + 2];
            const float dxo = cx - oxi, dyo = cy - oyi, dzo = cz - ozi, reach = sc.cell_reach[i] + r;
            if (valid && i < j && dxo * dxo + dyo * dyo + dzo * dzo < reach * reach) {
                const float ci = ps.bc[i][1].x, si = ps.bc[i][1].y;
                const float4 c0 = make_float4(ci, si, 0.f, half.x), c1 = make_float4(-si, ci, 0.f, half.y);
                const float4 c2 = make_float4(0.f, 0.f, 1.f, half.z);
                for (int kk = sc.cell_start[i]; kk < sc.cell_start[i + 1]; ++kk) {
                    const float2 off = sc.cell[kk];
                    const float4 o = make_float4(oxi + ci * off.x - si * off.y, oyi + si * off.x + ci * off.y, ozi, 0.f);
                    float gx, gy, gz;
                    const float pen = pen_cuboid<float>(cx, cy, cz, r, o, c0, c1, c2, gx, gy, gz);
                    if (pen > 0.f) {
                        hit = true;
                        maxpen = fmaxf(maxpen, pen);
                        coll += quad ? pen * pen : pen;
                        const float sg = quad ? 2.f * pen : 1.f;
                        gx *= sg; gy *= sg; gz *= sg;
                        ax += gx; ay += gy; az += gz;
                        // the block moves rigidly about its origin: d/dO = -g, d/dyaw = -((c - O) x g)_z
                        bx -= gx; by -= gy; bz -= gz;
                        byaw -= dxo * gy - dyo * gx;
                    }
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
            float gyaw = ax * (-s * lx - c * ly) + ay * (c * lx - s * ly);   // dc/dyaw_j
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, off);
                ay += __shfl_xor_sync(0xffffffffu, ay, off);
                az += __shfl_xor_sync(0xffffffffu, az, off);
                gyaw += __shfl_xor_sync(0xffffffffu, gyaw, off);
            }
            if (valid && m == 0) gcell[k] = make_float4(ax, ay, az, gyaw);
        }
    }
    __syncwarp();
    if (want_grad && lane < B) {
        const int i = lane;
        float sx = 0.f, sy = 0.f, sz = 0.f, syaw = 0.f;
        for (int k = sc.cell_start[i]; k < sc.cell_start[i + 1]; ++k) {
            const float4 v = gcell[k];
            sx += v.x; sy += v.y; sz += v.z; syaw += v.w;
        }
        g[4 * i] += s_coll * sx; g[4 * i + 1] += s_coll * sy; g[4 * i + 2] += s_coll * sz; g[4 * i + 3] += s_coll * syaw;
    }
    out.c_coll = warp_sum(coll);
    out.maxpen = warp_max(maxpen);
    out.c_stable = 0.f;
    out.c_height = warp_sum(lane < B ? fabsf(my_e) : 0.f);
    out.maxD = 0.f;
    out.maxdz = warp_max(lane < B ? fabsf(my_e) : 0.f);
    __syncwarp();
}

// The placement cost of the problem's goal (tower or packing).
__device__ __forceinline__ void place_eval(const Scalars& sc, const float4* __restrict__ cub, int n_cub,
                                           const float4* __restrict__ osph, int n_osph, const float* x, bool quad,
                                           int mode, float* g, PlaceScratch& ps, float4* gcell, uint32_t* cand,
                                           PlaceOut& out) {
    if (sc.kind == kKindPack)
        place_eval_pack_warp(sc, cub, n_cub, osph, n_osph, x, quad, mode, nullptr, 0.f, g, ps, gcell, out);
    else
        place_eval_warp(sc, cub, n_cub, osph, n_osph, x, quad, mode, nullptr, nullptr, 0.f, g, ps, cand, out);
}

}  // namespace spasm
