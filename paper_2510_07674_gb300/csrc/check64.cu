// FP64 feasibility check of returned trajectories (GetSatisfyingParticles applied to the
// final solutions, |f(x)| < eps of Sec. III), evaluated in double precision on the
// float32 joint values the optimiser returned.  `split` CTAs per solution share its
// configurations (arm / held-block penetrations, joint limits); the first also takes the
// grasp, tilt and placement metrics.  Each CTA folds its maxima into the solution's
// accumulator with atomics, and the CTA that arrives last (counter after a fence; nothing
// waits) turns them into the metrics and the flag and clears the accumulator.
#include "check64.h"
#include "stage2.cuh"

namespace spasm {

// Kinematics from the joint angles' sines and cosines.
__device__ __forceinline__ void fk64_sc(const Scalars64& s, const double sn7[7], const double cs7[7], double R[8][9],
                                        double o[8][3], double Rt[9], double pt[3]) {
    for (int i = 0; i < 9; ++i) R[0][i] = (i % 4 == 0) ? 1.0 : 0.0;
    o[0][0] = o[0][1] = o[0][2] = 0.0;
    for (int k = 0; k < 7; ++k) {
        const double sn = sn7[k], cs = cs7[k];
        for (int i = 0; i < 9; ++i) R[k + 1][i] = R[k][i];
        for (int i = 0; i < 3; ++i) o[k + 1][i] = o[k][i];
        dh_step<double>(R[k + 1], o[k + 1], s.ca[k], s.sa[k], s.a[k], s.d[k], cs, sn);
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            Rt[3 * i + j] = R[7][3 * i] * s.ee_R[j] + R[7][3 * i + 1] * s.ee_R[3 + j] + R[7][3 * i + 2] * s.ee_R[6 + j];
        pt[i] = o[7][i] + R[7][3 * i] * s.ee_p[0] + R[7][3 * i + 1] * s.ee_p[1] + R[7][3 * i + 2] * s.ee_p[2];
    }
}

__device__ __forceinline__ void fk64(const Scalars64& s, const double q[7], double R[8][9], double o[8][3],
                                     double Rt[9], double pt[3]) {
    double sn[7], cs[7];
    for (int k = 0; k < 7; ++k) sincos(s.th0[k] + q[k], &sn[k], &cs[k]);
    fk64_sc(s, sn, cs, R, o, Rt, pt);
}

__device__ __forceinline__ void held64(const Scalars64& s, int b, const double Rt[9], const double pt[3], double Rb[9],
                                       double pb[3]) {
    const double off = s.half[b][2] + s.grasp_off;
    for (int i = 0; i < 3; ++i) {
        Rb[3 * i] = Rt[3 * i];
        Rb[3 * i + 1] = -Rt[3 * i + 1];
        Rb[3 * i + 2] = -Rt[3 * i + 2];
        pb[i] = pt[i] + off * Rt[3 * i + 2];
    }
}

struct D4 { double x, y, z, w; };

__device__ __forceinline__ void block_cub64(const double pose[4], const double h[3], D4 c[4]) {
    double sn, cs;
    sincos(pose[3], &sn, &cs);
    c[0] = D4{pose[0], pose[1], pose[2], 0.0};
    c[1] = D4{cs, sn, 0.0, h[0]};
    c[2] = D4{-sn, cs, 0.0, h[1]};
    c[3] = D4{0.0, 0.0, 1.0, h[2]};
}

__device__ __forceinline__ double pen_env64(const Scalars64& s, const D4* cub, const D4* osph, double cx, double cy,
                                            double cz, double r) {
    double m = 0.0, gx, gy, gz;
    for (int o = 0; o < s.n_cub; ++o)
        m = fmax(m, pen_cuboid<double>(cx, cy, cz, r, cub[4 * o], cub[4 * o + 1], cub[4 * o + 2], cub[4 * o + 3], gx, gy, gz));
    for (int o = 0; o < s.n_osph; ++o) m = fmax(m, pen_sphere<double>(cx, cy, cz, r, osph[o], gx, gy, gz));
    return m;
}

constexpr int kChkThreads = 128;
constexpr int kChkLanes = 4;                            // lanes sharing one configuration's spheres
constexpr int kChkCfgs = kChkThreads / kChkLanes;       // configurations per CTA pass
constexpr int kChkMaxSplit = (1024 + kChkCfgs - 1) / kChkCfgs;
static_assert(kChkLanes == 4, "a quad computes the seven joints' sines and cosines as joints q and q + 4");

__global__ void __launch_bounds__(kChkThreads) k_check64(const __grid_constant__ Scalars64 s, const D4* __restrict__ cub,
                                                        const D4* __restrict__ osph, const float* __restrict__ q,
                                                        const int* __restrict__ n_sol, int P, double* __restrict__ metrics,
                                                        int* __restrict__ ok, CheckAcc* __restrict__ acc, int split) {
    const int r = blockIdx.x, slice = blockIdx.y;
    if (r >= P) return;
    const int n = n_sol ? min(*n_sol, P) : P;
    const int tid = threadIdx.x;
    if (r >= n) {
        if (tid == 0 && slice == 0) ok[r] = 0;
        return;
    }
    const int B = s.B, S = s.S, C = s.C;
    const float* qr = q + (size_t)r * C * 8;
    __shared__ double pose[kMaxB][4];
    __shared__ D4 bcub[kMaxB][4], icub[kMaxB][4];
    __shared__ double red[kChkThreads];
    __shared__ double vstart[kMaxB], vtilt[kMaxB];
    if (tid < B) {
        double qq[7], R[8][9], o[8][3], Rt[9], pt[3], Rb[9], pb[3];
        vtilt[tid] = 0.0;
        block_cub64(s.init[tid], s.half[tid], icub[tid]);
        if (!s.p2p) {
            // placed pose from the place configuration
            for (int j = 0; j < 7; ++j) qq[j] = qr[t_place(S, tid) * 8 + j];
            fk64(s, qq, R, o, Rt, pt);
            held64(s, tid, Rt, pt, Rb, pb);
            pose[tid][0] = pb[0]; pose[tid][1] = pb[1]; pose[tid][2] = pb[2]; pose[tid][3] = atan2(Rb[3], Rb[0]);
            block_cub64(pose[tid], s.half[tid], bcub[tid]);
            const double roll = atan2(Rb[7], Rb[8]), pitch = atan2(-Rb[6], sqrt(Rb[7] * Rb[7] + Rb[8] * Rb[8]));
            vtilt[tid] = roll * roll + pitch * pitch;
        } else {
            for (int i = 0; i < 4; ++i) pose[tid][i] = s.init[tid][i];
        }
        for (int j = 0; j < 7; ++j) qq[j] = qr[t_grasp(S, tid) * 8 + j];
        fk64(s, qq, R, o, Rt, pt);
        held64(s, tid, Rt, pt, Rb, pb);
        const double roll = atan2(Rb[7], Rb[8]), pitch = atan2(-Rb[6], sqrt(Rb[7] * Rb[7] + Rb[8] * Rb[8]));
        double e2 = 0.0;
        for (int i = 0; i < 3; ++i) { const double d = pb[i] - s.init[tid][i]; e2 += d * d; }
        vstart[tid] = e2 + roll * roll + pitch * pitch;
    }
    __syncthreads();

    // arm and held-block penetrations over every configuration, joint limits.  A quad of
    // lanes takes one configuration: each lane runs the kinematics and a quarter of its
    // spheres; every lane of a warp takes the same number of passes, so the quad shuffles
    // see all lanes.
    double maxpen = 0.0;
    int limits_ok = 1;
    const int quad = tid & (kChkLanes - 1);
    for (int base = slice * kChkCfgs; base < C - 1; base += kChkCfgs * split) {
        const int t = 1 + base + tid / kChkLanes;
        const bool valid = t < C;
        const int tt = valid ? t : C - 1;
        const int seg = (tt - 1) / S, b = seg >> 1, jj = tt - seg * S;
        const bool held = (seg & 1) && jj < S;
        double qq[7], R[8][9], o[8][3], Rt[9], pt[3];
        for (int j = 0; j < 7; ++j) {
            qq[j] = qr[tt * 8 + j];
            if (valid && (qq[j] < s.qlo[j] || qq[j] > s.qhi[j])) limits_ok = 0;
        }
        // the quad shares the joint angles' sines and cosines: lane `quad` takes joints quad and
        // quad + 4
        double sn7[7], cs7[7];
        {
            double s1, c1, s2 = 0.0, c2 = 1.0;
            sincos(s.th0[quad] + qq[quad], &s1, &c1);
            if (quad + 4 < 7) sincos(s.th0[quad + 4] + qq[quad + 4], &s2, &c2);
            const int first = (tid & 31) & ~(kChkLanes - 1);
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                sn7[k] = __shfl_sync(0xffffffffu, k < 4 ? s1 : s2, first + (k & 3));
                cs7[k] = __shfl_sync(0xffffffffu, k < 4 ? c1 : c2, first + (k & 3));
            }
        }
        fk64_sc(s, sn7, cs7, R, o, Rt, pt);
        const int n_items = s.n_rsph + (held ? 8 : 0);
        double Rb[9], pb[3];
        if (held) held64(s, b, Rt, pt, Rb, pb);
        auto centre = [&](int it, double& cx, double& cy, double& cz, double& rad) {
            if (it < s.n_rsph) {
                const int l = s.rlink[it];
                const double* ls = s.rsph[it];
                cx = R[l][0] * ls[0] + R[l][1] * ls[1] + R[l][2] * ls[2] + o[l][0];
                cy = R[l][3] * ls[0] + R[l][4] * ls[1] + R[l][5] * ls[2] + o[l][1];
                cz = R[l][6] * ls[0] + R[l][7] * ls[1] + R[l][8] * ls[2] + o[l][2];
                rad = ls[3];
            } else {
                const int m = it - s.n_rsph;
                const double lx = ((m & 1) ? 0.5 : -0.5) * s.half[b][0];
                const double ly = ((m & 2) ? 0.5 : -0.5) * s.half[b][1];
                const double lz = ((m & 4) ? 0.5 : -0.5) * s.half[b][2];
                cx = pb[0] + Rb[0] * lx + Rb[1] * ly + Rb[2] * lz;
                cy = pb[1] + Rb[3] * lx + Rb[4] * ly + Rb[5] * lz;
                cz = pb[2] + Rb[6] * lx + Rb[7] * ly + Rb[8] * lz;
                rad = s.hmin[b] * 0.5;
            }
        };
        // exact cull: box of all spheres of this configuration (the quad's four shares)
        // against each obstacle's box
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int it = quad; it < n_items; it += kChkLanes) {
            double cx, cy, cz, rad;
            centre(it, cx, cy, cz, rad);
            lo[0] = fmin(lo[0], cx - rad); lo[1] = fmin(lo[1], cy - rad); lo[2] = fmin(lo[2], cz - rad);
            hi[0] = fmax(hi[0], cx + rad); hi[1] = fmax(hi[1], cy + rad); hi[2] = fmax(hi[2], cz + rad);
        }
#pragma unroll
        for (int off = 1; off < kChkLanes; off <<= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
                hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
            }
        if (!valid) continue;
        auto visit = [&](const D4* c) {
            // box of a cuboid record: centre +- |R| h
            double e[3];
            for (int a = 0; a < 3; ++a)
                e[a] = fabs((&c[1].x)[a]) * c[1].w + fabs((&c[2].x)[a]) * c[2].w + fabs((&c[3].x)[a]) * c[3].w;
            if (c[0].x - e[0] > hi[0] || c[0].x + e[0] < lo[0] || c[0].y - e[1] > hi[1] || c[0].y + e[1] < lo[1] ||
                c[0].z - e[2] > hi[2] || c[0].z + e[2] < lo[2])
                return;
            for (int it = quad; it < n_items; it += kChkLanes) {
                double cx, cy, cz, rad, gx, gy, gz;
                centre(it, cx, cy, cz, rad);
                maxpen = fmax(maxpen, pen_cuboid<double>(cx, cy, cz, rad, c[0], c[1], c[2], c[3], gx, gy, gz));
            }
        };
        for (int ob = 0; ob < s.n_cub; ++ob) visit(&cub[4 * ob]);
        for (int ob = 0; ob < s.n_osph; ++ob) {
            const D4 sp = osph[ob];
            if (sp.x - sp.w > hi[0] || sp.x + sp.w < lo[0] || sp.y - sp.w > hi[1] || sp.y + sp.w < lo[1] ||
                sp.z - sp.w > hi[2] || sp.z + sp.w < lo[2])
                continue;
            for (int it = quad; it < n_items; it += kChkLanes) {
                double cx, cy, cz, rad, gx, gy, gz;
                centre(it, cx, cy, cz, rad);
                maxpen = fmax(maxpen, pen_sphere<double>(cx, cy, cz, rad, sp, gx, gy, gz));
            }
        }
        for (int k = 0; k < B; ++k) {
            if (k == b) continue;
            visit(k < b ? bcub[k] : icub[k]);
        }
    }
    // placement: spheres of block j vs the environment and the blocks below
    double place_pen = 0.0;
    for (int it = tid; it < ((s.p2p || slice != 0) ? 0 : 8 * B); it += kChkThreads) {
        const int j = it >> 3, m = it & 7;
        const double lx = ((m & 1) ? 0.5 : -0.5) * s.half[j][0];
        const double ly = ((m & 2) ? 0.5 : -0.5) * s.half[j][1];
        const double lz = ((m & 4) ? 0.5 : -0.5) * s.half[j][2];
        double sn, cs;
        sincos(pose[j][3], &sn, &cs);
        const double cx = pose[j][0] + cs * lx - sn * ly, cy = pose[j][1] + sn * lx + cs * ly, cz = pose[j][2] + lz;
        const double rad = s.hmin[j] * 0.5;
        place_pen = fmax(place_pen, pen_env64(s, cub, osph, cx, cy, cz, rad));
        for (int i = 0; i < j; ++i) {
            double gx, gy, gz;
            place_pen = fmax(place_pen, pen_cuboid<double>(cx, cy, cz, rad, bcub[i][0], bcub[i][1], bcub[i][2], bcub[i][3],
                                                           gx, gy, gz));
        }
    }
    // block reductions (max) of the penetrations and the limit flag
    red[tid] = maxpen;
    __syncthreads();
    for (int w = kChkThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
        __syncthreads();
    }
    const double mp = red[0];
    __syncthreads();
    red[tid] = place_pen;
    __syncthreads();
    for (int w = kChkThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
        __syncthreads();
    }
    const double pp = red[0];
    const int lim = __syncthreads_and(limits_ok);
    if (tid == 0) {
        CheckAcc& A = acc[r];
        atomicMax(&A.mp, (unsigned long long)__double_as_longlong(mp));   // non-negative: integer order
        if (!lim) atomicOr(&A.viol, 1);
        if (slice == 0) {
            double ms = 0.0, mt = 0.0, mD = 0.0, mz = 0.0;
            for (int b = 0; b < B; ++b) {
                ms = fmax(ms, vstart[b]);
                mt = fmax(mt, vtilt[b]);
                if (!s.p2p) mz = fmax(mz, fabs(pose[b][2] - s.zt[b]));
                if (b + 1 < B) {
                    double mx = 0.0, my = 0.0;
                    for (int j = b + 1; j < B; ++j) { mx += pose[j][0]; my += pose[j][1]; }
                    mx /= (double)(B - 1 - b);
                    my /= (double)(B - 1 - b);
                    double sn, cs;
                    sincos(pose[b][3], &sn, &cs);
                    const double vx = mx - pose[b][0], vy = my - pose[b][1];
                    const double ux = cs * vx + sn * vy, uy = -sn * vx + cs * vy;
                    const double ex = fmax(fabs(ux) - s.half[b][0], 0.0), ey = fmax(fabs(uy) - s.half[b][1], 0.0);
                    mD = fmax(mD, sqrt(ex * ex + ey * ey));
                }
            }
            A.pp = pp; A.ms = ms; A.mt = mt; A.mD = mD; A.mz = mz;
        }
        __threadfence();
        if (atomicAdd(&A.count, 1) == split - 1) {   // the last slice of this solution
            __threadfence();
            const volatile CheckAcc& V = A;
            const double mpa = __longlong_as_double((long long)V.mp);
            const int lim_all = V.viol == 0;
            double* m = metrics + (size_t)r * 6;
            m[0] = mpa; m[1] = V.ms; m[2] = V.mt; m[3] = V.pp; m[4] = V.mD; m[5] = V.mz;
            ok[r] = (mpa <= s.eps && V.ms <= s.eps_start && V.mt <= s.eps_start && V.pp <= s.eps && V.mD <= s.eps &&
                     V.mz <= s.eps && lim_all) ? 1 : 0;
            A.mp = 0ull; A.viol = 0; A.count = 0;   // ready for the next check
        }
    }
}

cudaError_t launch_check64(const Scalars64& s, const void* cub, const void* osph, const float* q, const int* n_sol, int P,
                           double* metrics, int* ok, CheckAcc* acc, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int split = max(1, min(kChkMaxSplit, (s.C - 1 + kChkCfgs - 1) / kChkCfgs));
    k_check64<<<dim3(P, split), kChkThreads, 0, st>>>(s, static_cast<const D4*>(cub), static_cast<const D4*>(osph), q, n_sol,
                                                      P, metrics, ok, acc, split);
    return cudaGetLastError();
}

}  // namespace spasm
