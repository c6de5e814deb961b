// Lift of Sec. III-B: placements -> joint-space trajectory particles.  The IK targets (the
// grasp of each block's initial pose and its placement) are solved by the closed-form IK of
// the Franka joint layout, one warp per target with a lane per value of the free last joint
// (ik_mode 1), or by damped least squares, one thread per target (ik_mode 0); one thread per
// remaining configuration interpolates start -> intermediate waypoint -> goal.
#include "launch_s2.h"
#include "stage2.cuh"

namespace spasm {

// ================================================================================== lift
// Damped-least-squares IK (Wampler 1986): dq = J^T (J J^T + damp^2 I)^-1 e with
//   e = (p* - p, 1/2 sum_c R[:,c] x R*[:,c]),  J_k = (z_k x (p - o_k), z_k),
// solved by a 6x6 Cholesky factorisation (the system matrix is SPD thanks to damping).
__device__ void ik_dls(const Scalars& sc, const float Rs[9], const float ps[3], float q[7]) {
    for (int it = 0; it < sc.K_ik; ++it) {
        float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, o[3] = {0, 0, 0};
        float z[7][3], org[7][3];
        for (int k = 0; k < 7; ++k) {
            float s, c;
            sincosf(sc.th0[k] + q[k], &s, &c);
            dh_step<float>(R, o, sc.ca[k], sc.sa[k], sc.a[k], sc.d[k], c, s);
            z[k][0] = R[2]; z[k][1] = R[5]; z[k][2] = R[8];
            org[k][0] = o[0]; org[k][1] = o[1]; org[k][2] = o[2];
        }
        float Rt[9], pt[3];
        tool_frame<float>(sc, R, o, Rt, pt);
        float e[6];
        e[0] = ps[0] - pt[0]; e[1] = ps[1] - pt[1]; e[2] = ps[2] - pt[2];
        e[3] = e[4] = e[5] = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float a0 = Rt[c], a1 = Rt[3 + c], a2 = Rt[6 + c];
            const float b0 = Rs[c], b1 = Rs[3 + c], b2 = Rs[6 + c];
            e[3] += 0.5f * (a1 * b2 - a2 * b1);
            e[4] += 0.5f * (a2 * b0 - a0 * b2);
            e[5] += 0.5f * (a0 * b1 - a1 * b0);
        }
        float J[6][7];
        for (int k = 0; k < 7; ++k) {
            const float rx = pt[0] - org[k][0], ry = pt[1] - org[k][1], rz = pt[2] - org[k][2];
            J[0][k] = z[k][1] * rz - z[k][2] * ry;
            J[1][k] = z[k][2] * rx - z[k][0] * rz;
            J[2][k] = z[k][0] * ry - z[k][1] * rx;
            J[3][k] = z[k][0]; J[4][k] = z[k][1]; J[5][k] = z[k][2];
        }
        // Cholesky of A = J J^T + damp^2 I (lower triangle L)
        float L[6][6];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j <= i; ++j) {
                float s = 0.f;
                for (int k = 0; k < 7; ++k) s += J[i][k] * J[j][k];
                if (i == j) s += sc.ik_damp * sc.ik_damp;
                for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
                L[i][j] = (i == j) ? sqrtf(fmaxf(s, 1e-30f)) : s / L[j][j];
            }
        float y[6];
        for (int i = 0; i < 6; ++i) {
            float s = e[i];
            for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
            y[i] = s / L[i][i];
        }
        for (int i = 5; i >= 0; --i) {
            float s = y[i];
            for (int k = i + 1; k < 6; ++k) s -= L[k][i] * y[k];
            y[i] = s / L[i][i];
        }
        for (int k = 0; k < 7; ++k) {
            float dq = 0.f;
            for (int i = 0; i < 6; ++i) dq += J[i][k] * y[i];
            q[k] = fminf(fmaxf(q[k] + dq, sc.qlo[k]), sc.qhi[k]);
        }
    }
}

// key: the Philox key (the problem's seed)
__device__ __forceinline__ void perturbed_home(const Scalars& sc, uint64_t key, uint32_t c0, int p, uint32_t tag,
                                               uint32_t attempt, float amp, float q[7]) {
    const U4 a = philox4x32_10(2u * c0, (uint32_t)p, tag, attempt, key);
    const U4 b = philox4x32_10(2u * c0 + 1u, (uint32_t)p, tag, attempt, key);
    const float u[7] = {u01(a.x), u01(a.y), u01(a.z), u01(a.w), u01(b.x), u01(b.y), u01(b.z)};
    for (int j = 0; j < 7; ++j) q[j] = fminf(fmaxf(sc.q_home[j] + amp * (2.f * u[j] - 1.f), sc.qlo[j]), sc.qhi[j]);
}

// ---------------------------------------------------------------------------- analytic IK
// Closed-form IK of the Franka joint layout (the lift of Sec. III-B uses an analytic IK for
// that arm; the layout is checked on the host): twists (0, -pi/2, pi/2, pi/2, -pi/2, pi/2,
// pi/2), a_0 = a_1 = a_2 = a_5 = 0, d_1 = d_3 = d_5 = d_6 = 0, any lengths and tool.  With
// the last joint fixed, frame 6 follows from the tool pose; the first three axes meet at
// the shoulder S = (0, 0, d_0) and |O6 - S| fixes theta_3 (two branches); the direction of
// S seen from frame 6 fixes theta_5 (two branches) and theta_4; frame 3's orientation
// Rz(t0) Ry(t1) Rz(t2) gives theta_0..2 (both signs of sin t1).  Every in-limit branch is
// compared with the seed and the nearest (squared joint distance) is kept in best.

// 3x3 rotation of one DH row, Rot_x(alpha) Rot_z(theta), row-major
__device__ __forceinline__ void rot_xz(float ca, float sa, float theta, float R[9]) {
    float st, ct;
    sincosf(theta, &st, &ct);
    R[0] = ct;      R[1] = -st;     R[2] = 0.f;
    R[3] = ca * st; R[4] = ca * ct; R[5] = -sa;
    R[6] = sa * st; R[7] = sa * ct; R[8] = ca;
}

__device__ __forceinline__ void mul33(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// joint angle -> q inside [lo, hi], shifted by 2 pi where that helps; false if outside
__device__ __forceinline__ bool into_limits(const Scalars& sc, int k, float theta, float& q) {
    const float two_pi = 2.f * kPi;
    float v = theta - sc.th0[k];
    v -= two_pi * floorf((v + kPi) / two_pi);
    if (v < sc.qlo[k]) v += two_pi;
    if (v > sc.qhi[k]) v -= two_pi;
    q = v;
    return v >= sc.qlo[k] && v <= sc.qhi[k];
}

__device__ void ik_analytic_nearest(const Scalars& sc, const float Rs[9], const float ps[3], float q6,
                                    const float seed[7], float best[7], float& best_d) {
    // frame 7 = target * tool^-1; frame 6 = frame 7 * T_6(q6)^-1
    float R7[9], O7[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            R7[3 * i + j] = Rs[3 * i] * sc.ee_R[3 * j] + Rs[3 * i + 1] * sc.ee_R[3 * j + 1] + Rs[3 * i + 2] * sc.ee_R[3 * j + 2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) O7[i] = ps[i] - (R7[3 * i] * sc.ee_p[0] + R7[3 * i + 1] * sc.ee_p[1] + R7[3 * i + 2] * sc.ee_p[2]);
    float R76[9];
    rot_xz(sc.ca[6], sc.sa[6], sc.th0[6] + q6, R76);
    const float t76[3] = {sc.a[6], -sc.d[6] * sc.sa[6], sc.d[6] * sc.ca[6]};   // origin of frame 7 in frame 6
    float R6[9], O6[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            R6[3 * i + j] = R7[3 * i] * R76[3 * j] + R7[3 * i + 1] * R76[3 * j + 1] + R7[3 * i + 2] * R76[3 * j + 2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) O6[i] = O7[i] - (R6[3 * i] * t76[0] + R6[3 * i + 1] * t76[1] + R6[3 * i + 2] * t76[2]);
    const float d0 = sc.d[0], d2 = sc.d[2], a3 = sc.a[3], a4 = sc.a[4], d4 = sc.d[4];
    const float v[3] = {-O6[0], -O6[1], d0 - O6[2]};                     // S - O6, world
    float w[3];                                                           // S - O6, frame 6
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = R6[i] * v[0] + R6[3 + i] * v[1] + R6[6 + i] * v[2];
    const float A = a3 * a4 + d2 * d4, Bs = d2 * a4 - a3 * d4, Rn = sqrtf(A * A + Bs * Bs);
    const float D = 0.5f * ((v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - (a3 * a3 + d2 * d2 + a4 * a4 + d4 * d4));
    if (fabsf(D) > Rn) return;                                            // out of reach for this q6
    const float phi = atan2f(Bs, A), c_3 = acosf(D / Rn);
    const float rho = sqrtf(w[0] * w[0] + w[1] * w[1]), psi = atan2f(w[0], w[1]);
    for (int i3 = 0; i3 < 2; ++i3) {
        const float t3 = i3 == 0 ? phi + c_3 : phi - c_3;
        float s3, c3;
        sincosf(t3, &s3, &c3);
        float q3, q4, q5;
        if (!into_limits(sc, 3, t3, q3)) continue;   // each joint is rejected as soon as it is known
        const float ux = -a3 * c3 - d2 * s3 - a4, uy = a3 * s3 - d2 * c3 - d4;
        if (fabsf(uy) > rho) continue;
        const float c_5 = acosf(uy / rho);
        float R34[9];
        rot_xz(sc.ca[3], sc.sa[3], t3, R34);
        for (int i5 = 0; i5 < 2; ++i5) {
            const float t5 = i5 == 0 ? psi + c_5 : psi - c_5;
            if (!into_limits(sc, 5, t5, q5)) continue;
            float s5, c5;
            sincosf(t5, &s5, &c5);
            const float sg = ux < 0.f ? -1.f : 1.f;
            const float t4 = atan2f(sg * w[2], sg * (c5 * w[0] - s5 * w[1]));
            if (!into_limits(sc, 4, t4, q4)) continue;
            float R45[9], R56[9], R35[9], R36[9], R3[9];
            rot_xz(sc.ca[4], sc.sa[4], t4, R45);
            rot_xz(sc.ca[5], sc.sa[5], t5, R56);
            mul33(R34, R45, R35);
            mul33(R35, R56, R36);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    R3[3 * i + j] = R6[3 * i] * R36[3 * j] + R6[3 * i + 1] * R36[3 * j + 1] + R6[3 * i + 2] * R36[3 * j + 2];
            }
            const float sb = sqrtf(R3[2] * R3[2] + R3[5] * R3[5]);
            for (int sgn = 1; sgn >= -1; sgn -= 2) {
                float th[3];
                if (sb < 1e-6f) {                                         // t1 = 0: only t0 + t2 is fixed
                    if (sgn < 0) break;
                    th[0] = 0.f; th[1] = atan2f(0.f, R3[8]); th[2] = atan2f(R3[3], R3[0]);
                } else {
                    const float g = (float)sgn;
                    th[1] = atan2f(g * sb, R3[8]);
                    th[0] = atan2f(g * R3[5], g * R3[2]);
                    th[2] = atan2f(g * R3[7], -g * R3[6]);
                }
                float q[7];
                bool ok = true;
                for (int k = 0; k < 3 && ok; ++k) ok = into_limits(sc, k, th[k], q[k]);
                if (!ok) continue;
                q[3] = q3; q[4] = q4; q[5] = q5; q[6] = q6;
                float d = 0.f;
#pragma unroll
                for (int j = 0; j < 7; ++j) d += (q[j] - seed[j]) * (q[j] - seed[j]);
                if (d < best_d) {
                    best_d = d;
#pragma unroll
                    for (int j = 0; j < 7; ++j) best[j] = q[j];
                }
            }
        }
    }
}

// The analytic lift tries, per target, the seed's value of the last joint and one uniform
// draw in each of kQ6Strips equal strips of its limit range (strip i: word i mod 4 of the
// Philox counter (8 c0 + i/4, particle, kTagQ6, attempt)), and keeps the in-limit solution
// nearest the seed, the first in that order on ties.
constexpr int kQ6Strips = 31;

// Tool target of IK target r = 2b + which of particle p: Rz(yaw + k pi/2) Rx(pi) at the top
// face of block b (+ grasp offset), at its initial pose (which = 0) or its placement (1).
__device__ __forceinline__ void lift_target(const Scalars& sc, uint64_t key, const float* __restrict__ place, int np, int p,
                                            int b, int which, uint32_t attempt, float Rs[9], float ps[3]) {
    const int B = sc.B;
    const U4 kk = philox4x32_10((uint32_t)b, (uint32_t)p, kTagGrasp, attempt, key);
    float pose[4];
    if (which == 0) {
        pose[0] = sc.init[b].x; pose[1] = sc.init[b].y; pose[2] = sc.init[b].z; pose[3] = sc.init[b].w;
    } else {
        const float* src = place + ((size_t)(p % np) * B + b) * 4;
        pose[0] = src[0]; pose[1] = src[1]; pose[2] = src[2]; pose[3] = src[3];
    }
    const int k = (int)((which == 0 ? kk.x : kk.y) & 3u);
    float s, c;
    sincosf(pose[3] + 0.5f * kPi * (float)k, &s, &c);
    Rs[0] = c;   Rs[1] = s;   Rs[2] = 0.f;
    Rs[3] = s;   Rs[4] = -c;  Rs[5] = 0.f;
    Rs[6] = 0.f; Rs[7] = 0.f; Rs[8] = -1.f;
    ps[0] = pose[0]; ps[1] = pose[1]; ps[2] = pose[2] + sc.half[b].z + sc.grasp_off;
}

// Analytic lift, one warp per IK target: lane 0 takes the seed's last-joint value, lane
// 1 + i strip i of ik_analytic_lift; each lane keeps its nearest in-limit branch and the warp
// takes the nearest over lanes, the lowest lane on ties, which is the choice of the
// sequential scan.  A target without an in-limit solution falls back to damped least
// squares on lane 0.
__global__ void k_lift_ik_analytic(const __grid_constant__ Scalars sc, int n, const float* __restrict__ place, int np,
                                   uint32_t attempt, float* __restrict__ q, const LoopCtl* __restrict__ ctl) {
    uint64_t key = sc.seed;
    if (ctl) { attempt = ctl->t_attempt; np = ctl->n_place; key = ctl->seed; }
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int B = sc.B;
    if (gw >= n * 2 * B || np <= 0) return;   // warp-uniform
    const int p = gw / (2 * B), r = gw % (2 * B), b = r >> 1, which = r & 1;
    if (which == 1 && sc.kind == kKindP2P) return;   // point to point: no placement
    float Rs[9], ps[3], seed[7], best[7];
    lift_target(sc, key, place, np, p, b, which, attempt, Rs, ps);
    const uint32_t c0 = (uint32_t)(2 * b + which);
    perturbed_home(sc, key, c0, p, kTagIkSeed, attempt, 0.3f, seed);
#pragma unroll
    for (int j = 0; j < 7; ++j) best[j] = seed[j];
    float q6 = seed[6];
    if (lane >= 1 && lane <= kQ6Strips) {
        const int i = lane - 1;
        const U4 u = philox4x32_10(8u * c0 + (uint32_t)(i >> 2), (uint32_t)p, kTagQ6, attempt, key);
        const uint32_t word = (i & 3) == 0 ? u.x : (i & 3) == 1 ? u.y : (i & 3) == 2 ? u.z : u.w;
        const float strip = ((float)i + u01(word)) / (float)kQ6Strips;
        q6 = sc.qlo[6] + strip * (sc.qhi[6] - sc.qlo[6]);
    }
    float d = INFINITY;
    if (lane <= kQ6Strips) ik_analytic_nearest(sc, Rs, ps, q6, seed, best, d);
    int win = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, d, off);
        const int ow = __shfl_xor_sync(0xffffffffu, win, off);
        if (od < d || (od == d && ow < win)) { d = od; win = ow; }
    }
    float qq[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) qq[j] = __shfl_sync(0xffffffffu, best[j], win);
    if (lane != 0) return;
    if (!(d < INFINITY)) {
        for (int j = 0; j < 7; ++j) qq[j] = seed[j];
        ik_dls(sc, Rs, ps, qq);
    }
    const int t = which == 0 ? t_grasp(sc.S, b) : t_place(sc.S, b);
    float* dst = q + ((size_t)p * sc.C + t) * 8;
    for (int j = 0; j < 7; ++j) dst[j] = qq[j];
    dst[7] = 0.f;
}

// Damped-least-squares lift (ik_mode 0), one thread per (particle, block, grasp|place)
__global__ void k_lift_ik(const __grid_constant__ Scalars sc, int n, const float* __restrict__ place, int np,
                          uint32_t attempt, float* __restrict__ q, const LoopCtl* __restrict__ ctl) {
    uint64_t key = sc.seed;
    if (ctl) { attempt = ctl->t_attempt; np = ctl->n_place; key = ctl->seed; }
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int B = sc.B;
    if (gid >= n * 2 * B) return;
    if (np <= 0) return;
    const int p = gid / (2 * B), r = gid % (2 * B), b = r >> 1, which = r & 1;
    if (which == 1 && sc.kind == kKindP2P) return;   // point to point: no placement
    float Rs[9], ps[3];
    lift_target(sc, key, place, np, p, b, which, attempt, Rs, ps);
    float qq[7];
    perturbed_home(sc, key, (uint32_t)(2 * b + which), p, kTagIkSeed, attempt, 0.3f, qq);
    ik_dls(sc, Rs, ps, qq);
    const int t = which == 0 ? t_grasp(sc.S, b) : t_place(sc.S, b);
    float* dst = q + ((size_t)p * sc.C + t) * 8;
    for (int j = 0; j < 7; ++j) dst[j] = qq[j];
    dst[7] = 0.f;
}

// one thread per (particle, configuration): home, or linear interpolation
// start -> via -> goal within the configuration's segment
__global__ void k_lift_interp(const __grid_constant__ Scalars sc, int n, int np, uint32_t attempt,
                              float* __restrict__ q, const LoopCtl* __restrict__ ctl) {
    uint64_t key = sc.seed;
    if (ctl) { attempt = ctl->t_attempt; np = ctl->n_place; key = ctl->seed; }
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n * sc.C) return;
    if (np <= 0) return;
    const int p = gid / sc.C, t = gid % sc.C, S = sc.S;
    float* dst = q + ((size_t)p * sc.C + t) * 8;
    if (t == 0) {
        for (int j = 0; j < 7; ++j) dst[j] = sc.q_home[j];
        dst[7] = 0.f;
        return;
    }
    const int jj = t % S;
    if (jj == 0) return;   // segment endpoint, written by the IK kernel
    const int s = t / S, m = S / 2;
    float via[7];
    perturbed_home(sc, key, (uint32_t)s, p, kTagVia, attempt, 0.3f, via);
    // segment 0 starts at home; this launch writes that row itself (t == 0 above), so it is
    // taken from the constants rather than read back from q
    const float* qa = s == 0 ? sc.q_home : q + ((size_t)p * sc.C + s * S) * 8;
    const float* qb = q + ((size_t)p * sc.C + (s + 1) * S) * 8;
    for (int j = 0; j < 7; ++j) {
        float v;
        if (jj <= m) v = qa[j] + ((float)jj / (float)m) * (via[j] - qa[j]);
        else v = via[j] + ((float)(jj - m) / (float)(S - m)) * (qb[j] - via[j]);
        dst[j] = v;
    }
    dst[7] = 0.f;
}

// ================================================================================== launcher
cudaError_t launch_lift(const Scalars& sc, int n, const float* place, int n_place, uint32_t attempt, float* q,
                        cudaStream_t st, const LoopCtl* ctl) {
    if (n <= 0) return cudaSuccess;
    const int n_ik = n * 2 * sc.B;
    if (sc.ik_mode == 1) {
        const long long threads = 32LL * n_ik;   // a warp per target
        k_lift_ik_analytic<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(sc, n, place, n_place, attempt, q, ctl);
    } else {
        k_lift_ik<<<(n_ik + 127) / 128, 128, 0, st>>>(sc, n, place, n_place, attempt, q, ctl);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n_cfg = n * sc.C;
    k_lift_interp<<<(n_cfg + 255) / 256, 256, 0, st>>>(sc, n, n_place, attempt, q, ctl);
    return cudaGetLastError();
}

}  // namespace spasm
