// Stage 2 of SPaSM: trajectory-optimisation helpers shared by the kernels.
//
// Configuration layout (two motion segments per block, S = W-1 steps each, shared
// endpoints stored once): C = 2BS + 1 configurations, q[0] = q_home (fixed), segment
// s covers (sS, (s+1)S], block b = s/2 is being approached (s even: transit) or carried
// (s odd: transfer).  Grasp of block b at t = (2b+1)S, place at t = (2b+2)S.
#pragma once
#include "common.cuh"

namespace spasm {

__host__ __device__ __forceinline__ int t_grasp(int S, int b) { return (2 * b + 1) * S; }
__host__ __device__ __forceinline__ int t_place(int S, int b) { return (2 * b + 2) * S; }

// Residual vector of the augmented Lagrangian (NR = 9B + 3):
//   [5b..5b+4] grasp of block b: position error (3), roll, pitch   (w_start)
//   [5B+2b..+1] place of block b: roll, pitch                        (w_start)
//   [7B+b] height residual, [8B+b] CoM distance,                    (w_height, w_stable)
//   [9B] placement collisions, [9B+1] C_arm, [9B+2] C_block.         (w_coll, w_arm, w_block)
__device__ __forceinline__ float residual_sqrt_weight(const Scalars& sc, int r) {
    const int B = sc.B;
    const int k = r < 7 * B ? 0 : r < 8 * B ? 1 : r < 9 * B ? 2 : r == 9 * B ? 3 : r == 9 * B + 1 ? 4 : 5;
    return sc.sqw[k];
}

// roll = atan2(R21, R22), pitch = atan2(-R20, hypot(R21, R22)) (ZYX) of a rotation R, and
// the vectors w_roll, w_pitch with d(roll) = w_roll . omega for R <- (I + [omega]x) R.
template <typename T>
__device__ __forceinline__ void roll_pitch_torque(const T R[9], T& roll, T& pitch, T wr[3], T wp[3]) {
    const T r20 = R[6], r21 = R[7], r22 = R[8];
    const T h2 = r21 * r21 + r22 * r22, h = sqrt(h2);
    roll = atan2(r21, r22);
    pitch = atan2(-r20, h);
    if (wr) {
        wr[0] = (r22 * R[4] - r21 * R[5]) / h2;
        wr[1] = (r21 * R[2] - r22 * R[1]) / h2;
        wr[2] = (T)0;
        const T den = r20 * r20 + h2;
        wp[0] = (-h * R[3] + r20 * (r21 * R[4] + r22 * R[5]) / h) / den;
        wp[1] = (h * R[0] - r20 * (r21 * R[1] + r22 * R[2]) / h) / den;
        wp[2] = (T)0;
    }
}

// d yaw / d omega for yaw = atan2(e_y, e_x) of a rotating unit vector e (the block's x axis)
__device__ __forceinline__ void yaw_torque(const float e[3], float w[3]) {
    const float den = e[0] * e[0] + e[1] * e[1];
    w[0] = -e[0] * e[2] / den;
    w[1] = -e[1] * e[2] / den;
    w[2] = 1.f;
}

}  // namespace spasm
