// ArgSort(C)[:k] of Alg. 1 on the GPU: the k smallest costs, ordered by (cost, index).
//
// One CTA of 1024 threads:  (1) costs become order-preserving 32-bit keys in shared
// memory; (2) a 4-pass radix select (8 bits per pass, shared-memory histograms with
// integer atomics) finds the k-th smallest key T and how many keys equal to T are taken;
// (3) a stable, scan-based compaction gathers every key < T and the lowest-index keys
// == T; (4) a bitonic sort of the k selected (key << 32 | index) pairs.  Integer work
// only, so the result is deterministic and equals a stable sort by (cost, index).
#pragma once
#include "common.cuh"

namespace spasm {

constexpr int kSelectThreads = 1024;

// NaN sorts last; -0 and +0 compare equal (both map to the key of +0).
__device__ __forceinline__ uint32_t cost_key(float c) {
    if (c != c) return 0xFFFFFFFFu;
    c = c + 0.0f;
    const uint32_t u = __float_as_uint(c);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// inclusive block scan of one int per thread (1024 threads); returns the inclusive value
// and the block total in *total.
__device__ __forceinline__ int block_scan_incl(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_tot[lane] = s;
    }
    __syncthreads();
    const int res = v + (w > 0 ? warp_tot[w - 1] : 0);
    *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return res;
}

// keys (n) and pairs (kp2 >= k, power of two) live in dynamic shared memory.
__global__ void __launch_bounds__(kSelectThreads) k_topk(const float* __restrict__ cost, int n, int k,
                                                          int* __restrict__ out_idx, float* __restrict__ out_cost,
                                                          int kp2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* pairs = reinterpret_cast<unsigned long long*>(smem_raw);
    uint32_t* keys = reinterpret_cast<uint32_t*>(pairs + kp2);
    __shared__ int hist[256];
    __shared__ int warp_tot[32];
    __shared__ uint32_t s_prefix;
    __shared__ int s_need;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (k > n) k = n;

    for (int i = tid; i < n; i += nt) keys[i] = cost_key(cost[i]);
    if (tid == 0) { s_prefix = 0; s_need = k; }
    __syncthreads();

    // radix select of the k-th smallest key (1-based rank k)
    uint32_t mask = 0;
    for (int shift = 24; shift >= 0 && k > 0; shift -= 8) {
        for (int i = tid; i < 256; i += nt) hist[i] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix;
        for (int i = tid; i < n; i += nt) {
            const uint32_t key = keys[i];
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncthreads();
        if (tid == 0) {
            int need = s_need, acc = 0, bkt = 0;
            for (; bkt < 256; ++bkt) {
                if (acc + hist[bkt] >= need) break;
                acc += hist[bkt];
            }
            s_need = need - acc;
            s_prefix = prefix | ((uint32_t)bkt << shift);
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    const uint32_t T = s_prefix;
    const int need_eq = s_need;   // keys == T to take (lowest indices first)

    // stable compaction over contiguous chunks
    const int chunk = (n + nt - 1) / nt;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    int n_less = 0, n_eq = 0;
    for (int i = lo; i < hi; ++i) {
        const uint32_t key = keys[i];
        n_less += key < T;
        n_eq += key == T;
    }
    int tot_less, tot_eq;
    const int less_incl = block_scan_incl(n_less, warp_tot, &tot_less);
    const int eq_incl = block_scan_incl(n_eq, warp_tot, &tot_eq);
    int pos_less = less_incl - n_less, pos_eq = eq_incl - n_eq;
    const int n_sel_less = k > 0 ? k - need_eq : 0;
    for (int i = lo; i < hi; ++i) {
        const uint32_t key = keys[i];
        if (k > 0 && key < T) {
            pairs[pos_less++] = ((unsigned long long)key << 32) | (uint32_t)i;
        } else if (k > 0 && key == T) {
            if (pos_eq < need_eq) pairs[n_sel_less + pos_eq] = ((unsigned long long)key << 32) | (uint32_t)i;
            ++pos_eq;
        }
    }
    for (int i = k + tid; i < kp2; i += nt) pairs[i] = ~0ull;
    __syncthreads();

    // bitonic sort of kp2 pairs (ascending)
    for (int size = 2; size <= kp2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < kp2 / 2; i += nt) {
                const int lo_i = 2 * i - (i & (stride - 1));
                const int hi_i = lo_i + stride;
                const bool up = (lo_i & size) == 0;
                const unsigned long long a = pairs[lo_i], b = pairs[hi_i];
                if ((a > b) == up) { pairs[lo_i] = b; pairs[hi_i] = a; }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < k; i += nt) {
        const int idx = (int)(uint32_t)(pairs[i] & 0xffffffffull);
        out_idx[i] = idx;
        if (out_cost) out_cost[i] = cost[idx];
    }
}

}  // namespace spasm
