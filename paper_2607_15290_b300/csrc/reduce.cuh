// reduce.cuh -- deterministic block reductions: every block writes its partial
// sums to partials[block * 64 + i]; a single block then sums them in a fixed
// order, so results do not depend on scheduling.
#pragma once
#include <cuda_runtime.h>

namespace llg {

static constexpr int RB_THREADS = 256;
static constexpr int RB_STRIDE = 64;

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NV], int nv, double *out) {
    __shared__ double red[RB_THREADS / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < nv) {
            double v = acc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][i] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < RB_THREADS / 32; ++w) s += red[w][i];
        out[i] = s;
    }
}

__device__ __forceinline__ void block_max_store(double v, double *out) {
    __shared__ double red[RB_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = red[0];
        for (int w = 1; w < RB_THREADS / 32; ++w) s = fmax(s, red[w]);
        *out = s;
    }
}

// Sum partials[b * RB_STRIDE + i] over b < nb for i < cnt with the whole block:
// warp w handles outputs i = w, w + 8, ...; lane l adds blocks l, l + 32, ... in
// order, then a fixed shuffle tree combines the lanes (deterministic).  The result
// for output i is returned to lane 0 of its warp through out[i].
__device__ __forceinline__ void block_sum_partials(const double *__restrict__ partials, int nb, int cnt,
                                                   double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < cnt; i += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += partials[(long long)b * RB_STRIDE + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
}

// The same sums read through L2 only (__ldcg), for partials that other blocks of the
// running kernel have just written; four interleaved accumulators per lane keep
// four loads in flight (fixed order: deterministic).
__device__ __forceinline__ void block_sum_partials_l2(const double *partials, int nb, int cnt, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < cnt; i += nw) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = lane;
        for (; b + 96 < nb; b += 128) {
            s0 += __ldcg(&partials[(long long)b * RB_STRIDE + i]);
            s1 += __ldcg(&partials[(long long)(b + 32) * RB_STRIDE + i]);
            s2 += __ldcg(&partials[(long long)(b + 64) * RB_STRIDE + i]);
            s3 += __ldcg(&partials[(long long)(b + 96) * RB_STRIDE + i]);
        }
        for (; b < nb; b += 32) s0 += __ldcg(&partials[(long long)b * RB_STRIDE + i]);
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
}

// true in every thread of the block that is the last of the grid to arrive here
// (after storing its partial sums); that block then reads all partials.  The
// counter is reset by the last block, ready for the next launch.
__device__ __forceinline__ bool last_block_arrived(unsigned int *counter) {
    __shared__ int s_last;
    __threadfence();   // this block's partials are visible device-wide before it is counted
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int c = atomicAdd(counter, 1u) + 1u;
        s_last = c == gridDim.x;
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// chunk [lo, hi) of n elements owned by this block (contiguous)
__device__ __forceinline__ void block_chunk(long long n, long long &lo, long long &hi) {
    long long per = (n + gridDim.x - 1) / gridDim.x;
    per = (per + 1) & ~1LL;
    lo = per * blockIdx.x;
    hi = lo + per;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
}

}  // namespace llg
