// gwam_common.cuh -- reductions and small helpers shared by the kernels.
#pragma once

#include "gwam_ctx.cuh"

namespace gwam {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum in a fixed order (deterministic); the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v)
{
    __shared__ T sh[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : T(0);
    if (wid == 0) r = warp_sum(r);
    return r;
}

// Segmented inclusive warp scan by key: after the call the last lane of every run of equal keys
// holds the run's total in v[]; returns true on that lane.  All 32 lanes must call it.
template <int NV>
__device__ __forceinline__ bool warp_segment_reduce(int key, double (&v)[NV])
{
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    // every lane its own run (the usual case once ray volumes spread): nothing to combine, and
    // no FP64 additions spent on it
    if (heads == 0xffffffffu) return true;
    const unsigned upto = heads & (0xffffffffu >> (31 - lane));
    const int start = 31 - __clz(upto);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double o = __shfl_up_sync(0xffffffffu, v[q], d);
            if (lane - d >= start) v[q] += o;
        }
    }
    return (lane == 31) || (next != key);
}

// True when this lane's run of equal keys touches neither lane 0 nor lane 31: with the ray array
// sorted by key and a warp holding 32 consecutive entries, no other warp holds that key, so the
// run's sum may be stored instead of added atomically (fewer L2 atomics, and deterministic).
__device__ __forceinline__ bool warp_run_interior(int key)
{
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    const unsigned tails = __ballot_sync(0xffffffffu, lane == 31 || next != key);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const int end = __ffs(tails & (0xffffffffu << lane)) - 1;
    return start > 0 && end < 31;
}

__device__ __forceinline__ void set_status(Ctl* ctl, int code)
{
    atomicCAS(&ctl->status, 0, code);
}

}  // namespace gwam
