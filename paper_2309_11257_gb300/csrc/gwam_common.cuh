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

// The projected fields a step accumulates into, cleared by the step's ray-advance kernel instead
// of by a memset before the projection: that kernel is bound by instruction issue (FP64 form) or by
// its L1 gathers (precision form) and leaves HBM nearly idle, where the memsets were a pass over
// all the fields on the step's critical path.  Nothing reads or writes these fields between the
// advance and the projection.  The FP64 form clears with thread stores after its ray loop
// (clear_fields); the precision form's gathers would compete with such stores for L1, so there one
// thread per block issues bulk copies of a zeroed shared-memory buffer to the tensor-memory-access
// unit, a few per iteration of its ray loop (clear_start / clear_issue / clear_finish).
constexpr int kClearPiece = 16384;  // bytes per bulk copy (measured: 4 KB 0.698, 8 KB 0.607, 16 KB 0.572 ms)

struct ClearSet {
    double* p[NFIELD];
    int64_t n[NFIELD];             // elements of each field
    int64_t first[NFIELD + 1];     // first piece of each field; first[nf] = all pieces
    int nf;
};

// the fields the step's projection accumulates into (the two temperature fields only when projected)
inline ClearSet clear_set(const Context& c)
{
    ClearSet z{};
    z.nf = c.P.theta_flux ? NFIELD : F_TL;
    z.first[0] = 0;
    for (int f = 0; f < z.nf; ++f) {
        z.p[f] = c.field[f];
        z.n[f] = c.field_len(f);
        // pieces over the field's whole 16-byte part (an odd last element is stored separately)
        z.first[f + 1] = z.first[f] + ((z.n[f] >> 1) * 16 + kClearPiece - 1) / kClearPiece;
    }
    return z;
}

// All threads: grid-stride 16-byte streaming stores of zeros (fields start on 256-byte allocation
// boundaries; an odd last element is stored by thread 0).
__device__ __forceinline__ void clear_fields(const ClearSet& z)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int f = 0; f < z.nf; ++f) {
        double2* q = reinterpret_cast<double2*>(z.p[f]);
        const int64_t n2 = z.n[f] >> 1;
        for (int64_t i = t; i < n2; i += T) __stcs(q + i, make_double2(0.0, 0.0));
        if ((z.n[f] & 1) && t == 0) z.p[f][z.n[f] - 1] = 0.0;
    }
}

struct ClearState {
    int64_t g;         // next piece of this block (blocks take every gridDim.x-th piece)
    int per;           // pieces issued per ray-loop iteration
    uint32_t zbuf;     // shared-memory address of the zeroed buffer
};

// All threads of the block: zero the buffer, make it visible to the bulk-copy unit, and spread the
// block's pieces over the ray loop of thread 0 (n rays, grid-stride loop).
__device__ __forceinline__ void clear_start(const ClearSet& z, float4* zbuf, int n, ClearState& st)
{
    for (int q = threadIdx.x; q < kClearPiece / 16; q += blockDim.x) zbuf[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int64_t total = z.first[z.nf];
    st.g = blockIdx.x;
    st.zbuf = (uint32_t)__cvta_generic_to_shared(zbuf);
    const int64_t mine = st.g < total ? (total - 1 - st.g) / gridDim.x + 1 : 0;
    const int64_t b0 = (int64_t)blockIdx.x * blockDim.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = n > b0 ? (n - b0 + stride - 1) / stride : 0;
    st.per = iters > 0 ? (int)((mine + iters - 1) / iters) : 0;
}

// Thread 0: issue up to `count` of the block's pieces as one bulk group.
__device__ __forceinline__ void clear_issue(const ClearSet& z, ClearState& st, int count)
{
    const int64_t total = z.first[z.nf];
    int issued = 0;
    for (; issued < count && st.g < total; ++issued, st.g += gridDim.x) {
        int f = 0;
        while (f + 1 < z.nf && st.g >= z.first[f + 1]) ++f;
        const int64_t off = (st.g - z.first[f]) * kClearPiece;
        const int64_t bytes16 = (z.n[f] >> 1) * 16;
        const uint32_t bytes = (uint32_t)(bytes16 - off < kClearPiece ? bytes16 - off : kClearPiece);
        char* dst = reinterpret_cast<char*>(z.p[f]) + off;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                     :: "l"(dst), "r"(st.zbuf), "r"(bytes) : "memory");
    }
    if (issued) asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Thread 0 of every block: the rest of its pieces, then wait until all its copies are done (the
// shared buffer must outlive them); thread 0 of block 0 also clears the odd last elements.
__device__ __forceinline__ void clear_finish(const ClearSet& z, ClearState& st)
{
    if (threadIdx.x != 0) return;
    clear_issue(z, st, 0x7fffffff);
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (blockIdx.x == 0)
        for (int f = 0; f < z.nf; ++f)
            if (z.n[f] & 1) z.p[f][z.n[f] - 1] = 0.0;
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
