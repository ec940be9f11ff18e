// gwam_offsets.cu -- per-cell segment offsets of a cell-sorted ray array (the parent-cell storage
// of App. B.2): offsets[c] = number of ray volumes with cell < c, offsets[ncell] = n.
#include "gwam_common.cuh"

namespace gwam {

// counts[c] += 1 for every ray volume in cell c; cells outside [0, ncell) raise flag
__global__ void k_cell_histogram(const int32_t* __restrict__ cells, int64_t n, int32_t ncell, int* __restrict__ counts,
                                 int* flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cells[i];
        if (c < 0 || c >= ncell) {
            atomicOr(flag, 1);
            continue;
        }
        atomicAdd(&counts[c], 1);
    }
}

int offsets_scratch_ints(int32_t ncell) { return scan_block_count(ncell) + 2; }

}  // namespace gwam

using namespace gwam;

extern "C" int gwam_cell_offsets(const int32_t* cells, int64_t n, int32_t ncell, int32_t* offsets, void* stream)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || ncell < 1 || ncell >= 0x7fffffff || !offsets || (n > 0 && !cells))
        return GWAM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nsc = offsets_scratch_ints(ncell);
    int* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, sizeof(int) * (size_t)nsc, s) != cudaSuccess) return GWAM_ENOMEM;
    int* flag = scratch + nsc - 1;
    int hflag = 0;
    int rc = GWAM_OK;
    if (cudaMemsetAsync(offsets, 0, sizeof(int32_t) * ((size_t)ncell + 1), s) != cudaSuccess ||
        cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) {
        rc = GWAM_ECUDA;
    } else {
        if (n > 0) {
            const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096);
            k_cell_histogram<<<blocks, kThreads, 0, s>>>(cells, n, ncell, offsets, flag);
        }
        scan_with_scratch(offsets, offsets, ncell, scratch, s);
        if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = GWAM_ECUDA;
    }
    cudaFreeAsync(scratch, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWAM_ECUDA;
    if (rc) return rc;
    return hflag ? GWAM_EINVAL : GWAM_OK;
}
