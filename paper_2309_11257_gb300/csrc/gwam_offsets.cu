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

__global__ void k_scan_reduce(const int* __restrict__ in, int64_t n, const int* n_dev, int* __restrict__ bsum);
__global__ void k_scan_blocks(int* bsum, int nb);
__global__ void k_scan_apply(const int* in, int* out, int64_t n, const int* n_dev, const int* __restrict__ bsum,
                             int nb);

// The histogram of the cells into counts (zeroed by the caller) and its exclusive scan in place,
// block sums in scratch (scan_block_count(ncell) + 1 ints), bad cells raising *flag.  Each launch
// returns its own status (cudaLaunchKernel), so an error that the caller's earlier work left
// pending is neither reported as this call's nor cleared by it.
cudaError_t launch_cell_offsets(const int32_t* cells, int64_t n, int32_t ncell, int* counts, int* scratch, int* flag,
                                cudaStream_t s)
{
    int64_t n64 = n, ncell64 = ncell;
    const int* no_dev = nullptr;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096);
        void* a[] = {(void*)&cells, (void*)&n64, (void*)&ncell, (void*)&counts, (void*)&flag};
        e = cudaLaunchKernel((const void*)k_cell_histogram, dim3(blocks), dim3(kThreads), a, 0, s);
    }
    const int nb = scan_block_count(ncell64);
    if (e == cudaSuccess) {
        void* a[] = {(void*)&counts, (void*)&ncell64, (void*)&no_dev, (void*)&scratch};
        e = cudaLaunchKernel((const void*)k_scan_reduce, dim3(nb), dim3(kThreads), a, 0, s);
    }
    if (e == cudaSuccess) {
        int nbv = nb;
        void* a[] = {(void*)&scratch, (void*)&nbv};
        e = cudaLaunchKernel((const void*)k_scan_blocks, dim3(1), dim3(1024), a, 0, s);
    }
    if (e == cudaSuccess) {
        int nbv = nb;
        const int* in = counts;
        const int* bs = scratch;
        void* a[] = {(void*)&in, (void*)&counts, (void*)&ncell64, (void*)&no_dev, (void*)&bs, (void*)&nbv};
        e = cudaLaunchKernel((const void*)k_scan_apply, dim3(nb), dim3(kThreads), a, 0, s);
    }
    return e;
}

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
    } else if (launch_cell_offsets(cells, n, ncell, offsets, scratch, flag, s) != cudaSuccess) {
        cudaGetLastError();   // clear this call's own launch error
        rc = GWAM_ECUDA;
    } else if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        rc = GWAM_ECUDA;
    }
    cudaFreeAsync(scratch, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GWAM_ECUDA;
    if (rc) return rc;
    return hflag ? GWAM_EINVAL : GWAM_OK;
}
