// gwam_offsets_noalloc.cu -- gwam_cell_offsets for callers that cannot allocate device memory.
//
// Some host models reserve all device memory up front for their own pool allocator, or run under a
// hard device-memory budget, and so must not call cudaMalloc (or anything that allocates) after
// start-up.  This entry point computes the same per-cell segment offsets as gwam_cell_offsets but
// keeps its scratch (the scan's block sums and an error flag) in a fixed array compiled into the
// library.  Every GPU that loads the library holds that array (about 32 KB) until the process exits.
#include <mutex>

#include "gwam_common.cuh"

namespace gwam {

// block sums of the scan (scan_block_count(ncell) + 1 ints) followed by one error flag
constexpr int kNoallocScratchInts = 8194;
static __device__ __align__(256) int g_noalloc_scratch[kNoallocScratchInts];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
int* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code only sees a host-side
// stand-in under the array's name, so the address is looked up once per device (with that device
// current) and remembered.
int* scratch_on_current_device(int* rc)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *rc = GWAM_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        int* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();   // the failed lookup is this call's error: leave none behind
            *rc = GWAM_ECUDA;
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace gwam

using namespace gwam;

extern "C" int gwam_cell_offsets_noalloc(const int32_t* cells, int64_t n, int32_t ncell, int32_t* offsets,
                                         void* stream)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || ncell < 1 || !offsets || (n > 0 && !cells)) return GWAM_EINVAL;
    if (ncell > GWAM_NOALLOC_MAX_CELLS || scan_block_count(ncell) + 2 > kNoallocScratchInts) return GWAM_ECAPACITY;
    int rc = GWAM_OK;
    int* scratch = scratch_on_current_device(&rc);
    if (!scratch) return rc;
    int* flag = scratch + kNoallocScratchInts - 1;
    cudaStream_t s = (cudaStream_t)stream;
    int hflag = 0;
    // the array keeps the previous call's contents: the flag must start at zero, the block sums
    // are written before they are read
    if (cudaMemsetAsync(offsets, 0, sizeof(int32_t) * ((size_t)ncell + 1), s) != cudaSuccess ||
        cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess)
        return GWAM_ECUDA;
    const cudaError_t e = launch_cell_offsets(cells, n, ncell, offsets, scratch, flag, s);
    if (e != cudaSuccess) {
        cudaGetLastError();       // clear this call's own launch error
        cudaStreamSynchronize(s);
        return GWAM_ECUDA;
    }
    if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GWAM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GWAM_ECUDA;
    return hflag ? GWAM_EINVAL : GWAM_OK;
}
