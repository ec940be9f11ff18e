// gwam_io.cu -- copies of device state into caller layouts (results, diagnostics, tests).
#include "gwam_common.cuh"
#include "gwam_fp32.cuh"

namespace gwam {

__global__ void k_gather_rays(Grid G, RaySoA A, const Ctl* ctl, double* __restrict__ out, long long* __restrict__ ids,
                              int* __restrict__ cells, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double s[NSTATE];
        long long id;
        load_ray(A, p, s, id);
        for (int q = 0; q < NSTATE; ++q) out[q * n + p] = s[q];
        ids[p] = id;
        cells[p] = member_of(id) * G.ncell + cell_of(G, s);
    }
}

void launch_gather_rays(Context& c, double* state13, long long* ids, int* cells, int64_t n)
{
    const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096);
    k_gather_rays<<<blocks, kThreads, 0, c.stream>>>(c.G, c.A, c.ctl, state13, ids, cells, n);
}

// column-major [member][col][nlev] -> [member][nlev][ny][nx]
__global__ void k_to_caller(Grid G, const double* __restrict__ src, double* __restrict__ dst, int nlev)
{
    const int64_t per = (int64_t)G.ncol * nlev;
    const int64_t total = per * G.members;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = t / per, r = t - m * per;
        const int64_t col = r % G.ncol;
        const int lev = (int)(r / G.ncol);
        dst[t] = src[m * per + col * nlev + lev];
    }
}

__global__ void k_gamma_to_caller(Grid G, const Node* __restrict__ bg, double* __restrict__ dst)
{
    const int64_t per = (int64_t)G.ncell;
    const int64_t total = per * G.members;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = t / per, r = t - m * per;
        const int64_t col = r % G.ncol;
        const int lev = (int)(r / G.ncol);
        dst[t] = bg[m * per + col * G.nz + lev].v[3];
    }
}

void launch_field_to_caller(Context& c, const double* src, double* dst, int nlev)
{
    const int64_t total = (int64_t)c.G.ncol_all * nlev;
    const int blocks = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, 8192);
    k_to_caller<<<blocks, kThreads, 0, c.stream>>>(c.G, src, dst, nlev);
}

void launch_gamma_to_caller(Context& c, double* dst)
{
    const int blocks = (int)std::min<int64_t>((c.G.ncell_all + kThreads - 1) / kThreads, 8192);
    k_gamma_to_caller<<<blocks, kThreads, 0, c.stream>>>(c.G, c.bg, dst);
}

__global__ void k_selftest_math(const double* __restrict__ x, int64_t n, double* __restrict__ r,
                                double* __restrict__ q)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        r[i] = rcp_nr(x[i]);
        q[i] = rsqrt_nr(x[i]);
    }
}

__global__ void k_selftest_widen(const float* __restrict__ x, int64_t n, double* __restrict__ w,
                                 double* __restrict__ prod)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        w[i] = widen(x[i]);
        if (prod) {
            // the double-float product chain of N Px Py Pz on (x_i, x_{i+1}, x_{i+2}, x_{i+3})
            S32 s{};
            s.n = x[i];
            s.p[0] = x[(i + 1) % n];
            s.p[1] = x[(i + 2) % n];
            s.p[2] = x[(i + 3) % n];
            prod[i] = df_to_double(action_df(s));
        }
    }
}

__global__ void k_selftest_narrow(const double* __restrict__ x, int64_t n, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = narrow(x[i]);
}

__global__ void k_selftest_split(const double* __restrict__ x, int64_t n, float* __restrict__ hi,
                                 float* __restrict__ lo)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const DF d = df_split(x[i]);
        hi[i] = d.hi;
        lo[i] = d.lo;
    }
}

__global__ void k_selftest_logratio(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                    double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df_to_double(df_log_ratio(a[i], b[i]));
}

}  // namespace gwam

extern "C" int gwam_selftest_logratio(const double* a, const double* b, int64_t n, double* out, void* stream)
{
    if (n < 0 || (n > 0 && (!a || !b || !out))) return GWAM_EINVAL;
    if (n == 0) return GWAM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + gwam::kThreads - 1) / gwam::kThreads, 4096);
    gwam::k_selftest_logratio<<<blocks, gwam::kThreads, 0, s>>>(a, b, n, out);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWAM_ECUDA;
    return GWAM_OK;
}

extern "C" int gwam_selftest_split(const double* x, int64_t n, float* hi, float* lo, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !hi || !lo))) return GWAM_EINVAL;
    if (n == 0) return GWAM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + gwam::kThreads - 1) / gwam::kThreads, 4096);
    gwam::k_selftest_split<<<blocks, gwam::kThreads, 0, s>>>(x, n, hi, lo);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWAM_ECUDA;
    return GWAM_OK;
}

extern "C" int gwam_selftest_narrow(const double* x, int64_t n, float* out, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !out))) return GWAM_EINVAL;
    if (n == 0) return GWAM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + gwam::kThreads - 1) / gwam::kThreads, 4096);
    gwam::k_selftest_narrow<<<blocks, gwam::kThreads, 0, s>>>(x, n, out);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWAM_ECUDA;
    return GWAM_OK;
}

extern "C" int gwam_selftest_widen(const float* x, int64_t n, double* widened, double* action, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !widened))) return GWAM_EINVAL;
    if (n == 0) return GWAM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + gwam::kThreads - 1) / gwam::kThreads, 4096);
    gwam::k_selftest_widen<<<blocks, gwam::kThreads, 0, s>>>(x, n, widened, action);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWAM_ECUDA;
    return GWAM_OK;
}

extern "C" int gwam_selftest_math(const double* x, int64_t n, double* rcp_out, double* rsqrt_out, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !rcp_out || !rsqrt_out))) return GWAM_EINVAL;
    if (n == 0) return GWAM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + gwam::kThreads - 1) / gwam::kThreads, 4096);
    gwam::k_selftest_math<<<blocks, gwam::kThreads, 0, s>>>(x, n, rcp_out, rsqrt_out);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWAM_ECUDA;
    return GWAM_OK;
}
