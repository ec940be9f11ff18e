// gwam_mlp.cu -- the column drag surrogate: an MLP (n_in -> n_hidden x n_layers (GELU) -> n_out)
// trained and evaluated on the tensor cores (BF16 operands, FP32 accumulation) with the GEMM of
// gwam_gemm.cu.  Everything of a training step and of inference runs in the kernels below.
//
// Layout (B = rows of a batch, D_l = dimension l padded to a multiple of 64):
//   weights      W_l [D_l][D_{l-1}] FP32 master copy, Wb_l the BF16 copy (K-major operand of the
//                forward GEMM), WbT_l [D_{l-1}][D_l] BF16 (operand of the input-gradient GEMM);
//                Adam moments m, v FP32 like W; padding rows/columns stay zero.
//   activations  act_l [B][D_l] BF16 (l = 0 the normalised input), actT_l [D_l][B] BF16 (operand of
//                the weight-gradient GEMM), Z_l [B][D_l] FP32 pre-activations, dz_l / dzT_l the
//                BF16 gradients of Z_l in both layouts.
//   gradients    dW_l by split-K GEMM into FP32 partial slices, summed in a fixed order by the Adam
//                kernel (deterministic), db_l by row sums of dzT_l.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/gwam.h"
#include "gwam_gemm.cuh"

namespace {

constexpr int kMaxL = 8;

int pad64(int n) { return (n + 63) / 64 * 64; }

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    // SplitMix64 output function (Steele, Lea & Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t batch_row(const int32_t* rows, uint64_t seed, int64_t n, int r)
{
    if (rows) return rows[r];
    return (int64_t)(splitmix64(seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull) % (uint64_t)n);
}

// normalised, zero-padded input batch in both layouts: Xb [B][D0], XT [D0][ldT]
__global__ void k_batch_inputs(const float* __restrict__ X, int64_t n, int n_in, int D0, const int32_t* rows,
                               uint64_t seed, const float* __restrict__ mu, const float* __restrict__ isig,
                               __nv_bfloat16* Xb, __nv_bfloat16* XT, int ldT, int* err)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int f0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, f = f0 + tx;
        const int64_t src = batch_row(rows, seed, n, r);
        float xn = 0.0f;
        if (src < 0 || src >= n) {
            if (tx == 0) atomicOr(err, 2);
        } else if (f < n_in) {
            xn = (X[src * n_in + f] - mu[f]) * isig[f];
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(xn);
        if (f < D0) Xb[(size_t)r * D0 + f] = h;
        tile[rr][tx] = h;
    }
    __syncthreads();
    for (int ff = ty; ff < 32; ff += 8) {
        const int f = f0 + ff;
        if (f < D0) XT[(size_t)f * ldT + r0 + tx] = tile[tx][ff];
    }
}

// normalised, zero-padded targets T [B][Dn]
__global__ void k_batch_targets(const float* __restrict__ Y, int64_t n, int n_out, int Dn, int B, const int32_t* rows,
                                uint64_t seed, const float* __restrict__ mu, const float* __restrict__ isig,
                                float* T)
{
    const int r = blockIdx.x;
    if (r >= B) return;
    const int64_t src = batch_row(rows, seed, n, r);
    const bool okrow = src >= 0 && src < n;
    for (int o = threadIdx.x; o < Dn; o += blockDim.x)
        T[(size_t)r * Dn + o] = (o < n_out && okrow) ? (Y[src * n_out + o] - mu[o]) * isig[o] : 0.0f;
}

// db[o] = sum over the batch of dzT[o][r] (FP32 sum of BF16 values in a fixed order)
__global__ void k_rowsum(const __nv_bfloat16* __restrict__ dzT, int ld, int B, int D, float* db)
{
    const int o = blockIdx.x;
    if (o >= D) return;
    float s = 0.0f;
    for (int r = threadIdx.x; r < B; r += blockDim.x) s += __bfloat162float(dzT[(size_t)o * ld + r]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[o] = red[0];
}

// sum of the split-K partial slices (fixed order) -> g; Adam update of the master weights when
// lr > 0, refreshing the BF16 copies in both layouts.  Entries outside [n_o][n_i] stay zero.
__global__ void k_adam_weights(const float* __restrict__ part, int S, long long slice, int Do, int Di, int n_o,
                               int n_i, float* g, float* W, float* m, float* v, __nv_bfloat16* Wb,
                               __nv_bfloat16* WbT, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long total = (long long)Do * Di;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(idx / Di), i = (int)(idx - (long long)o * Di);
        float s = 0.0f;
        for (int k = 0; k < S; ++k) s += part[k * slice + idx];
        if (o >= n_o || i >= n_i) s = 0.0f;
        g[idx] = s;
        if (lr > 0.0f && o < n_o && i < n_i) {
            const float mm = b1 * m[idx] + (1.0f - b1) * s;
            const float vv = b2 * v[idx] + (1.0f - b2) * s * s;
            m[idx] = mm;
            v[idx] = vv;
            const float w = W[idx] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
            W[idx] = w;
            const __nv_bfloat16 h = __float2bfloat16_rn(w);
            Wb[idx] = h;
            WbT[(size_t)i * Do + o] = h;
        }
    }
}

__global__ void k_adam_bias(const float* __restrict__ gsrc, int D, int n_o, float* g, float* b, float* m, float* v,
                            float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= D) return;
    const float s = o < n_o ? gsrc[o] : 0.0f;
    g[o] = s;
    if (lr > 0.0f && o < n_o) {
        const float mm = b1 * m[o] + (1.0f - b1) * s;
        const float vv = b2 * v[o] + (1.0f - b2) * s * s;
        m[o] = mm;
        v[o] = vv;
        b[o] = b[o] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// inference input: one warp per column -- normalise, envelope test, BF16 row; mask = 1 (ray
// tracer) when a feature lies outside [lo, hi] or is not finite
__global__ void k_pack_infer(const float* __restrict__ X, int64_t ncol, int64_t c0, int rows, int n_in, int D0,
                             const float* __restrict__ mu, const float* __restrict__ isig,
                             const float* __restrict__ lo, const float* __restrict__ hi, __nv_bfloat16* Xb,
                             int32_t* mask, int32_t* nfb)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const int64_t c = c0 + warp;
    bool out = false;
    const float* x = X + c * n_in;
    __nv_bfloat16* xb = Xb + (size_t)warp * D0;
    // four features per lane and pass (16-byte loads, 8-byte stores) when the rows allow it
    const bool vec = (n_in % 4 == 0) && (D0 % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0);
    if (vec) {
        for (int f = 4 * lane; f < D0; f += 128) {
            float4 xn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (f < n_in) {
                const float4 v = *reinterpret_cast<const float4*>(x + f);
                const float4 m = *reinterpret_cast<const float4*>(mu + f);
                const float4 is = *reinterpret_cast<const float4*>(isig + f);
                const float4 l = *reinterpret_cast<const float4*>(lo + f);
                const float4 h = *reinterpret_cast<const float4*>(hi + f);
                xn = make_float4((v.x - m.x) * is.x, (v.y - m.y) * is.y, (v.z - m.z) * is.z, (v.w - m.w) * is.w);
                out |= !(xn.x >= l.x && xn.x <= h.x) || !(xn.y >= l.y && xn.y <= h.y) ||
                       !(xn.z >= l.z && xn.z <= h.z) || !(xn.w >= l.w && xn.w <= h.w);
            }
            __nv_bfloat162 p0 = __floats2bfloat162_rn(xn.x, xn.y), p1 = __floats2bfloat162_rn(xn.z, xn.w);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&p0);
            pk.y = *reinterpret_cast<uint32_t*>(&p1);
            *reinterpret_cast<uint2*>(xb + f) = pk;
        }
    } else {
        for (int f = lane; f < D0; f += 32) {
            float xn = 0.0f;
            if (f < n_in) {
                xn = (x[f] - mu[f]) * isig[f];
                out |= !(xn >= lo[f] && xn <= hi[f]);
            }
            xb[f] = __float2bfloat16_rn(xn);
        }
    }
    out = __any_sync(0xffffffffu, out);
    if (lane == 0) {
        mask[c] = out ? 1 : 0;
        if (out) atomicAdd(nfb, 1);
    }
}

// fallback columns take the ray tracer's drag
__global__ void k_merge(const int32_t* __restrict__ mask, int64_t ncol, const double* __restrict__ du_t,
                        const double* __restrict__ dv_t, double* du, double* dv)
{
    const int k = blockIdx.y;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncol; c += (int64_t)gridDim.x * blockDim.x) {
        if (mask[c]) {
            const size_t i = (size_t)k * ncol + c;
            du[i] = du_t[i];
            dv[i] = dv_t[i];
        }
    }
}

// per-column statistics of a row-major [n][nf] FP32 array: mean, population std, min, max (FP64 sums)
__global__ void k_colstats(const float* __restrict__ X, int64_t n, int nf, double* out4)
{
    const int f = blockIdx.x;
    double s = 0.0, q = 0.0, mn = INFINITY, mx = -INFINITY;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double x = X[r * nf + f];
        s += x;
        q += x * x;
        mn = fmin(mn, x);
        mx = fmax(mx, x);
    }
    __shared__ double red[4][256];
    red[0][threadIdx.x] = s;
    red[1][threadIdx.x] = q;
    red[2][threadIdx.x] = mn;
    red[3][threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
            red[2][threadIdx.x] = fmin(red[2][threadIdx.x], red[2][threadIdx.x + w]);
            red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = red[0][0] / (double)n;
        const double var = fmax(red[1][0] / (double)n - mean * mean, 0.0);
        out4[4 * f + 0] = mean;
        out4[4 * f + 1] = sqrt(var);
        out4[4 * f + 2] = red[2][0];
        out4[4 * f + 3] = red[3][0];
    }
}

// column features from a gridded background ([nz][ncol] FP64 fields): u, v, N^2, ln rho on every
// level, then n_src source parameters (per column with stride n_src, or shared when src_stride = 0)
__global__ void k_features(const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ n2,
                           const double* __restrict__ rho, int nz, int64_t ncol, const float* __restrict__ src,
                           int n_src, int src_stride, float* X)
{
    const int nf = 4 * nz + n_src;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < ncol * nf;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx / nf;
        const int f = (int)(idx - c * nf);
        float x;
        if (f < 4 * nz) {
            const int q = f / nz, k = f - q * nz;
            const size_t g = (size_t)k * ncol + c;
            x = q == 0 ? (float)u[g] : q == 1 ? (float)v[g] : q == 2 ? (float)n2[g] : (float)log(rho[g]);
        } else {
            x = src[c * src_stride + (f - 4 * nz)];
        }
        X[idx] = x;
    }
}

// drag targets [ncol][2 nz] FP32 = scale * (du, dv) from [nz][ncol] FP64 sums
__global__ void k_targets(const double* __restrict__ du, const double* __restrict__ dv, int nz, int64_t ncol,
                          double scale, float* Y)
{
    const int nf = 2 * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < ncol * nf;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx / nf;
        const int f = (int)(idx - c * nf);
        const size_t g = (size_t)(f < nz ? f : f - nz) * ncol + c;
        Y[idx] = (float)(scale * (f < nz ? du[g] : dv[g]));
    }
}

}  // namespace

struct gwam_mlp {
    int dev = 0;
    cudaStream_t s = nullptr;
    int nl = 0;                         // number of weight layers
    int N[kMaxL + 1] = {}, D[kMaxL + 1] = {};
    int nlev = 0, max_batch = 0;
    float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    long long t = 0;
    float *W[kMaxL + 1] = {}, *b[kMaxL + 1] = {}, *mW[kMaxL + 1] = {}, *vW[kMaxL + 1] = {}, *mb[kMaxL + 1] = {},
          *vb[kMaxL + 1] = {}, *gW[kMaxL + 1] = {}, *gb[kMaxL + 1] = {}, *db_raw[kMaxL + 1] = {};
    __nv_bfloat16 *Wb[kMaxL + 1] = {}, *WbT[kMaxL + 1] = {};
    __nv_bfloat16 *act[kMaxL + 1] = {}, *actT[kMaxL + 1] = {}, *dz[kMaxL + 1] = {}, *dzT[kMaxL + 1] = {};
    float* Z[kMaxL + 1] = {};
    float *Y = nullptr, *T = nullptr, *partial = nullptr;
    size_t partial_elems = 0;
    float *xmu = nullptr, *xisig = nullptr, *ymu = nullptr, *yisig = nullptr, *ysig = nullptr, *lo = nullptr,
          *hi = nullptr;
    int* err = nullptr;
    double* loss = nullptr;
    int32_t* nfb = nullptr;
    bool has_norm = false;
    int last_batch = 0;
    CUtensorMap tf_a[kMaxL + 1], tf_b[kMaxL + 1], tx_a[kMaxL + 1], tx_b[kMaxL + 1], tw_a[kMaxL + 1], tw_b[kMaxL + 1];
    CUtensorMap to_act[kMaxL + 1], to_dz[kMaxL + 1];   // BF16 outputs written by TMA stores
    int bn_f[kMaxL + 1] = {}, bn_x[kMaxL + 1] = {}, bn_w[kMaxL + 1] = {};
    std::vector<void*> allocs;
    std::string last_error;
    // inference timing: events before the pack kernel, before the first GEMM, after the last GEMM
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;
    size_t prof_used = 0;
    double prof_ms[2] = {0.0, 0.0};
    long long prof_passes = 0;
};

namespace {

void prof_harvest(gwam_mlp* m)
{
    if (m->prof_used == 0) return;
    cudaEventSynchronize(m->prof_ev[m->prof_used - 1]);
    for (size_t i = 0; i + 3 <= m->prof_used; i += 3) {
        float a = 0.0f, b = 0.0f;
        cudaEventElapsedTime(&a, m->prof_ev[i], m->prof_ev[i + 1]);
        cudaEventElapsedTime(&b, m->prof_ev[i + 1], m->prof_ev[i + 2]);
        m->prof_ms[0] += a;
        m->prof_ms[1] += b;
        ++m->prof_passes;
    }
    m->prof_used = 0;
}

cudaEvent_t prof_mark(gwam_mlp* m)
{
    if (m->prof_used == m->prof_ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        m->prof_ev.push_back(e);
    }
    cudaEvent_t e = m->prof_ev[m->prof_used++];
    cudaEventRecord(e, m->s);
    return e;
}

int fail(gwam_mlp* m, int code, const char* what)
{
    if (m) m->last_error = what;
    return code;
}

template <class T>
bool dalloc(gwam_mlp* m, T** p, size_t elems)
{
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(elems, 1) * sizeof(T)) != cudaSuccess) return false;
    cudaMemsetAsync(q, 0, std::max<size_t>(elems, 1) * sizeof(T), m->s);
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

// split-K factor of the weight-gradient GEMM of layer l for a batch of B rows
int wgrad_split(const gwam_mlp* m, int l, int B)
{
    const int kb = B / 64;
    const int tiles = ((m->D[l] + 127) / 128) * ((m->D[l - 1] + m->bn_w[l] - 1) / m->bn_w[l]);
    int S = 1;
    while (S * 2 <= 64 && kb % (S * 2) == 0 && tiles * S * 2 <= 2 * 152) S *= 2;
    return S;
}

uint64_t host_splitmix(uint64_t& state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void refresh_bf16(gwam_mlp* m, int l, const std::vector<float>& Wp)
{
    const int Do = m->D[l], Di = m->D[l - 1];
    std::vector<__nv_bfloat16> wb((size_t)Do * Di), wt((size_t)Do * Di);
    for (int o = 0; o < Do; ++o)
        for (int i = 0; i < Di; ++i) {
            const __nv_bfloat16 h = __float2bfloat16_rn(Wp[(size_t)o * Di + i]);
            wb[(size_t)o * Di + i] = h;
            wt[(size_t)i * Do + o] = h;
        }
    cudaMemcpyAsync(m->Wb[l], wb.data(), wb.size() * 2, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->WbT[l], wt.data(), wt.size() * 2, cudaMemcpyHostToDevice, m->s);
    cudaStreamSynchronize(m->s);
}

int check_err(gwam_mlp* m)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->s) != cudaSuccess ||
        cudaStreamSynchronize(m->s) != cudaSuccess)
        return fail(m, GWAM_ECUDA, cudaGetErrorString(cudaGetLastError()));
    if (h & 1) return fail(m, GWAM_ETIMEOUT, "a bounded wait in the tensor-core GEMM gave up");
    if (h & 2) return fail(m, GWAM_EINVAL, "a batch row index lies outside the data set");
    return GWAM_OK;
}

bool gemm(gwam_mlp* m, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap* tc, int K, int bn, int ks,
          gwam::GemmEpi e)
{
    e.err = m->err;
    return gwam::gemm_bf16_launch(ta, tb, tc, K, bn, ks, e, m->s);
}

// forward through every layer for B rows of act[0]; last layer per `last`
bool forward(gwam_mlp* m, int B, bool train, const gwam::GemmEpi& last)
{
    for (int l = 1; l < m->nl; ++l) {
        gwam::GemmEpi e{};
        e.mode = gwam::EPI_STORE;
        e.act = 1;
        e.M = B;
        e.N = m->D[l];
        e.bias = m->b[l];
        e.cb = m->act[l];
        e.ldcb = m->D[l];
        if (train) {
            e.z = m->Z[l];
            e.ldz = m->D[l];
            e.ct = m->actT[l];
            e.ldct = m->max_batch;
        }
        if (!gemm(m, m->tf_a[l], m->tf_b[l], &m->to_act[l], m->D[l - 1], m->bn_f[l], 1, e)) return false;
    }
    gwam::GemmEpi e = last;
    e.M = B;
    e.N = m->D[m->nl];
    e.bias = m->b[m->nl];
    return gemm(m, m->tf_a[m->nl], m->tf_b[m->nl], e.cb ? &m->to_dz[m->nl] : nullptr, m->D[m->nl - 1],
                m->bn_f[m->nl], 1, e);
}

}  // namespace

extern "C" {

int gwam_mlp_create(gwam_mlp** out, const gwam_mlp_config* cfg, void* stream)
{
    if (!out || !cfg) return GWAM_EINVAL;
    *out = nullptr;
    if (cfg->n_in < 1 || cfg->n_in > 8192 || cfg->n_out < 1 || cfg->n_out > 8192 || cfg->n_hidden < 64 ||
        cfg->n_hidden > 4096 || cfg->n_hidden % 64 || cfg->n_layers < 1 || cfg->n_layers > kMaxL - 1 ||
        cfg->max_batch < 128 || cfg->max_batch % 128 || cfg->max_batch > (1 << 20) || cfg->nlev < 0 ||
        2 * cfg->nlev > cfg->n_out || !(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) ||
        !(cfg->eps > 0))
        return GWAM_EINVAL;
    gwam_mlp* m = new gwam_mlp();
    cudaGetDevice(&m->dev);
    m->s = (cudaStream_t)stream;
    m->nl = cfg->n_layers + 1;
    m->N[0] = cfg->n_in;
    for (int l = 1; l < m->nl; ++l) m->N[l] = cfg->n_hidden;
    m->N[m->nl] = cfg->n_out;
    for (int l = 0; l <= m->nl; ++l) m->D[l] = pad64(m->N[l]);
    m->nlev = cfg->nlev;
    m->max_batch = cfg->max_batch;
    m->b1 = cfg->beta1;
    m->b2 = cfg->beta2;
    m->eps = cfg->eps;
    const int Bm = m->max_batch;
    bool ok = true;
    for (int l = 1; l <= m->nl && ok; ++l) {
        m->bn_f[l] = gwam::gemm_pick_bn(Bm, m->D[l]);
        m->bn_x[l] = gwam::gemm_pick_bn(Bm, m->D[l - 1]);
        m->bn_w[l] = gwam::gemm_pick_bn(m->D[l], m->D[l - 1]);
        const size_t nw = (size_t)m->D[l] * m->D[l - 1];
        ok = ok && dalloc(m, &m->W[l], nw) && dalloc(m, &m->mW[l], nw) && dalloc(m, &m->vW[l], nw) &&
             dalloc(m, &m->gW[l], nw) && dalloc(m, &m->Wb[l], nw) && dalloc(m, &m->WbT[l], nw) &&
             dalloc(m, &m->b[l], m->D[l]) && dalloc(m, &m->mb[l], m->D[l]) && dalloc(m, &m->vb[l], m->D[l]) &&
             dalloc(m, &m->gb[l], m->D[l]) && dalloc(m, &m->db_raw[l], m->D[l]) &&
             dalloc(m, &m->dz[l], (size_t)Bm * m->D[l]) && dalloc(m, &m->dzT[l], (size_t)Bm * m->D[l]);
        const int Smax = 64;
        m->partial_elems = std::max(m->partial_elems, (size_t)Smax * nw);
    }
    for (int l = 0; l < m->nl && ok; ++l) {
        ok = ok && dalloc(m, &m->act[l], (size_t)Bm * m->D[l]) && dalloc(m, &m->actT[l], (size_t)Bm * m->D[l]);
        if (l > 0) ok = ok && dalloc(m, &m->Z[l], (size_t)Bm * m->D[l]);
    }
    const int Dn = m->D[m->nl];
    ok = ok && dalloc(m, &m->Y, (size_t)Bm * Dn) && dalloc(m, &m->T, (size_t)Bm * Dn) &&
         dalloc(m, &m->partial, m->partial_elems) && dalloc(m, &m->xmu, m->D[0]) && dalloc(m, &m->xisig, m->D[0]) &&
         dalloc(m, &m->lo, m->D[0]) && dalloc(m, &m->hi, m->D[0]) && dalloc(m, &m->ymu, Dn) &&
         dalloc(m, &m->yisig, Dn) && dalloc(m, &m->ysig, Dn) && dalloc(m, &m->err, 1) && dalloc(m, &m->loss, 1) &&
         dalloc(m, &m->nfb, 1);
    if (!ok) {
        gwam_mlp_destroy(m);
        return GWAM_ENOMEM;
    }
    // tensor maps of every GEMM operand (fixed buffers)
    for (int l = 1; l <= m->nl && ok; ++l) {
        const int Di = m->D[l - 1], Do = m->D[l];
        ok = ok && gwam::make_tmap_bf16(&m->tf_a[l], m->act[l - 1], Bm, Di, Di, 128) &&
             gwam::make_tmap_bf16(&m->tf_b[l], m->Wb[l], Do, Di, Di, m->bn_f[l]) &&
             gwam::make_tmap_bf16(&m->tx_a[l], m->dz[l], Bm, Do, Do, 128) &&
             gwam::make_tmap_bf16(&m->tx_b[l], m->WbT[l], Di, Do, Do, m->bn_x[l]) &&
             gwam::make_tmap_bf16(&m->tw_a[l], m->dzT[l], Do, Bm, Bm, 128) &&
             gwam::make_tmap_bf16(&m->tw_b[l], m->actT[l - 1], Di, Bm, Bm, m->bn_w[l]) &&
             gwam::make_tmap_bf16(&m->to_dz[l], m->dz[l], Bm, Do, Do, 32) &&
             (l == m->nl || gwam::make_tmap_bf16(&m->to_act[l], m->act[l], Bm, Do, Do, 32));
    }
    if (!ok) {
        gwam_mlp_destroy(m);
        return GWAM_ECUDA;
    }
    // seeded initial weights W ~ N(0, 1/n_in) (SplitMix64 + Box-Muller), b = 0
    uint64_t st = cfg->seed;
    for (int l = 1; l <= m->nl; ++l) {
        const int Do = m->D[l], Di = m->D[l - 1];
        std::vector<float> Wp((size_t)Do * Di, 0.0f);
        const double sd = 1.0 / std::sqrt((double)m->N[l - 1]);
        for (int o = 0; o < m->N[l]; ++o)
            for (int i = 0; i < m->N[l - 1]; ++i) {
                const double u1 = ((host_splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
                const double u2 = (host_splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
                Wp[(size_t)o * Di + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
            }
        cudaMemcpyAsync(m->W[l], Wp.data(), Wp.size() * 4, cudaMemcpyHostToDevice, m->s);
        refresh_bf16(m, l, Wp);
    }
    if (cudaStreamSynchronize(m->s) != cudaSuccess) {
        gwam_mlp_destroy(m);
        return GWAM_ECUDA;
    }
    *out = m;
    return GWAM_OK;
}

void gwam_mlp_destroy(gwam_mlp* m)
{
    if (!m) return;
    if (m->s) cudaStreamSynchronize(m->s);
    for (void* p : m->allocs) cudaFree(p);
    for (cudaEvent_t e : m->prof_ev) cudaEventDestroy(e);
    delete m;
}

const char* gwam_mlp_last_error(const gwam_mlp* m) { return m ? m->last_error.c_str() : "null surrogate"; }

int gwam_mlp_set_normalization_host(gwam_mlp* m, const float* x_mu, const float* x_sigma, const float* y_mu,
                                    const float* y_sigma, const float* lo, const float* hi)
{
    if (!m || !x_mu || !x_sigma || !y_mu || !y_sigma || !lo || !hi) return fail(m, GWAM_EINVAL, "null pointer");
    const int ni = m->N[0], no = m->N[m->nl];
    std::vector<float> xi(ni), yi(no);
    for (int f = 0; f < ni; ++f) {
        if (!(x_sigma[f] > 0) || !std::isfinite(x_mu[f]) || !std::isfinite(x_sigma[f]))
            return fail(m, GWAM_EINVAL, "feature sigma must be positive and finite");
        xi[f] = 1.0f / x_sigma[f];
    }
    for (int o = 0; o < no; ++o) {
        if (!(y_sigma[o] > 0) || !std::isfinite(y_mu[o]) || !std::isfinite(y_sigma[o]))
            return fail(m, GWAM_EINVAL, "target sigma must be positive and finite");
        yi[o] = 1.0f / y_sigma[o];
    }
    cudaMemcpyAsync(m->xmu, x_mu, ni * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->xisig, xi.data(), ni * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->lo, lo, ni * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->hi, hi, ni * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->ymu, y_mu, no * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->ysig, y_sigma, no * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->yisig, yi.data(), no * 4, cudaMemcpyHostToDevice, m->s);
    if (cudaStreamSynchronize(m->s) != cudaSuccess) return fail(m, GWAM_ECUDA, "copy failed");
    m->has_norm = true;
    return GWAM_OK;
}

int gwam_mlp_fit_normalization(gwam_mlp* m, const float* X, const float* Y, int64_t n, float margin,
                               float* stats_host)
{
    if (!m || !X || !Y || n < 2 || !(margin >= 0)) return fail(m, GWAM_EINVAL, "bad arguments");
    const int ni = m->N[0], no = m->N[m->nl];
    double* d = nullptr;
    if (cudaMallocAsync((void**)&d, (size_t)4 * (ni + no) * sizeof(double), m->s) != cudaSuccess)
        return fail(m, GWAM_ENOMEM, "scratch");
    k_colstats<<<ni, 256, 0, m->s>>>(X, n, ni, d);
    k_colstats<<<no, 256, 0, m->s>>>(Y, n, no, d + 4 * ni);
    std::vector<double> h((size_t)4 * (ni + no));
    cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, m->s);
    cudaFreeAsync(d, m->s);
    if (cudaStreamSynchronize(m->s) != cudaSuccess) return fail(m, GWAM_ECUDA, "statistics failed");
    std::vector<float> xm(ni), xs(ni), lo(ni), hi(ni), ym(no), ys(no);
    for (int f = 0; f < ni; ++f) {
        const double mu = h[4 * f], sd = h[4 * f + 1] > 0 ? h[4 * f + 1] : 1.0;
        xm[f] = (float)mu;
        xs[f] = (float)sd;
        const double a = (h[4 * f + 2] - mu) / sd, b = (h[4 * f + 3] - mu) / sd, w = b - a;
        lo[f] = (float)(a - margin * w);
        hi[f] = (float)(b + margin * w);
    }
    // targets: per-output mean, one shared scale = the RMS of the per-output standard deviations,
    // so the loss is proportional to the squared error of the drag itself (every level weighted by
    // its physical size; an output that is always zero is not amplified)
    double s2 = 0.0;
    for (int o = 0; o < no; ++o) s2 += h[4 * (ni + o) + 1] * h[4 * (ni + o) + 1];
    const double scale = s2 > 0 ? std::sqrt(s2 / no) : 1.0;
    for (int o = 0; o < no; ++o) {
        ym[o] = (float)h[4 * (ni + o)];
        ys[o] = (float)scale;
    }
    if (stats_host) {
        // mu, sigma, lo, hi of the features, then mu, sigma of the targets
        std::copy(xm.begin(), xm.end(), stats_host);
        std::copy(xs.begin(), xs.end(), stats_host + ni);
        std::copy(lo.begin(), lo.end(), stats_host + 2 * ni);
        std::copy(hi.begin(), hi.end(), stats_host + 3 * ni);
        std::copy(ym.begin(), ym.end(), stats_host + 4 * ni);
        std::copy(ys.begin(), ys.end(), stats_host + 4 * ni + no);
    }
    return gwam_mlp_set_normalization_host(m, xm.data(), xs.data(), ym.data(), ys.data(), lo.data(), hi.data());
}

int gwam_mlp_set_params_host(gwam_mlp* m, int layer, const float* W, const float* b)
{
    if (!m || layer < 1 || layer > m->nl || !W || !b) return fail(m, GWAM_EINVAL, "bad layer or null pointer");
    const int Do = m->D[layer], Di = m->D[layer - 1], no = m->N[layer], ni = m->N[layer - 1];
    std::vector<float> Wp((size_t)Do * Di, 0.0f), bp(Do, 0.0f);
    for (int o = 0; o < no; ++o) {
        for (int i = 0; i < ni; ++i) Wp[(size_t)o * Di + i] = W[(size_t)o * ni + i];
        bp[o] = b[o];
    }
    cudaMemcpyAsync(m->W[layer], Wp.data(), Wp.size() * 4, cudaMemcpyHostToDevice, m->s);
    cudaMemcpyAsync(m->b[layer], bp.data(), bp.size() * 4, cudaMemcpyHostToDevice, m->s);
    refresh_bf16(m, layer, Wp);
    return cudaStreamSynchronize(m->s) == cudaSuccess ? GWAM_OK : fail(m, GWAM_ECUDA, "copy failed");
}

int gwam_mlp_get_params_host(gwam_mlp* m, int layer, int which, float* W, float* b)
{
    // which: 0 master weights, 1 gradients of the last train step
    if (!m || layer < 1 || layer > m->nl || (which != 0 && which != 1)) return fail(m, GWAM_EINVAL, "bad arguments");
    const int Do = m->D[layer], Di = m->D[layer - 1], no = m->N[layer], ni = m->N[layer - 1];
    std::vector<float> Wp((size_t)Do * Di), bp(Do);
    cudaMemcpyAsync(Wp.data(), which ? m->gW[layer] : m->W[layer], Wp.size() * 4, cudaMemcpyDeviceToHost, m->s);
    cudaMemcpyAsync(bp.data(), which ? m->gb[layer] : m->b[layer], bp.size() * 4, cudaMemcpyDeviceToHost, m->s);
    if (cudaStreamSynchronize(m->s) != cudaSuccess) return fail(m, GWAM_ECUDA, "copy failed");
    for (int o = 0; o < no; ++o) {
        if (W)
            for (int i = 0; i < ni; ++i) W[(size_t)o * ni + i] = Wp[(size_t)o * Di + i];
        if (b) b[o] = bp[o];
    }
    return GWAM_OK;
}

int gwam_mlp_train_step(gwam_mlp* m, const float* X, const float* Y, int64_t n, const int32_t* rows, int batch,
                        uint64_t seed, float lr)
{
    if (!m || !X || !Y || n < 1 || batch < 64 || batch % 64 || batch > m->max_batch || !(lr >= 0))
        return fail(m, GWAM_EINVAL, "bad arguments (batch must be a multiple of 64 up to max_batch)");
    if (!m->has_norm) return fail(m, GWAM_ESTATE, "normalisation not set");
    const int B = batch, L = m->nl, Dn = m->D[L];
    cudaMemsetAsync(m->loss, 0, sizeof(double), m->s);
    cudaMemsetAsync(m->err, 0, sizeof(int), m->s);
    k_batch_inputs<<<dim3((m->D[0] + 31) / 32, B / 32), dim3(32, 8), 0, m->s>>>(
        X, n, m->N[0], m->D[0], rows, seed, m->xmu, m->xisig, m->act[0], m->actT[0], m->max_batch, m->err);
    k_batch_targets<<<B, 128, 0, m->s>>>(Y, n, m->N[L], Dn, B, rows, seed, m->ymu, m->yisig, m->T);
    gwam::GemmEpi last{};
    last.mode = gwam::EPI_LOSS;
    last.cf = m->Y;
    last.ldcf = Dn;
    last.tgt = m->T;
    last.ldt = Dn;
    last.n_true = m->N[L];
    last.gscale = 2.0f / ((float)B * (float)m->N[L]);
    last.loss = m->loss;
    last.cb = m->dz[L];
    last.ldcb = Dn;
    last.ct = m->dzT[L];
    last.ldct = m->max_batch;
    bool ok = forward(m, B, true, last);
    for (int l = L; l >= 1 && ok; --l) {
        // weight gradient: dW_l = dz_l^T act_{l-1} (split-K partial slices)
        const int S = wgrad_split(m, l, B);
        gwam::GemmEpi e{};
        e.mode = gwam::EPI_STORE;
        e.M = m->D[l];
        e.N = m->D[l - 1];
        e.cf = m->partial;
        e.ldcf = m->D[l - 1];
        e.cf_slice = (long long)m->D[l] * m->D[l - 1];
        ok = gemm(m, m->tw_a[l], m->tw_b[l], nullptr, B, m->bn_w[l], S, e);
        k_rowsum<<<m->D[l], 256, 0, m->s>>>(m->dzT[l], m->max_batch, B, m->D[l], m->db_raw[l]);
        // input gradient of the layer below, times GELU'(Z_{l-1})
        if (l > 1 && ok) {
            gwam::GemmEpi x{};
            x.mode = gwam::EPI_BWD;
            x.M = B;
            x.N = m->D[l - 1];
            x.z = m->Z[l - 1];
            x.ldz = m->D[l - 1];
            x.cb = m->dz[l - 1];
            x.ldcb = m->D[l - 1];
            x.ct = m->dzT[l - 1];
            x.ldct = m->max_batch;
            ok = gemm(m, m->tx_a[l], m->tx_b[l], &m->to_dz[l - 1], m->D[l], m->bn_x[l], 1, x);
        }
        // Adam (or gradients only when lr = 0)
        if (ok) {
            const long long t = lr > 0 ? m->t + 1 : std::max(1ll, m->t);
            const float c1 = (float)(1.0 - std::pow((double)m->b1, (double)t));
            const float c2 = (float)(1.0 - std::pow((double)m->b2, (double)t));
            const long long nw = (long long)m->D[l] * m->D[l - 1];
            const int blocks = (int)std::min<long long>((nw + 255) / 256, 4 * 152);
            k_adam_weights<<<blocks, 256, 0, m->s>>>(m->partial, S, nw, m->D[l], m->D[l - 1], m->N[l], m->N[l - 1],
                                                     m->gW[l], m->W[l], m->mW[l], m->vW[l], m->Wb[l], m->WbT[l], lr,
                                                     m->b1, m->b2, m->eps, c1, c2);
            k_adam_bias<<<(m->D[l] + 127) / 128, 128, 0, m->s>>>(m->db_raw[l], m->D[l], m->N[l], m->gb[l], m->b[l],
                                                                 m->mb[l], m->vb[l], lr, m->b1, m->b2, m->eps, c1, c2);
        }
    }
    if (!ok || cudaPeekAtLastError() != cudaSuccess) return fail(m, GWAM_ECUDA, "kernel launch failed");
    if (lr > 0) ++m->t;
    m->last_batch = B;
    return GWAM_OK;
}

int gwam_mlp_last_loss_host(gwam_mlp* m, double* loss)
{
    if (!m || !loss) return fail(m, GWAM_EINVAL, "null pointer");
    double h = 0;
    cudaMemcpyAsync(&h, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->s);
    const int rc = check_err(m);
    if (rc != GWAM_OK) return rc;
    *loss = m->last_batch ? h / ((double)m->last_batch * m->N[m->nl]) : 0.0;
    return GWAM_OK;
}

int gwam_mlp_output_host(gwam_mlp* m, float* Yout, int rows)
{
    if (!m || !Yout || rows < 0 || rows > m->last_batch) return fail(m, GWAM_EINVAL, "bad arguments");
    const int Dn = m->D[m->nl], no = m->N[m->nl];
    std::vector<float> h((size_t)rows * Dn);
    cudaMemcpyAsync(h.data(), m->Y, h.size() * 4, cudaMemcpyDeviceToHost, m->s);
    const int rc = check_err(m);
    if (rc != GWAM_OK) return rc;
    for (int r = 0; r < rows; ++r)
        for (int o = 0; o < no; ++o) Yout[(size_t)r * no + o] = h[(size_t)r * Dn + o];
    return GWAM_OK;
}

int gwam_mlp_infer(gwam_mlp* m, const float* X, int64_t ncol, double* dudt, double* dvdt, int32_t* fallback_mask,
                   int32_t* n_fallback)
{
    if (!m || !X || ncol < 1 || ncol > INT32_MAX || !dudt || !dvdt || !fallback_mask || !n_fallback ||
        m->nlev < 1 || 2 * m->nlev != m->N[m->nl])
        return fail(m, GWAM_EINVAL, "bad arguments (the output must be du/dt and dv/dt on nlev levels)");
    if (!m->has_norm) return fail(m, GWAM_ESTATE, "normalisation not set");
    cudaMemsetAsync(n_fallback, 0, sizeof(int32_t), m->s);
    for (int64_t c0 = 0; c0 < ncol; c0 += m->max_batch) {
        const int rows = (int)std::min<int64_t>(m->max_batch, ncol - c0);
        if (m->prof && m->prof_used + 3 > 3 * 64) prof_harvest(m);
        if (m->prof) prof_mark(m);
        k_pack_infer<<<(rows + 7) / 8, 256, 0, m->s>>>(X, ncol, c0, rows, m->N[0], m->D[0], m->xmu, m->xisig, m->lo,
                                                      m->hi, m->act[0], fallback_mask, n_fallback);
        gwam::GemmEpi last{};
        last.mode = gwam::EPI_DRAG;
        last.n_true = m->N[m->nl];
        last.ysig = m->ysig;
        last.ymu = m->ymu;
        last.mask = fallback_mask + c0;
        last.du = dudt + c0;
        last.dv = dvdt + c0;
        last.ncol = (int)ncol;
        last.nlev = m->nlev;
        if (m->prof) prof_mark(m);
        if (!forward(m, rows, false, last)) {
            m->prof_used -= m->prof_used % 3;
            return fail(m, GWAM_ECUDA, "kernel launch failed");
        }
        if (m->prof) prof_mark(m);
    }
    return cudaPeekAtLastError() == cudaSuccess ? GWAM_OK : fail(m, GWAM_ECUDA, "kernel launch failed");
}

int gwam_mlp_profile_enable(gwam_mlp* m, int enable)
{
    if (!m) return GWAM_EINVAL;
    prof_harvest(m);
    if (enable) {
        m->prof_ms[0] = m->prof_ms[1] = 0.0;
        m->prof_passes = 0;
    }
    m->prof = enable != 0;
    return GWAM_OK;
}

int gwam_mlp_profile_read(gwam_mlp* m, double* ms_host, int64_t* passes)
{
    if (!m || !ms_host) return GWAM_EINVAL;
    prof_harvest(m);
    ms_host[0] = m->prof_ms[0];
    ms_host[1] = m->prof_ms[1];
    if (passes) *passes = m->prof_passes;
    return GWAM_OK;
}

int gwam_mlp_status(gwam_mlp* m)
{
    if (!m) return GWAM_EINVAL;
    return check_err(m);
}

int gwam_mlp_merge_fallback(const int32_t* mask, int64_t ncol, int nlev, const double* dudt_tracer,
                            const double* dvdt_tracer, double* dudt, double* dvdt, void* stream)
{
    if (!mask || ncol < 1 || nlev < 1 || nlev > 65535 || !dudt_tracer || !dvdt_tracer || !dudt || !dvdt)
        return GWAM_EINVAL;
    const int blocks = (int)std::min<int64_t>((ncol + 255) / 256, 152);
    k_merge<<<dim3(blocks, nlev), 256, 0, (cudaStream_t)stream>>>(mask, ncol, dudt_tracer, dvdt_tracer, dudt, dvdt);
    return cudaPeekAtLastError() == cudaSuccess ? GWAM_OK : GWAM_ECUDA;
}

int gwam_column_features(const double* u, const double* v, const double* n2, const double* rho, int nz, int64_t ncol,
                         const float* src, int n_src, int src_stride, float* X, void* stream)
{
    if (!u || !v || !n2 || !rho || nz < 1 || ncol < 1 || n_src < 0 || (n_src > 0 && !src) || src_stride < 0 || !X)
        return GWAM_EINVAL;
    const int64_t total = ncol * (4 * nz + n_src);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8 * 152);
    k_features<<<blocks, 256, 0, (cudaStream_t)stream>>>(u, v, n2, rho, nz, ncol, src, n_src, src_stride, X);
    return cudaPeekAtLastError() == cudaSuccess ? GWAM_OK : GWAM_ECUDA;
}

int gwam_column_targets(const double* du_sum, const double* dv_sum, int nz, int64_t ncol, double scale, float* Y,
                        void* stream)
{
    if (!du_sum || !dv_sum || nz < 1 || ncol < 1 || !Y) return GWAM_EINVAL;
    const int64_t total = ncol * 2 * nz;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8 * 152);
    k_targets<<<blocks, 256, 0, (cudaStream_t)stream>>>(du_sum, dv_sum, nz, ncol, scale, Y);
    return cudaPeekAtLastError() == cudaSuccess ? GWAM_OK : GWAM_ECUDA;
}

}  // extern "C"
