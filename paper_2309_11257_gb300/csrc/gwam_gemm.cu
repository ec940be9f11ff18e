// gwam_gemm.cu -- tcgen05 / TMA BF16 GEMM with fused epilogues (see gwam_gemm.cuh) and its
// self-test entry point.
#include <cudaTypedefs.h>

#include <algorithm>

#include "gwam_df.cuh"
#include "gwam_gemm.cuh"

namespace gwam {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr uint32_t kABytes = kBM * kBK * 2;          // 16 KB per stage
constexpr unsigned long long kWaitNs = 2000000000ull; // 2 s per wait

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for completion of the mbarrier phase with the given parity; false if it gave up
// (after limit_ns of %globaltimer time, or 2^31 polls)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0; it < 0x7fffffffu; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63u) == 0) {
            const uint64_t t = gtime();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor of a 128-byte swizzled K-major tile: start address >> 4,
// leading offset 16 B (unused for swizzled K-major), stride 1024 B between 8-row groups,
// descriptor version 1, swizzle mode 2 (128 B)
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1), B BF16
// (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Phi(z) = (1 + erf(z / sqrt 2)) / 2 with erf by Abramowitz & Stegun, Handbook of Mathematical
// Functions, formula 7.1.26 (absolute error <= 1.5e-7): for x = |z| / sqrt 2 >= 0,
// erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1 / (1 + p x).
// erf_abs returns erf(|z| / sqrt 2) and exp(-z^2 / 2); 1/sqrt 2 is folded into p, and exp(-z^2/2)
// = 2^(-z^2 log2(e) / 2).  Hardware reciprocal and base-2 exponential approximations (PTX
// rcp.approx / ex2.approx, relative errors near 2^-23 and 2^-22).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float erf_abs(float z, float& e)
{
    const float t = rcp_approx(fmaf(0.23164189961f, fabsf(z), 1.0f));   // p / sqrt 2, p = 0.3275911
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    e = ex2_approx(z * z * -0.72134752044f);                             // -log2(e) / 2
    return fmaf(-(t * poly), e, 1.0f);
}

// GELU(z) = z Phi(z) = z / 2 + |z| erf(|z| / sqrt 2) / 2
__device__ __forceinline__ float gelu(float z)
{
    float e;
    const float r = erf_abs(z, e);
    const float h = 0.5f * z;
    return fmaf(fabsf(h), r, h);
}

// GELU'(z) = Phi(z) + z phi(z), phi(z) = exp(-z^2 / 2) / sqrt(2 pi)
__device__ __forceinline__ float gelu_grad(float z)
{
    float e;
    const float r = erf_abs(z, e);
    return fmaf(z * 0.39894228040143268f, e, fmaf(0.5f, copysignf(r, z), 0.5f));
}

// Epilogue of 32 consecutive accumulator columns n = nb .. nb+31 of one row.  Per-column
// parameters arrive one per lane (lane j holds column nb + j) and are broadcast with shuffles, so
// every lane of the warp must call this (rows >= M only skip the stores).  zz: the prefetched
// pre-activations of EPI_BWD.
template <int MODE>
__device__ __forceinline__ void epi32(const GemmEpi& e, int z, int row, int nb, float (&v)[32], const float* sbias,
                                      float ps, float pm, const float (&zz)[32], int rowmask, double& sq,
                                      uint32_t stg, int cc0)
{
    const bool live = row < e.M;
    const bool full = nb + 32 <= e.N;
    if (MODE == EPI_BWD) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= gelu_grad(zz[j]);
    } else {
        if (e.bias) {
            // the tile's bias from shared memory (zero beyond N), broadcast to every lane
            const float4* bp = reinterpret_cast<const float4*>(sbias + nb);
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
                const float4 b = bp[qq];
                v[4 * qq] += b.x;
                v[4 * qq + 1] += b.y;
                v[4 * qq + 2] += b.z;
                v[4 * qq + 3] += b.w;
            }
        }
        if (MODE == EPI_DRAG) {
            // de-normalised in FP32 (one FMA, relative error 6e-8, far below the BF16 network's) and
            // widened exactly by integer operations: FP64 arithmetic and float -> double conversions
            // run at 1/64 of the FP32 rate on GB300
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float sj = __shfl_sync(0xffffffffu, ps, j), mj = __shfl_sync(0xffffffffu, pm, j);
                const int n = nb + j;
                if (live && rowmask == 0 && n < e.n_true) {
                    const double y = gwam::widen(__fmaf_rn(v[j], sj, mj));
                    if (n < e.nlev) e.du[(size_t)n * e.ncol + row] = y;
                    else e.dv[(size_t)(n - e.nlev) * e.ncol + row] = y;
                }
            }
            return;
        }
        if (!live) return;
        if (MODE == EPI_STORE) {
            if (e.z) {
                float* p = e.z + (size_t)row * e.ldz + nb;
                if (full && (e.ldz & 3) == 0) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (nb + j < e.N) p[j] = v[j];
                }
            }
            if (e.act) {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = gelu(v[j]);
            }
        } else {  // EPI_LOSS
            if (e.cf) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (nb + j < e.N) e.cf[(size_t)row * e.ldcf + nb + j] = v[j];
            }
            const float* tp = e.tgt + (size_t)row * e.ldt + nb;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float d = nb + j < e.n_true ? v[j] - tp[j] : 0.0f;
                sq += (double)d * (double)d;
                v[j] = e.gscale * d;
            }
        }
    }
    if (!live) return;
    if (MODE == EPI_STORE && e.cf) {
        float* p = e.cf + (size_t)z * e.cf_slice + (size_t)row * e.ldcf + nb;
        if (full && (e.ldcf & 3) == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < e.N) p[j] = v[j];
        }
    }
    if (e.cb && stg) {
        // this row's 64 bytes into the warp's 128-byte-swizzled staging box (16-byte chunk c of
        // row r at r * 128 + ((c ^ (r % 8)) * 16)); a TMA store writes the box out
        uint32_t w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            w[q] = *reinterpret_cast<const uint32_t*>(&h);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t a = stg + ((uint32_t)((cc0 + q) ^ (row & 7)) << 4);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[4 * q]), "r"(w[4 * q + 1]),
                         "r"(w[4 * q + 2]), "r"(w[4 * q + 3])
                         : "memory");
        }
    } else if (e.cb) {
        __nv_bfloat16* p = e.cb + (size_t)row * e.ldcb + nb;
        if (full && (e.ldcb & 7) == 0) {
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                reinterpret_cast<uint4*>(p)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < e.N) p[j] = __float2bfloat16_rn(v[j]);
        }
    }
    if (e.ct) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (nb + j < e.N) e.ct[(size_t)(nb + j) * e.ldct + row] = __float2bfloat16_rn(v[j]);
    }
}

// Persistent, warp-specialised GEMM.  Warp 0 (one lane) streams the K blocks of every tile the
// CTA owns through the shared-memory ring; warp 1 allocates TMEM and (one lane) issues the MMAs of
// tile i into accumulator i % 2; warps 2 .. 2+EPW-1 drain accumulator (i % 2) while the MMAs of tile
// i + 1 run into the other one.  Epilogue warp w reads TMEM lane quarter w % 4 and, with EPW / 4
// warps per quarter, its share of the columns.  Tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// over (k slice, m tile, n tile), n fastest.
template <int BN, int ST, int EPW, int MODE>
__global__ void __launch_bounds__(64 + 32 * EPW, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                const __grid_constant__ CUtensorMap tc, int K, int ksplit, GemmEpi e)
{
    constexpr uint32_t kBBytes = BN * kBK * 2;
    constexpr uint32_t kStage = kABytes + kBBytes;   // a multiple of 1024
    constexpr uint32_t kAccStride = BN <= 64 ? 64 : (BN <= 128 ? 128 : 256);
    constexpr uint32_t kCols = 2 * kAccStride;
    constexpr int kEpiThreads = 32 * EPW;
    constexpr int kColsPerWarp = BN / (EPW / 4);
    static_assert(kColsPerWarp % 64 == 0, "epilogue column share must be a multiple of 64");
    constexpr uint32_t kStgWarp = 32u * kColsPerWarp * 2u;   // BF16 staging of a warp's 32 rows
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[ST], empty_bar[ST], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = (e.N + BN - 1) / BN, m_tiles = (e.M + kBM - 1) / kBM;
    const int per_slice = n_tiles * m_tiles;
    const int total = per_slice * ksplit;
    const int nk = K / kBK / ksplit;
    const uint32_t base = (saddr(smem_raw) + 1023u) & ~1023u;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty_bar[s])));
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&accf_bar[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&acce_bar[a])), "r"(kEpiThreads));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    // behind the stage ring: the epilogue warps' BF16 staging boxes (TMA-store mode), then the bias
    // of all N columns, zero-padded to a multiple of 32
    const uint32_t stg_base = base + (uint32_t)ST * kStage;
    float* sbias = reinterpret_cast<float*>(smem_raw + (base - saddr(smem_raw)) + (size_t)ST * kStage +
                                            (e.tstore ? (size_t)EPW * kStgWarp : 0));
    // programmatic dependent launch: the next kernel in the stream may start its own set-up now; this
    // one waits until the previous kernel has completed before it reads anything from global memory
    // (the set-up above touched only shared and tensor memory and the kernel parameters)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (e.bias) {
        const int npad = (e.N + 31) & ~31;
        for (int i = tid; i < npad; i += blockDim.x) sbias[i] = i < e.N ? e.bias[i] : 0.0f;
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_slot;
    const unsigned long long wlim = e.wait_ns ? e.wait_ns : kWaitNs;
    bool ok = true;
    double sq = 0.0;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
            int it = 0;
            // (self-test of the give-up path: no copy is issued, so the MMA and epilogue warps wait
            // on stages that never fill and give up after wait_ns)
            for (int t = blockIdx.x; t < total && ok && !e.skip_copies; t += gridDim.x) {
                const int z = t / per_slice, r = t - z * per_slice;
                const int m0 = (r / n_tiles) * kBM, n0 = (r % n_tiles) * BN;
                for (int i = 0; i < nk; ++i, ++it) {
                    const int s = it % ST;
                    if (it >= ST && !mbar_wait(saddr(&empty_bar[s]), (uint32_t)((it / ST - 1) & 1), wlim)) {
                        ok = false;
                        break;
                    }
                    if (abort_flag) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = saddr(&full_bar[s]);
                    const uint32_t dA = base + (uint32_t)s * kStage, dB = dA + kABytes;
                    const int kx = (z * nk + i) * kBK;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStage)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
                        "{%2, %3}], [%4];" ::"r"(dA),
                        "l"(reinterpret_cast<uint64_t>(&ta)), "r"(kx), "r"(m0), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
                        "{%2, %3}], [%4];" ::"r"(dB),
                        "l"(reinterpret_cast<uint64_t>(&tb)), "r"(kx), "r"(n0), "r"(fb)
                        : "memory");
                }
            }
            if (!ok) abort_flag = 1;
            // every issued copy has landed before the CTA may exit (immediate in the normal case)
            for (int i = it > ST ? it - ST : 0; i < it; ++i)
                if (!mbar_wait(saddr(&full_bar[i % ST]), (uint32_t)((i / ST) & 1), wlim)) ok = false;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            constexpr uint32_t idesc = idesc_bf16(kBM, BN);
            int it = 0, tl = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
                const int acc = tl & 1;
                if (tl >= 2 && !mbar_wait(saddr(&acce_bar[acc]), (uint32_t)((tl / 2 - 1) & 1), wlim)) {
                    ok = false;
                    break;
                }
                tc_after();
                const uint32_t d = tmem + (uint32_t)acc * kAccStride;
                for (int i = 0; i < nk; ++i, ++it) {
                    const int s = it % ST;
                    if (abort_flag || !mbar_wait(saddr(&full_bar[s]), (uint32_t)((it / ST) & 1), wlim)) {
                        ok = false;
                        break;
                    }
                    tc_after();
                    const uint32_t a0 = base + (uint32_t)s * kStage, b0 = a0 + kABytes;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t ad = desc_sw128(a0 + 32u * kk), bd = desc_sw128(b0 + 32u * kk);
                        const uint32_t accum = (i > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     saddr(&empty_bar[s]))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 saddr(&accf_bar[acc]))
                             : "memory");
            }
            if (!ok) abort_flag = 1;
            // tracks every MMA issued above (also after a give-up): released TMEM is never written
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&done_bar))
                         : "memory");
        }
        __syncwarp();
    } else {
        // epilogue warps
        constexpr int kChunks = kColsPerWarp / 32;
        const int q = warp & 3, part = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int tl = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++tl) {
            const int acc = tl & 1;
            const int z = t / per_slice, r = t - z * per_slice;
            const int m0 = (r / n_tiles) * kBM, n0 = (r % n_tiles) * BN;
            const int row = m0 + q * 32 + lane;
            const int cbeg = n0 + part * kColsPerWarp;
            // de-normalisation of this warp's columns, one per lane, fetched before the wait
            float ps[kChunks], pm[kChunks];
#pragma unroll
            for (int k = 0; k < kChunks; ++k) {
                const int n = cbeg + 32 * k + lane;
                ps[k] = (MODE == EPI_DRAG && n < e.n_true) ? e.ysig[n] : 0.0f;
                pm[k] = (MODE == EPI_DRAG && n < e.n_true) ? e.ymu[n] : 0.0f;
            }
            const int rowmask = (MODE == EPI_DRAG && row < e.M) ? e.mask[row] : 0;
            const bool got = mbar_wait(saddr(&accf_bar[acc]), (uint32_t)((tl / 2) & 1), wlim);
            if (!__all_sync(0xffffffffu, got) || abort_flag) {
                ok = false;
                break;
            }
            tc_after();
            const uint32_t stg_warp = stg_base + (uint32_t)(warp - 2) * kStgWarp;
            if (e.tstore) {
                // the previous tile's TMA store has finished reading this warp's staging boxes
                if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                __syncwarp();
            }
            const uint32_t tacc = tmem + lane_base + (uint32_t)acc * kAccStride + (uint32_t)(part * kColsPerWarp);
            // the 32-column chunks as a rolled loop (one copy of the epilogue arithmetic: the epilogue
            // warps stalled on instruction fetch; GEMM chain 0.173 -> 0.165 ms per 32 768 columns)
#pragma unroll 1
            for (int k = 0; k < kChunks; ++k) {
                const int nb = cbeg + 32 * k;
                if (nb >= e.N) break;
                float zz[32];
                if (MODE == EPI_BWD) {
                    // pre-activations in flight while the accumulator is read
                    if (row < e.M && nb + 32 <= e.N && (e.ldz & 3) == 0) {
                        const float4* zp = reinterpret_cast<const float4*>(e.z + (size_t)row * e.ldz + nb);
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq) {
                            const float4 w = zp[qq];
                            zz[4 * qq] = w.x;
                            zz[4 * qq + 1] = w.y;
                            zz[4 * qq + 2] = w.z;
                            zz[4 * qq + 3] = w.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            zz[j] = (row < e.M && nb + j < e.N) ? e.z[(size_t)row * e.ldz + nb + j] : 0.0f;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) zz[j] = 0.0f;
                }
                uint32_t rr[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                      "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                      "=r"(rr[14]), "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]),
                      "=r"(rr[21]), "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]),
                      "=r"(rr[28]), "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                    : "r"(tacc + (uint32_t)(32 * k)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(rr[j]);
                const uint32_t stg =
                    e.tstore ? stg_warp + (uint32_t)((32 * k) / 64) * 4096u + (uint32_t)lane * 128u : 0u;
                // this chunk's de-normalisation, selected rather than indexed (stays in registers)
                float psk = ps[0], pmk = pm[0];
#pragma unroll
                for (int u = 1; u < kChunks; ++u)
                    if (k == u) {
                        psk = ps[u];
                        pmk = pm[u];
                    }
                epi32<MODE>(e, z, row, nb, v, sbias, psk, pmk, zz, rowmask, sq, stg, ((32 * k) % 64) / 8);
            }
            tc_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&acce_bar[acc])) : "memory");
            if (e.tstore) {
                // staging -> global by TMA (rows and columns outside the tensor are clipped)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
#pragma unroll
                    for (int b = 0; b < kColsPerWarp / 64; ++b) {
                        const int x = cbeg + 64 * b;
                        if (x < e.N)
                            asm volatile(
                                "cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                                    reinterpret_cast<uint64_t>(&tc)),
                                "r"(x), "r"(m0 + q * 32), "r"(stg_warp + (uint32_t)b * 4096u)
                                : "memory");
                    }
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            }
        }
        // this warp's TMA stores have completed before the CTA exits
        if (e.tstore && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
        if (!ok) abort_flag = 1;
        if (MODE == EPI_LOSS) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0 && sq != 0.0) atomicAdd(e.loss, sq);
        }
    }
    // every MMA has finished before the TMEM is released (bounded wait; immediate normally)
    const bool fin = mbar_wait(saddr(&done_bar), 0u, wlim);
    if (!__syncthreads_and(ok && fin) && tid == 0 && e.err) atomicOr(e.err, 1);
    tc_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <int BN, int ST, int EPW, int MODE>
bool launch_mode(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc, int K, int ksplit,
                 const GemmEpi& e, cudaStream_t s)
{
    constexpr size_t kMaxShm = 232448 - 256;   // 227 KB opt-in per block, less the static part
    constexpr size_t kStg = (size_t)32 * BN / (EPW / 4) * 2 * EPW;
    const size_t shm = (size_t)ST * (kABytes + BN * kBK * 2) + 1024 + (e.tstore ? kStg : 0) +
                       (e.bias ? (size_t)((e.N + 31) & ~31) * 4 : 0);
    if (shm > kMaxShm) return false;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64) return false;
    // dynamic shared memory limit raised per device to the largest size launched so far (the
    // opt-in limit counts the kernel's static shared memory too)
    static size_t configured[64] = {};
    static int sms[64] = {};
    if (shm > configured[dev]) {
        if (cudaFuncSetAttribute(k_gemm_bf16<BN, ST, EPW, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) !=
            cudaSuccess)
            return false;
        configured[dev] = shm;
        sms[dev] = sm_count();
    }
    const long long tiles = (long long)((e.N + BN - 1) / BN) * ((e.M + kBM - 1) / kBM) * ksplit;
    const int grid = (int)std::min<long long>(tiles, sms[dev]);
    // launched with programmatic stream serialisation: the set-up of this GEMM (barriers, tensor
    // memory) overlaps the tail of the kernel before it, which it waits for before its first read
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(64 + 32 * EPW);
    cfg.dynamicSmemBytes = shm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gemm_bf16<BN, ST, EPW, MODE>, ta, tb, tc, K, ksplit, e) == cudaSuccess;
}

// one kernel per epilogue mode: each holds only its own epilogue code (a smaller instruction
// footprint for the epilogue warps, whose instruction fetch otherwise stalls them)
template <int BN, int ST, int EPW>
bool launch(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc, int K, int ksplit, const GemmEpi& e,
            cudaStream_t s)
{
    switch (e.mode) {
    case EPI_STORE: return launch_mode<BN, ST, EPW, EPI_STORE>(ta, tb, tc, K, ksplit, e, s);
    case EPI_BWD: return launch_mode<BN, ST, EPW, EPI_BWD>(ta, tb, tc, K, ksplit, e, s);
    case EPI_LOSS: return launch_mode<BN, ST, EPW, EPI_LOSS>(ta, tb, tc, K, ksplit, e, s);
    case EPI_DRAG: return launch_mode<BN, ST, EPW, EPI_DRAG>(ta, tb, tc, K, ksplit, e, s);
    default: return false;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows)
{
    auto fn = encode_fn();
    if (!fn || !map || !base || rows == 0 || cols == 0 || ld < cols || (ld * 2) % 16 || box_rows == 0 ||
        box_rows > 256 || (reinterpret_cast<uintptr_t>(base) & 15))
        return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int gemm_pick_bn(int M, int N)
{
    (void)M;
    if (N <= 64) return 64;
    if (N <= 128) return 128;
    if (N <= 192) return 192;
    return 256;
}

bool gemm_bf16_launch(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap* tc, int K, int bn, int ksplit,
                      const GemmEpi& e_in, cudaStream_t s)
{
    if (e_in.M < 1 || e_in.N < 1 || K < kBK || K % kBK || ksplit < 1 || (K / kBK) % ksplit || ksplit > 65535)
        return false;
    if (ksplit > 1 && e_in.mode != EPI_STORE) return false;
    GemmEpi e = e_in;
    e.tstore = (tc && e.cb) ? 1 : 0;
    static const CUtensorMap none{};
    const CUtensorMap& tcm = e.tstore ? *tc : none;
    if (bn == 0) bn = gemm_pick_bn(e.M, e.N);
    switch (bn) {
    case 64: return launch<64, 8, 4>(ta, tb, tcm, K, ksplit, e, s);
    case 128: return launch<128, 5, 8>(ta, tb, tcm, K, ksplit, e, s);
    case 192: return launch<192, 4, 12>(ta, tb, tcm, K, ksplit, e, s);
    case 256: return launch<256, 3, 16>(ta, tb, tcm, K, ksplit, e, s);
    default: return false;
    }
}

}  // namespace gwam

namespace {

int gemm_selftest(const void* A, const void* B, int M, int N, int K, const float* bias, int gelu, int bn, int out_bf16,
                  void* C, unsigned long long wait_ns, int skip_copies, void* stream)
{
    if (!A || !B || !C || M < 1 || N < 1 || K < 64 || K % 64 || (bn != 0 && bn != 64 && bn != 128 && bn != 192 &&
                                                                  bn != 256))
        return -1;
    cudaStream_t s = (cudaStream_t)stream;
    const int use_bn = bn ? bn : gwam::gemm_pick_bn(M, N);
    CUtensorMap ta, tb, tc;
    if (!gwam::make_tmap_bf16(&ta, A, (uint64_t)M, (uint64_t)K, (uint64_t)K, 128) ||
        !gwam::make_tmap_bf16(&tb, B, (uint64_t)N, (uint64_t)K, (uint64_t)K, (uint32_t)use_bn))
        return -1;
    const bool have_tc = out_bf16 && N % 8 == 0 && gwam::make_tmap_bf16(&tc, C, (uint64_t)M, (uint64_t)N, (uint64_t)N, 32);
    int* err = nullptr;
    if (cudaMallocAsync((void**)&err, sizeof(int), s) != cudaSuccess) return -2;
    cudaMemsetAsync(err, 0, sizeof(int), s);
    gwam::GemmEpi e{};
    e.mode = gwam::EPI_STORE;
    e.act = gelu ? 1 : 0;
    e.M = M;
    e.N = N;
    e.bias = bias;
    if (out_bf16) {
        e.cb = (__nv_bfloat16*)C;
        e.ldcb = N;
    } else {
        e.cf = (float*)C;
        e.ldcf = N;
    }
    e.err = err;
    e.wait_ns = wait_ns;
    e.skip_copies = skip_copies;
    const bool launched = gwam::gemm_bf16_launch(ta, tb, have_tc ? &tc : nullptr, K, use_bn, 1, e, s);
    int h = 0;
    cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || !launched) return -5;
    return h ? -6 : 0;
}

}  // namespace

// Self-test entry point (declared in gwam.h): C = act(A . B^T + bias) with BF16 A [M][K] and
// B [N][K]; C FP32 [M][N], or BF16 [M][N] (written by TMA stores when N is a multiple of 8);
// bn = 0 picks the tile width.
extern "C" int gwam_gemm_bf16(const void* A, const void* B, int M, int N, int K, const float* bias, int gelu, int bn,
                              int out_bf16, void* C, void* stream)
{
    return gemm_selftest(A, B, M, N, K, bias, gelu, bn, out_bf16, C, 0ull, 0, stream);
}

// Self-test of the bounded waits (declared in gwam.h): the same GEMM with its producer told to
// issue no copies and every wait limited to wait_us microseconds; the kernel gives up, frees its
// TMEM and reports, and the call returns GWAM_ETIMEOUT.
extern "C" int gwam_selftest_gemm_timeout(const void* A, const void* B, int M, int N, int K, int bn, float* C,
                                          unsigned int wait_us, void* stream)
{
    if (wait_us < 1 || wait_us > 2000000u) return -1;
    return gemm_selftest(A, B, M, N, K, nullptr, 0, bn, 0, C, 1000ull * wait_us, 1, stream);
}
