// gwam_gemm.cu -- tcgen05 / TMA BF16 GEMM with fused epilogues (see gwam_gemm.cuh) and its
// self-test entry point.
#include <cudaTypedefs.h>

#include "gwam_gemm.cuh"

namespace gwam {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kThreads = 128;
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
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
            else if (t - t0 > kWaitNs) return false;
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

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// epilogue of 16 consecutive accumulator columns n = nb .. nb+15 of one row
__device__ __forceinline__ void epi16(const GemmEpi& e, int row, int nb, const uint32_t (&r)[16], double& sq)
{
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
    const bool full = nb + 16 <= e.N;
    if (e.mode == EPI_BWD) {
        if (full && (e.ldz & 3) == 0) {
            const float4* zp = reinterpret_cast<const float4*>(e.z + (size_t)row * e.ldz + nb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 zz = zp[q];
                v[4 * q] *= gelu_grad(zz.x);
                v[4 * q + 1] *= gelu_grad(zz.y);
                v[4 * q + 2] *= gelu_grad(zz.z);
                v[4 * q + 3] *= gelu_grad(zz.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < e.N) v[j] *= gelu_grad(e.z[(size_t)row * e.ldz + nb + j]);
        }
    } else {
        if (e.bias) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < e.N) v[j] += e.bias[nb + j];
        }
        if (e.mode == EPI_STORE) {
            if (e.z) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (nb + j < e.N) e.z[(size_t)row * e.ldz + nb + j] = v[j];
            }
            if (e.act) {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = gelu(v[j]);
            }
        } else if (e.mode == EPI_LOSS) {
            if (e.cf) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (nb + j < e.N) e.cf[(size_t)row * e.ldcf + nb + j] = v[j];
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = nb + j;
                const float d = n < e.n_true ? v[j] - e.tgt[(size_t)row * e.ldt + n] : 0.0f;
                sq += (double)d * (double)d;
                v[j] = e.gscale * d;
            }
        } else {  // EPI_DRAG
            if (e.mask[row] == 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = nb + j;
                    if (n < e.n_true) {
                        const double y = (double)v[j] * (double)e.ysig[n] + (double)e.ymu[n];
                        if (n < e.nlev) e.du[(size_t)n * e.ncol + row] = y;
                        else e.dv[(size_t)(n - e.nlev) * e.ncol + row] = y;
                    }
                }
            }
            return;
        }
    }
    if (e.mode == EPI_STORE && e.cf) {
        float* p = e.cf + (size_t)blockIdx.z * e.cf_slice + (size_t)row * e.ldcf + nb;
        if (full && (e.ldcf & 3) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < e.N) p[j] = v[j];
        }
    }
    if (e.cb) {
        __nv_bfloat16* p = e.cb + (size_t)row * e.ldcb + nb;
        if (full && (e.ldcb & 7) == 0) {
            uint32_t w[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            }
            reinterpret_cast<uint4*>(p)[0] = make_uint4(w[0], w[1], w[2], w[3]);
            reinterpret_cast<uint4*>(p)[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < e.N) p[j] = __float2bfloat16_rn(v[j]);
        }
    }
    if (e.ct) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (nb + j < e.N) e.ct[(size_t)(nb + j) * e.ldct + row] = __float2bfloat16_rn(v[j]);
    }
}

template <int BN, int ST>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int K, GemmEpi e)
{
    constexpr uint32_t kBBytes = BN * kBK * 2;
    constexpr uint32_t kStage = kABytes + kBBytes;   // a multiple of 1024
    constexpr uint32_t kCols = BN <= 64 ? 64 : (BN <= 128 ? 128 : 256);
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[ST], empty_bar[ST], acc_bar;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM;
    const int kb_total = K / kBK;
    const int kb_per = kb_total / (int)gridDim.z;
    const int kb0 = blockIdx.z * kb_per;
    const int nk = kb_per;
    const uint32_t base = (saddr(smem_raw) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int s = 0; s < ST; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty_bar[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&acc_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (tid == 0) {
        // TMA producer
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % ST;
            if (i >= ST && !mbar_wait(saddr(&empty_bar[s]), (uint32_t)((i / ST - 1) & 1))) {
                ok = false;
                break;
            }
            const uint32_t fb = saddr(&full_bar[s]);
            const uint32_t dA = base + (uint32_t)s * kStage, dB = dA + kABytes;
            const int kx = (kb0 + i) * kBK;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStage) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(dA),
                "l"(reinterpret_cast<uint64_t>(&ta)), "r"(kx), "r"(m0), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(dB),
                "l"(reinterpret_cast<uint64_t>(&tb)), "r"(kx), "r"(n0), "r"(fb)
                : "memory");
            ++issued;
        }
        // every issued copy has landed before the CTA may exit (immediate in the normal case)
        for (int i = issued > ST ? issued - ST : 0; i < issued; ++i)
            if (!mbar_wait(saddr(&full_bar[i % ST]), (uint32_t)((i / ST) & 1))) ok = false;
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kBM, BN);
        for (int i = 0; i < nk; ++i) {
            const int s = i % ST;
            if (!mbar_wait(saddr(&full_bar[s]), (uint32_t)((i / ST) & 1))) {
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
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&empty_bar[s]))
                         : "memory");
        }
        // tracks every MMA issued above, also after a give-up
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr(&acc_bar))
                     : "memory");
    }
    __syncwarp();

    bool acc_ok = mbar_wait(saddr(&acc_bar), 0u);
    tc_after();
    if (!__syncthreads_and(ok && acc_ok)) {
        if (tid == 0 && e.err) atomicOr(e.err, 1);
        // MMAs still in flight must finish before the TMEM is released: wait once more (bounded)
        if (!acc_ok) acc_ok = mbar_wait(saddr(&acc_bar), 0u);
    } else {
        const int row = m0 + warp * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        double sq = 0.0;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            if (n0 + c0 >= e.N) break;
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tl + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < e.M) epi16(e, row, n0 + c0, r, sq);
        }
        if (e.mode == EPI_LOSS) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0 && sq != 0.0) atomicAdd(e.loss, sq);
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

template <int BN, int ST>
bool launch(const CUtensorMap& ta, const CUtensorMap& tb, int K, int ksplit, const GemmEpi& e, cudaStream_t s)
{
    constexpr size_t shm = (size_t)ST * (kABytes + BN * kBK * 2) + 1024;
    int dev = 0;
    cudaGetDevice(&dev);
    static unsigned long long configured = 0;  // one bit per device
    if (dev < 64 && !(configured >> dev & 1ull)) {
        if (cudaFuncSetAttribute(k_gemm_bf16<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) !=
            cudaSuccess)
            return false;
        configured |= 1ull << dev;
    }
    const dim3 grid((unsigned)((e.N + BN - 1) / BN), (unsigned)((e.M + kBM - 1) / kBM), (unsigned)ksplit);
    k_gemm_bf16<BN, ST><<<grid, kThreads, shm, s>>>(ta, tb, K, e);
    return cudaPeekAtLastError() == cudaSuccess;
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
    return 128;
}

bool gemm_bf16_launch(const CUtensorMap& ta, const CUtensorMap& tb, int K, int bn, int ksplit, const GemmEpi& e,
                      cudaStream_t s)
{
    if (e.M < 1 || e.N < 1 || K < kBK || K % kBK || ksplit < 1 || (K / kBK) % ksplit || ksplit > 65535) return false;
    if (ksplit > 1 && e.mode != EPI_STORE) return false;
    if (bn == 0) bn = gemm_pick_bn(e.M, e.N);
    switch (bn) {
    case 64: return launch<64, 4>(ta, tb, K, ksplit, e, s);
    case 128: return launch<128, 3>(ta, tb, K, ksplit, e, s);
    case 192: return launch<192, 4>(ta, tb, K, ksplit, e, s);
    case 256: return launch<256, 4>(ta, tb, K, ksplit, e, s);
    default: return false;
    }
}

}  // namespace gwam

// Self-test entry point (declared in gwam.h): C = act(A . B^T + bias) with BF16 A [M][K] and
// B [N][K], FP32 C [M][N]; bn = 0 picks the tile width.
extern "C" int gwam_gemm_bf16(const void* A, const void* B, int M, int N, int K, const float* bias, int gelu, int bn,
                              float* C, void* stream)
{
    if (!A || !B || !C || M < 1 || N < 1 || K < 64 || K % 64 || (bn != 0 && bn != 64 && bn != 128 && bn != 192 &&
                                                                  bn != 256))
        return -1;
    cudaStream_t s = (cudaStream_t)stream;
    const int use_bn = bn ? bn : gwam::gemm_pick_bn(M, N);
    CUtensorMap ta, tb;
    if (!gwam::make_tmap_bf16(&ta, A, (uint64_t)M, (uint64_t)K, (uint64_t)K, 128) ||
        !gwam::make_tmap_bf16(&tb, B, (uint64_t)N, (uint64_t)K, (uint64_t)K, (uint32_t)use_bn))
        return -1;
    int* err = nullptr;
    if (cudaMallocAsync((void**)&err, sizeof(int), s) != cudaSuccess) return -2;
    cudaMemsetAsync(err, 0, sizeof(int), s);
    gwam::GemmEpi e{};
    e.mode = gwam::EPI_STORE;
    e.act = gelu ? 1 : 0;
    e.M = M;
    e.N = N;
    e.bias = bias;
    e.cf = C;
    e.ldcf = N;
    e.err = err;
    const bool launched = gwam::gemm_bf16_launch(ta, tb, K, use_bn, 1, e, s);
    int h = 0;
    cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || !launched) return -5;
    return h ? -6 : 0;
}
