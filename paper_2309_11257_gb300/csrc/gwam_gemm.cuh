// gwam_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) for the drag
// surrogate: C[M, N] = A[M, K] . B[N, K]^T, FP32 accumulation in tensor memory (TMEM), both
// operands K-major (row-major with K contiguous), fused epilogues.
//
// One CTA computes a 128 x BN tile (BN in {64, 128, 192, 256}).  Thread 0 is the TMA producer:
// it streams 64-wide K blocks of A and B into a ring of shared-memory stages (128-byte swizzled
// K-major layout, written by cp.async.bulk.tensor) and signals a "full" mbarrier per stage with
// the transaction byte count.  Thread 32 issues four 128 x BN x 16 tcgen05.mma per K block into
// the TMEM accumulator and commits them to the stage's "empty" mbarrier, which hands the stage
// back to the producer; a final commit signals the accumulator.  All four warps then read the
// accumulator with tcgen05.ld (warp w owns TMEM lanes = tile rows 32w..32w+31) and run the
// epilogue.  Every mbarrier wait is bounded in time; a wait that gives up sets the error word,
// the kernel still waits (bounded) for its own copies and MMAs and releases its TMEM.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gwam {

enum GemmEpiMode {
    EPI_STORE = 0,  // v = acc (+ bias) (-> GELU if act); writes cf (FP32), cb (BF16), ct (BF16
                    // transposed); z receives the pre-activation
    EPI_BWD = 1,    // v = acc * GELU'(z[row][n]); writes cb and ct
    EPI_LOSS = 2,   // y = acc + bias; e = y - tgt (n < n_true, else 0); d = gscale * e -> cb, ct;
                    // y -> cf; sum of e^2 added to *loss
    EPI_DRAG = 3,   // y = acc + bias; for n < n_true and mask[row] == 0: y * ysig[n] + ymu[n]
                    // -> du[n * ncol + row] (n < nlev) or dv[(n - nlev) * ncol + row]
};

struct GemmEpi {
    int mode;
    int act;                  // EPI_STORE: apply GELU
    int M, N;                 // valid rows and columns of C
    const float* bias;        // [N] or null
    float* cf;                // FP32 [M][ldcf] (+ blockIdx.z * cf_slice for split-K partials)
    int ldcf;
    long long cf_slice;
    __nv_bfloat16* cb;        // BF16 [M][ldcb]
    int ldcb;
    __nv_bfloat16* ct;        // BF16 transposed [N][ldct]
    int ldct;
    float* z;                 // FP32 pre-activation [M][ldz]
    int ldz;
    const float* tgt;         // EPI_LOSS: normalised targets [M][ldt]
    int ldt;
    int n_true;               // EPI_LOSS / EPI_DRAG: number of real outputs (N may be padded)
    float gscale;             // EPI_LOSS: dL/dy = gscale * (y - t)
    double* loss;             // EPI_LOSS: sum of squared errors (FP64 atomic per warp)
    const float* ysig;        // EPI_DRAG: de-normalisation
    const float* ymu;
    const int* mask;          // EPI_DRAG: 1 = column goes to the ray tracer
    double* du;
    double* dv;
    int ncol, nlev;
    int* err;                 // bit 0 set when a bounded wait gave up
    int tstore;               // set by gemm_bf16_launch: cb is written through an output tensor map
    unsigned long long wait_ns;   // limit of every bounded wait (0: 2 s)
    int skip_copies;          // self-test of the give-up path only: the producer issues no copies
};

// 2-D BF16 tensor map of a row-major [rows][cols] matrix with leading dimension ld (elements),
// box = 64 columns x box_rows rows, 128-byte swizzle.  false if the driver refuses it.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                    uint32_t box_rows);

// Launch: A described by ta (box rows 128), B by tb (box rows bn); K a multiple of 64, split into
// ksplit slices along K (K / 64 must be divisible by ksplit).  tc (or null): tensor map of the BF16
// output cb (box 64 columns x 32 rows) -- the epilogue then stages each warp's rows in shared memory
// and writes them with TMA stores.  bn = 0 picks the tile width from N.  false on an unsupported
// shape.
bool gemm_bf16_launch(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap* tc, int K, int bn, int ksplit,
                      const GemmEpi& e, cudaStream_t s);

// The tile width gemm_bf16_launch uses for N when bn = 0 (the caller builds tb with this box).
int gemm_pick_bn(int M, int N);

}  // namespace gwam
