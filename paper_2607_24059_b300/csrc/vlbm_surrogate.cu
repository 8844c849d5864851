// Tensor-core (tcgen05) kernels of the learned surrogate: a BF16 GEMM core
// (D = A B^T, FP32 accumulation in tensor memory) that the convolution layers
// are built on.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "vlbm.h"
#include "vlbm_tc.cuh"

using namespace vlbm;

namespace {

constexpr int kTcThreads = 128;          // one warpgroup: TMEM lanes 0..127
constexpr int kKChunk = 64;              // K columns staged per round
constexpr long long kWaitPolls = 1 << 22;

// D[M x N] = A[M x K] B[N x K]^T for one 128-row block of A.  A, B row-major
// BF16 (K contiguous), D row-major FP32.  N % 16 == 0, 16 <= N <= 256, K % 64 == 0.
__global__ void __launch_bounds__(kTcThreads)
k_tc_gemm_bf16(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B, float* __restrict__ D,
               int N, int K, int* __restrict__ err) {
    __shared__ __align__(1024) uint8_t sA[128 * kKChunk * 2];
    __shared__ __align__(1024) uint8_t sB[256 * kKChunk * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long m0 = (long long)blockIdx.x * 128;
    const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));

    if (warp == 0) {
        tc::tmem_alloc(&s_taddr, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = tc::idesc_bf16_f32(128, N);
    uint32_t phase = 0;
    bool ok = true;

    for (int kc = 0; kc < K && ok; kc += kKChunk) {
        // stage A (128 x 64) and B (N x 64) as K-major core matrices, 16 bytes per copy
        for (int i = tid; i < 128 * (kKChunk / 8); i += kTcThreads) {
            const int row = i / (kKChunk / 8), kb = i % (kKChunk / 8);
            const uint4 v = *reinterpret_cast<const uint4*>(A + (m0 + row) * K + kc + kb * 8);
            *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, kb * 8, kKChunk)) = v;
        }
        for (int i = tid; i < N * (kKChunk / 8); i += kTcThreads) {
            const int row = i / (kKChunk / 8), kb = i % (kKChunk / 8);
            const uint4 v = *reinterpret_cast<const uint4*>(B + (long long)row * K + kc + kb * 8);
            *reinterpret_cast<uint4*>(sB + tc::kmajor_offset(row, kb * 8, kKChunk)) = v;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
            const uint32_t sbo = 128 * (kKChunk / 8);
#pragma unroll
            for (int s = 0; s < kKChunk / 16; ++s) {
                const uint64_t da = tc::smem_desc(a0 + s * 256, 128, sbo);
                const uint64_t db = tc::smem_desc(b0 + s * 256, 128, sbo);
                tc::mma_bf16(taddr, da, db, idesc, (kc > 0 || s > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar);
        }
        // every thread waits: the staging buffers are rewritten next round
        if (!tc::mbar_wait(&bar, phase, kWaitPolls)) {
            ok = false;
            atomicExch(err, 1);
        }
        phase ^= 1;
        __syncthreads();
    }

    if (ok) {
        tc::fence_after_sync();
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const long long row = m0 + warp * 32 + (tid & 31);
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + lane_base + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) D[row * N + c + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

}  // namespace

extern "C" int vlbm_tc_gemm_bf16(const void* A, const void* B, float* D, int64_t M, int64_t N, int64_t K,
                                 int32_t* err_dev, void* stream) {
    if (!A || !B || !D || !err_dev || M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K <= 0 || K % kKChunk)
        return VLBM_EINVAL;
    k_tc_gemm_bf16<<<(unsigned)(M / 128), kTcThreads, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)A, (const __nv_bfloat16*)B, D, (int)N, (int)K, err_dev);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}
