// kernels_tc.cu -- tensor-core (tcgen05) kernels: a layout self-test and the reduced-precision
// PRISM beam contraction.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "params.h"
#include "tc.cuh"

namespace prism {

// ------------------------------------------------------------------ self-test
// One MMA D[128][16] = A[128][16] B[16][16]^T with small-integer FP16 operands (exact in FP32),
// operands in the K-major core-matrix layout of tc.cuh.  The operand buffer is oversized so that
// every core matrix the descriptors can address lies inside it.  out[m*16 + n] = D[m][n];
// status[0] = 1 if the MMA did not complete within the poll limit.
__global__ void __launch_bounds__(128) k_tc_selftest(float *out, int *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __half *A = reinterpret_cast<__half *>(sm);                // cores (mc, kc) at (kc*16 + mc)*128 B
    __half *B = reinterpret_cast<__half *>(sm + 36 * 1024);    // cores (nc, kc) at (kc*2 + nc)*128 B
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 44 * 1024);
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(sm + 44 * 1024 + 16);
    int *flag = reinterpret_cast<int *>(sm + 44 * 1024 + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 36 * 1024 / 2; i += 128) A[i] = __float2half(0.f);
    for (int i = tid; i < 8 * 1024 / 2; i += 128) B[i] = __float2half(0.f);
    __syncthreads();
    for (int i = tid; i < 128 * 16; i += 128) {
        const int m = i / 16, k = i % 16;
        const int mc = m / 8, r = m % 8, kc = k / 8, j = k % 8;
        A[((kc * 16 + mc) * 128 + r * 16 + j * 2) / 2] = __float2half((float)((m + 3 * k) % 7 - 3));
    }
    for (int i = tid; i < 16 * 16; i += 128) {
        const int n = i / 16, k = i % 16;
        const int nc = n / 8, r = n % 8, kc = k / 8, j = k % 8;
        B[((kc * 2 + nc) * 128 + r * 16 + j * 2) / 2] = __float2half((float)((5 * n + k) % 5 - 2));
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        *flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_base, 32);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tmem_base;
    if (tid == 0) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(A), 16 * 128, 128);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(B), 2 * 128, 128);
        tc::mma_f16(taddr, ad, bd, tc::idesc_f16_f32(128, 16), 0);
        tc::mma_commit(mbar);
        *flag = tc::mbar_wait_bounded(mbar, 0, 1u << 22) ? 1 : -1;
    }
    __syncthreads();
    tc::fence_after_sync();
    if (*flag == 1) {
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
            float v[4];
            tc::tmem_ld4(taddr + ((uint32_t)(warp * 32) << 16) + c, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) out[(warp * 32 + lane) * 16 + c + q] = v[q];
        }
    } else if (tid == 0) {
        status[0] = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

cudaError_t launch_tc_selftest(float *out, int *status, cudaStream_t s) {
    const int smem = 45 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_tc_selftest<<<1, 128, smem, s>>>(out, status);
    return cudaGetLastError();
}

}  // namespace prism
