// kernels_tc.cu -- tensor-core (tcgen05) kernels: a layout self-test and the reduced-precision
// PRISM beam contraction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "fft.cuh"
#include "params.h"
#include "scan_common.cuh"
#include "tc.cuh"
#include "scan_tc.cuh"  // k_scan_tc, TcMode, the 16-bit packing helpers

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
        *flag = tc::mbar_wait_bounded(mbar, 0, TC_WAIT_CYCLES) ? 1 : -1;
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

// ------------------------------------------------------------------ bounded-wait diagnostic
// The waits of the tensor-core scan and of the TMA-staged passes are mbarrier waits that give up
// after a clock budget.  This kernel makes one run out on purpose without any fault: one CTA
// initialises a barrier expecting one arrival, thread 0 arrives or not (`arrive`), and every thread
// waits for the barrier's first phase for at most `limit_cycles`.  status[0] = 1 if the wait ran
// out (no arrival: the expected outcome), 0 if the phase completed.
__device__ __forceinline__ void mbar_arrive_once(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(mbar)) : "memory");
}

__global__ void __launch_bounds__(128) k_wait_selftest(int *status, long long limit_cycles, int arrive) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) mbar_arrive_once(&bar);
    const bool done = tc::mbar_wait_bounded(&bar, 0, limit_cycles);
    if (__syncthreads_or(!done) && threadIdx.x == 0) status[0] = 1;
}

cudaError_t launch_wait_selftest(int *status, long long limit_cycles, int arrive, cudaStream_t s) {
    if (limit_cycles < 0 || limit_cycles > 4000000000LL) return cudaErrorInvalidValue;
    k_wait_selftest<<<1, 128, 0, s>>>(status, limit_cycles, arrive);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ 16-bit S-matrix
// (storage layout and the packing helpers: scan_tc.cuh)

// smallest power of two strictly above x >= 0 (1 for x == 0), from the exponent field
__device__ __forceinline__ float pow2_above(float x) {
    if (!(x > 0.f)) return 1.f;
    unsigned e = __float_as_uint(x) >> 23;  // biased exponent (x is non-negative)
    e = e < 253u ? e + 1u : 254u;
    return __uint_as_float(e << 23);
}

// one CTA per beam: scale[beam0 + b] = pow2_above(max |Re|, |Im| over the beam)
__global__ void __launch_bounds__(512) k_beam_scale(const QuantArgs a) {
    __shared__ float red[16];
    const int b = blockIdx.x;
    const float2 *src = a.S + (size_t)b * a.npix;
    float m = 0.f;
    for (int i = threadIdx.x; i < a.npix; i += 512) {
        const float2 v = src[i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < 16 ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) a.scale[a.beam0 + b] = pow2_above(m);
    }
}

// 32 pixels x 32 beams per tile through shared memory: coalesced reads along pixels of one beam,
// coalesced 4-byte (Re, Im) writes along the beams of one pixel
template <int MODE>
__global__ void __launch_bounds__(256) k_quantize(const QuantArgs a) {
    __shared__ float2 tile[32][33];
    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int pix0 = blockIdx.x * 32;
    const size_t row = (size_t)(MODE == TC_SPLIT ? 2 : 1) * a.kp / 2;  // 32-bit words per pixel
    for (int c0 = 0; c0 < a.nb; c0 += 32) {
        for (int j = ty; j < 32; j += 8) {
            const int b = c0 + j;
            tile[j][lane] = b < a.nb && pix0 + lane < a.npix ? a.S[(size_t)b * a.npix + pix0 + lane] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int b = c0 + lane;
        if (b < a.nb) {
            const float inv = 1.0f / a.scale[a.beam0 + b];  // exact: a power of two
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.S16);
            for (int p = ty; p < 32; p += 8) {
                if (pix0 + p >= a.npix) break;
                const float2 v = tile[lane][p];
                uint32_t *d = dst + (size_t)(pix0 + p) * row + a.beam0 + b;
                if constexpr (MODE == TC_SPLIT) {
                    uint32_t hi, lo;
                    split2(v.x * inv, v.y * inv, hi, lo);
                    d[0] = hi;
                    d[a.kp / 2] = lo;
                } else {
                    d[0] = pack2<MODE == TC_BF16>(v.x * inv, v.y * inv);
                }
            }
        }
        __syncthreads();
    }
}

template <int MODE>
__global__ void k_dequantize(const uint32_t *S16, const float *scale, float2 *out, int n_beams, int npix, int kp) {
    const size_t n = (size_t)n_beams * npix;
    const size_t row = (size_t)(MODE == TC_SPLIT ? 2 : 1) * kp / 2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / npix);
        const size_t j = i - (size_t)b * npix;
        float2 v = unpack2<MODE == TC_BF16>(S16[j * row + b]);
        if constexpr (MODE == TC_SPLIT) {
            const float2 l = unpack2<false>(S16[j * row + kp / 2 + b]);
            v = make_float2(v.x + l.x, v.y + l.y);
        }
        out[i] = make_float2(v.x * scale[b], v.y * scale[b]);
    }
}

cudaError_t launch_quantize(const QuantArgs &a, cudaStream_t s) {
    if (a.nb <= 0) return cudaSuccess;
    k_beam_scale<<<a.nb, 512, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int blocks = (a.npix + 31) / 32;
    switch (a.mode) {
        case TC_FP16: k_quantize<TC_FP16><<<blocks, 256, 0, s>>>(a); break;
        case TC_BF16: k_quantize<TC_BF16><<<blocks, 256, 0, s>>>(a); break;
        case TC_SPLIT: k_quantize<TC_SPLIT><<<blocks, 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_dequantize(const void *S16, const float *scale, float2 *out, int n_beams, int npix, int kp, int mode,
                              cudaStream_t s) {
    const size_t n = (size_t)n_beams * npix;
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    const uint32_t *src = (const uint32_t *)S16;
    switch (mode) {
        case TC_FP16: k_dequantize<TC_FP16><<<blocks, 256, 0, s>>>(src, scale, out, n_beams, npix, kp); break;
        case TC_BF16: k_dequantize<TC_BF16><<<blocks, 256, 0, s>>>(src, scale, out, n_beams, npix, kp); break;
        case TC_SPLIT: k_dequantize<TC_SPLIT><<<blocks, 256, 0, s>>>(src, scale, out, n_beams, npix, kp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool scan_tc_supported(int nw) { return nw == 16 || nw == 32 || nw == 64; }

int scan_tc_shapes(int mode) { return mode == TC_SPLIT ? 1 : N_TC_SHAPES; }

const char *scan_tc_shape_name(int shape) {
    static const char *names[N_TC_SHAPES] = {"3 x 96 K ring", "2 x 128 K ring", "4 x 64 K ring"};
    return shape >= 0 && shape < N_TC_SHAPES ? names[shape] : "?";
}

template <int NW>
static int tc_grid_mode(int mode, int kp, int px, int py) {
    switch (mode) {
        case TC_FP16: return tc_grid<NW, TC_FP16>(kp, px, py);
        case TC_BF16: return tc_grid<NW, TC_BF16>(kp, px, py);
        case TC_SPLIT: return tc_grid<NW, TC_SPLIT>(kp, px, py);
    }
    return 0;
}

int scan_tc_grid(int nw, int kp, int mode, int shape, int scan_px, int scan_py) {
    if (shape != 0) return scan_tc_grid_tuned(nw, kp, mode, shape, scan_px, scan_py);
    switch (nw) {
        case 16: return tc_grid_mode<16>(mode, kp, scan_px, scan_py);
        case 32: return tc_grid_mode<32>(mode, kp, scan_px, scan_py);
        case 64: return tc_grid_mode<64>(mode, kp, scan_px, scan_py);
        default: return 0;
    }
}

size_t scan_tc_win_bytes(int nw, int grid, int scan_px, int scan_py) {
    using C = TcCfg<16>;
    if (grid <= 0 || scan_px <= 0 || scan_py <= 0) return 0;
    const long long groups = (long long)((scan_px + C::GX - 1) / C::GX) * ((scan_py + C::GY - 1) / C::GY);
    const long long tail = groups % grid, slots = tail + (groups > tail ? grid : 0);  // split blocks, CTAs
    return (size_t)slots * C::G * nw * nw * sizeof(float2);
}
static_assert(TcCfg<16>::G == TcCfg<32>::G && TcCfg<16>::G == TcCfg<64, true>::G, "one group size for every window");

template <int NW>
static cudaError_t tc_launch_mode(int mode, int grid, const ScanArgs &a, cudaStream_t s) {
    switch (mode) {
        case TC_FP16: return tc_launch<NW, TC_FP16>(grid, a, s);
        case TC_BF16: return tc_launch<NW, TC_BF16>(grid, a, s);
        case TC_SPLIT: return tc_launch<NW, TC_SPLIT>(grid, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_scan_tc(int nw, int mode, int shape, int grid, const ScanArgs &a, cudaStream_t s) {
    if (grid <= 0 || a.kp % 16 || a.kp < 2 * a.n_beams || !a.S16 || !a.beam_scale || !a.win || !a.win_cnt) return cudaErrorInvalidValue;
    if (shape != 0) return launch_scan_tc_tuned(nw, mode, shape, grid, a, s);
    switch (nw) {
        case 16: return tc_launch_mode<16>(mode, grid, a, s);
        case 32: return tc_launch_mode<32>(mode, grid, a, s);
        case 64: return tc_launch_mode<64>(mode, grid, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace prism
