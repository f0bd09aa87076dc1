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

namespace prism {

// an mbarrier wait gives up (and the kernel reports through its error word) after about 1 s
constexpr long long TC_WAIT_CYCLES = 2000000000LL;

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
// Storage reduction of the S-matrix (PRISM Algorithm section): after the build, each beam's
// real-space exit wave is divided by a power-of-two scale (the smallest power of two above its
// largest |Re| or |Im|, so the division is exact and the values lie in (-1, 1)) and rounded to
// FP16 or BF16.  The layout is pixel-major: pixel j holds (Re, Im) of beams 0..B-1 at
// S16[j*K + 2b], beams B..K/2-1 are zero.  That row is the K dimension of the tensor-core beam
// sum.  Split mode (TC_SPLIT) stores two FP16 rows per pixel, S16[j*2K + 2b] the rounded value hi
// and S16[j*2K + K + 2b] the rounding of the remainder lo = v - hi, so that hi + lo carries about
// 22 significant bits.

enum TcMode { TC_FP16 = 0, TC_BF16 = 1, TC_SPLIT = 2 };

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (BF) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&v);
    } else {
        const __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&v);
    }
}
template <bool BF>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
    if constexpr (BF) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&w);
        return __bfloat1622float2(v);
    } else {
        const __half2 v = *reinterpret_cast<const __half2 *>(&w);
        return __half22float2(v);
    }
}
// (x, y) -> FP16 pair of the values and FP16 pair of their rounding remainders
__device__ __forceinline__ void split2(float x, float y, uint32_t &hi, uint32_t &lo) {
    hi = pack2<false>(x, y);
    const float2 h = unpack2<false>(hi);
    lo = pack2<false>(x - h.x, y - h.y);  // x - h is exact in FP32 (the low bits of x), rounded once
}

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

// ------------------------------------------------------------------ tensor-core PRISM scan
// The beam sum of Eq. PRISMfinal for a group of GX x GY neighbouring probes of the raster is one
// real GEMM on the union tile R of their windows:
//     D[r][n] = sum_k A[r][k] Bc[n][k],   A[r][2b + c] = (Re, Im)_c S16_b(r)   (r in R, M side)
//     Bc[2p][2b] = s_b Re a_bp,  Bc[2p][2b+1] = -s_b Im a_bp,  Bc[2p+1][2b] = s_b Im a_bp,
//     Bc[2p+1][2b+1] = s_b Re a_bp      (a_bp the coefficient of beam b for probe p, s_b its scale)
// so D[r][2p] + i D[r][2p+1] = psi_p(r).  The tile is streamed in M tiles of 128 pixels and K
// chunks (a 2-stage cp.async ring), one thread issues tcgen05.mma (M = 128, N = 2 G, K = 16) into
// one of two TMEM accumulators, all warps drain a finished accumulator (tcgen05.ld) and scatter
// each probe's window pixels to a per-CTA global scratch.  When the group is done the windows come
// back through shared memory for the window FFT, |.|^2 and the bins (the epilogue of the FP32
// path).  A group whose union tile is larger than its windows together is run probe by probe.
// Split mode: A and Bc are each a value part and a remainder part (hi, lo) and every K step issues
// hi*hi + hi*lo + lo*hi into the same FP32 accumulator (the lo*lo term is below FP32 rounding),
// which carries the products to about 22 significant bits.
template <int NW, bool SPLIT = false>
struct TcCfg {
    using FS = FftShape<NW>;
    static constexpr int GX = 8, GY = 4, G = GX * GY, N = 2 * G;
    static constexpr int BLOCK = 256;
    static constexpr int PARTS = SPLIT ? 2 : 1;              // hi (and lo) operand parts
    // ring of K chunks: 3 stages of 96 (a load is issued two steps before its MMAs; K = 272 of the
    // 129-beam set is 3 chunks, as with 2 stages of 128), or 2 of 32 in split mode (its two operand
    // parts fill the shared memory of two CTAs per SM)
    static constexpr int STAGES = SPLIT ? 2 : 3;
    static constexpr int KCMAX = SPLIT ? 32 : 96;            // K (16-bit values) per ring stage
    static constexpr int PART_BYTES = 128 * KCMAX * 2;       // 128 pixels x KCMAX of one part
    static constexpr int STAGE_BYTES = PARTS * PART_BYTES;
    static constexpr int RING = STAGES * STAGE_BYTES;
    static constexpr int PW = NW + 4;                         // window row pitch (bank spread)
    static constexpr int EW = NW >= 64 ? 2 : NW == 32 ? 8 : 16;  // windows per epilogue pass
    static constexpr int T = FS::T;
    static constexpr int RSLOTS = BLOCK / T, CW = BLOCK / T;
    static constexpr int EXR = RSLOTS * FS::N1 * (FS::N2 + 1);
    static constexpr int EXC = FS::N1 * (FS::N2 + 1) * CW;
    static constexpr int EX = EXR > EXC ? EXR : EXC;
    static constexpr size_t EPI = (size_t)(EW * NW * PW + EX) * sizeof(float2);
    static constexpr int META = 256;                        // ints
    static constexpr int META_LAST = META - 1;              // flag: this CTA completed a split block
    static constexpr int MAXP = 16;                         // parts per split block at most
    static constexpr size_t MISC = (size_t)NW * sizeof(float2) + META * sizeof(int) + STAGES * 8 + 16;
    static constexpr uint32_t TMEM_COLS = 2 * N;            // two accumulators
    __host__ __device__ static constexpr size_t bmat_bytes(int kp) { return (size_t)PARTS * kp * N * 2; }
    __host__ __device__ static constexpr size_t region0(int kp) {
        const size_t r = (size_t)RING + bmat_bytes(kp);
        return ((r > EPI ? r : EPI) + 127) & ~(size_t)127;
    }
    __host__ __device__ static constexpr size_t smem(int kp) { return region0(kp) + MISC; }
};
// meta: the layout of raster_group_geometry (scan_common.cuh)


template <int NW, int MODE>
__global__ void __maxnreg__(112) k_scan_tc(const __grid_constant__ ScanArgs a) {
    constexpr bool BF = MODE == TC_BF16, SPLIT = MODE == TC_SPLIT;
    using C = TcCfg<NW, SPLIT>;
    constexpr int G = C::G, N = C::N, GX = C::GX, GY = C::GY, BLOCK = C::BLOCK, PW = C::PW, S = C::STAGES;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int kp = a.kp;
    unsigned char *ring = sm;
    unsigned char *bmat = sm + C::RING;
    float2 *win = reinterpret_cast<float2 *>(sm);  // epilogue: windows, then exchange (aliases ring + bmat)
    float2 *ex = win + C::EW * NW * PW;
    float2 *twf = reinterpret_cast<float2 *>(sm + C::region0(kp));
    int *meta = reinterpret_cast<int *>(twf + NW);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(meta + C::META);
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(mbar + S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint16_t *S16 = reinterpret_cast<const uint16_t *>(a.S16);

    for (int i = tid; i < NW; i += BLOCK) twf[i] = a.tw_fwd[i];
    if (tid == 0) {
        for (int i = 0; i < S; ++i) tc::mbar_init(&mbar[i], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_base, C::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_base;
    const uint32_t idesc = tc::idesc_f16_f32(128, N, BF);
    const uint32_t bbase = tc::smem_u32(bmat);
    const int ngx = (a.scan_px + GX - 1) / GX, ngy = (a.scan_py + GY - 1) / GY;
    const int ngroups = ngx * ngy;
    const int bp = kp / 2;  // beams incl. padding
    uint32_t st = 0;        // pipeline steps issued by this CTA (same value in every thread)
    bool dead = false;  // set uniformly (through __syncthreads_or) once any thread's wait ran out
    int my_fail = 0;

    auto fail = [&]() {
        my_fail = 1;
        if (a.err) atomicOr(a.err, 1);
    };

    // work units as in the FP32 GEMM scan: the blocks of all full rounds whole, the blocks of the
    // last, partial round split into up to MAXP parts of their M tiles (or probes) over the idle
    // CTAs; a split block's windows in a scratch slot of its own ([0, tail)), the CTA slots after
    const int tail = ngroups % gridDim.x, full = ngroups - tail;
    const int parts = tail ? min(C::MAXP, (int)gridDim.x / tail) : 1;
    for (int u = blockIdx.x; u < full + tail * parts && !dead; u += gridDim.x) {
        int grp = u, part = 0, np = 1, slot = tail + blockIdx.x;
        if (u >= full) {
            const int tg = (u - full) / parts;
            grp = full + tg;
            part = u - full - tg * parts;
            np = parts;
            slot = tg;
        }
        const int gy = grp / ngx, gx = grp - gy * ngx;
        // coefficient operand Bc, K-major core matrices: core (k/8, n/8) at ((k/8)(N/8) + n/8) * 128 B
        for (int i = tid; i < G * bp; i += BLOCK) {
            const int p = i / bp, b = i - p * bp;
            const int row = gy * GY + p / GX, col = gx * GX + p % GX;
            float ar = 0.f, ai = 0.f;
            if (row < a.scan_py && col < a.scan_px && b < a.n_beams) {
                const int pr = row * a.scan_px + col;
                double c = a.qx[b] * (a.x0[pr] - a.shift_x) + a.qy[b] * (a.y0[pr] - a.shift_y);
                c -= rint(c);
                float sn, cs;
                sincospif(-2.0f * (float)c, &sn, &cs);
                const float2 v = cmul(__ldg(a.base + b), make_float2(cs, sn));
                const float sc = __ldg(a.beam_scale + b);
                ar = v.x * sc;
                ai = v.y * sc;
            }
            const int k = 2 * b;
            unsigned char *core = bmat + ((k >> 3) * (N / 8)) * 128 + (k & 7) * 2;
            const int n0 = 2 * p, n1 = 2 * p + 1;
            uint32_t *w0 = reinterpret_cast<uint32_t *>(core + (n0 >> 3) * 128 + (n0 & 7) * 16);
            uint32_t *w1 = reinterpret_cast<uint32_t *>(core + (n1 >> 3) * 128 + (n1 & 7) * 16);
            if constexpr (SPLIT) {
                const size_t lo_off = (size_t)kp * N * 2 / sizeof(uint32_t);  // the remainder matrix
                split2(ar, -ai, w0[0], w0[lo_off]);
                split2(ai, ar, w1[0], w1[lo_off]);
            } else {
                *w0 = pack2<BF>(ar, -ai);
                *w1 = pack2<BF>(ai, ar);
            }
        }
        // group geometry (warp 0, one lane per slot): window origins of Eq. RegionBounds, union tile
        if (warp == 0) raster_group_geometry<NW, NW, GX, GY>(a, gx, gy, meta, lane);
        tc::fence_proxy_async();  // Bc was written through the generic proxy; the MMAs read it
        __syncthreads();
        const bool uni = meta[0] != 0;
        const int nkc = (kp + C::KCMAX - 1) / C::KCMAX;
        const int kcs = ((kp + nkc - 1) / nkc + 15) & ~15;
        for (int sg = 0; sg < (uni ? 1 : G) && !dead; ++sg) {
            if (!uni && (meta[136 + sg] < 0 || sg % np != part)) continue;
            const int tw = uni ? meta[1] : NW, th = uni ? meta[2] : NW;
            const int tx0 = uni ? meta[3] : meta[8 + sg], ty0 = uni ? meta[4] : meta[40 + sg];
            const int npx = tw * th, nmt = (npx + 127) / 128;
            // M tiles [m0, m1) of this unit: all, or a split block's share
            const int m0 = uni ? part * nmt / np : 0, m1 = uni ? (part + 1) * nmt / np : nmt;
            const int nsteps = (m1 - m0) * nkc;
            if (nsteps == 0) continue;
            const uint32_t st0 = st;
            // A chunk of local step ls: thread -> pixel m = 16 warp + lane/2 of the M tile, K cores
            // kc = lane%2, lane%2 + 2, ...  (a lane pair reads one 32-byte sector of a pixel; a warp
            // writes 2 x 256 contiguous shared-memory bytes)
            auto load = [&](int ls) {
                if (ls < nsteps) {
                    const int mt = m0 + ls / nkc, c = ls % nkc;
                    const int k0 = c * kcs, kn = min(kcs, kp - k0);
                    const int m = warp * 16 + (lane >> 1);
                    const int idx = mt * 128 + m;
                    if (idx < npx) {
                        const int ty = idx / tw, tx = idx - ty * tw;
                        const size_t gp = (size_t)((ty0 + ty) & (a.ny_s - 1)) * a.nx_s + ((tx0 + tx) & (a.nx_s - 1));
                        const uint16_t *src = S16 + gp * (C::PARTS * kp) + k0;
                        unsigned char *dst = ring + ((st0 + ls) % S) * C::STAGE_BYTES + (m >> 3) * 128 + (m & 7) * 16;
                        for (int kc = lane & 1; kc < kn / 8; kc += 2) {
                            cp_async16(dst + kc * 2048, src + kc * 8);
                            if constexpr (SPLIT) cp_async16(dst + C::PART_BYTES + kc * 2048, src + kp + kc * 8);
                        }
                    }
                }
                cp_async_commit();
            };
            // accumulator of M tile mt -> window scratch of every probe whose window holds the pixel
            auto drain = [&](int mt) {
                tc::fence_after_sync();
                const int q = warp & 3, h = warp >> 2;  // lane quarter, half of the N columns
                const int idx = mt * 128 + 32 * q + lane;
                const int ty = idx / tw, tx = idx - ty * tw;
#pragma unroll
                for (int c16 = 0; c16 < N / 32; ++c16) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((mt & 1) * N + h * (N / 2) + c16 * 16), v);
                    if (idx < npx) {
#pragma unroll
                        for (int pp = 0; pp < 8; ++pp) {
                            const int p = h * (G / 2) + c16 * 8 + pp;
                            const bool act = uni ? meta[136 + p] >= 0 : p == sg;
                            const int wy = ty - (uni ? meta[104 + p] : 0), wx = tx - (uni ? meta[72 + p] : 0);
                            if (act && (unsigned)wy < (unsigned)NW && (unsigned)wx < (unsigned)NW)
                                a.win[((size_t)slot * G + p) * (NW * NW) + wy * NW + wx] = make_float2(v[2 * pp], v[2 * pp + 1]);
                        }
                    }
                }
                tc::fence_before_sync();
            };
#pragma unroll
            for (int l = 0; l < S - 1; ++l) load(l);
            for (int ls = 0; ls < nsteps; ++ls) {
                const uint32_t s = st0 + ls;
                cp_async_wait<S - 2>();
                tc::fence_proxy_async();
                if (__syncthreads_or(my_fail)) {
                    dead = true;
                    break;
                }
                const int mt = m0 + ls / nkc, c = ls % nkc;
                if (tid == 0) {
                    tc::fence_after_sync();
                    const int k0 = c * kcs, kn = min(kcs, kp - k0);
                    const uint32_t abase = tc::smem_u32(ring + (s % S) * C::STAGE_BYTES);
                    for (int j = 0; j < kn / 16; ++j) {
                        const uint32_t d = tmem + (uint32_t)((mt & 1) * N);
                        const uint32_t boff = (uint32_t)((k0 / 16 + j) * 2 * (N / 8)) * 128;
                        const uint64_t ad = tc::smem_desc(abase + j * 4096, 2048, 128);
                        const uint64_t bd = tc::smem_desc(bbase + boff, (N / 8) * 128, 128);
                        tc::mma_f16(d, ad, bd, idesc, (c > 0 || j > 0) ? 1u : 0u);
                        if constexpr (SPLIT) {
                            const uint32_t blo = (uint32_t)((size_t)kp * N * 2);
                            tc::mma_f16(d, ad, tc::smem_desc(bbase + blo + boff, (N / 8) * 128, 128), idesc, 1u);
                            tc::mma_f16(d, tc::smem_desc(abase + C::PART_BYTES + j * 4096, 2048, 128), bd, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&mbar[s % S]);
                }
                // ring slot (s + S - 1) % S was read by step s - 1: wait for its MMAs before refilling it
                if (ls >= 1 && !tc::mbar_wait_bounded(&mbar[(s - 1) % S], ((s - 1) / S) & 1, TC_WAIT_CYCLES)) fail();
                load(ls + S - 1);
                if (c == 0 && mt > m0) drain(mt - 1);  // the previous tile of this unit
            }
            st = st0 + nsteps;
            if (dead) break;
            if (!tc::mbar_wait_bounded(&mbar[(st - 1) % S], ((st - 1) / S) & 1, TC_WAIT_CYCLES)) fail();
            drain(m1 - 1);
            if (__syncthreads_or(my_fail)) dead = true;
        }
        cp_async_wait<0>();
        __syncthreads();  // window scratch written by this CTA is visible to all its threads
        if (dead) break;
        if (np > 1) {
            // split block: count this part done; the part that completes the block runs its epilogue
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const int last = atomicAdd(a.win_cnt + slot, 1) == np - 1;
                if (last) a.win_cnt[slot] = 0;  // all parts counted: zero for the next launch
                __threadfence();
                meta[C::META_LAST] = last;
            }
            __syncthreads();
            if (!meta[C::META_LAST]) continue;
        }
        // epilogue: EW windows at a time through shared memory
        const int nvalid = meta[5];
        for (int e0 = 0; e0 < nvalid; e0 += C::EW) {
            const int ne = min(C::EW, nvalid - e0);
            // the windows in 16-byte pieces (two pixels of a row), every piece in flight at once
            for (int i = tid; i < ne * (NW * NW / 2); i += BLOCK) {
                const int e = i / (NW * NW / 2), u = 2 * (i - e * (NW * NW / 2));
                cp_async16(win + (e * NW + u / NW) * PW + (u & (NW - 1)), a.win + ((size_t)slot * G + meta[168 + e0 + e]) * (NW * NW) + u);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            window_epilogue<NW, NW, BLOCK, C::EW, PW>(a, win, ex, twf, twf, ne, meta + 200 + e0, tid);
            __syncthreads();
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    if (dead && tid == 0 && st > 0) tc::mbar_wait_bounded(&mbar[(st - 1) % S], ((st - 1) / S) & 1, TC_WAIT_CYCLES);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

bool scan_tc_supported(int nw) { return nw == 16 || nw == 32 || nw == 64; }

template <int NW, int MODE>
static int tc_grid(int kp, int scan_px, int scan_py) {
    using C = TcCfg<NW, MODE == TC_SPLIT>;
    const size_t smem = C::smem(kp);
    if (smem > 227 * 1024) return 0;
    if (allow_max_dynamic_smem(k_scan_tc<NW, MODE>) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_scan_tc<NW, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        return 0;
    // Resident CTAs per SM from the kernel's own limits.  The runtime's occupancy query reports one
    // CTA per SM for every kernel that uses tcgen05, but CTAs whose registers, shared memory and
    // TMEM columns fit do run side by side (each allocates TMEM_COLS of the SM's 512 columns; an
    // allocation that does not fit waits for another CTA to free its columns).
    cudaFuncAttributes fa;
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&fa, k_scan_tc<NW, MODE>) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    const int by_regs = regs_sm / (((fa.numRegs + 7) & ~7) * C::BLOCK);
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + reserved);
    const int by_tmem = 512 / (int)C::TMEM_COLS;
    const int per_sm = std::min(std::min(by_regs, by_smem), std::min(by_tmem, 2048 / C::BLOCK));
    if (per_sm < 1) return 0;
    const long long groups = (long long)((scan_px + C::GX - 1) / C::GX) * ((scan_py + C::GY - 1) / C::GY);
    return (int)std::max<long long>(1, std::min<long long>(groups * C::MAXP, (long long)per_sm * sms));
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

int scan_tc_grid(int nw, int kp, int mode, int scan_px, int scan_py) {
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

template <int NW, int MODE>
static cudaError_t tc_launch(int grid, const ScanArgs &a, cudaStream_t s) {
    using C = TcCfg<NW, MODE == TC_SPLIT>;
    const size_t smem = C::smem(a.kp);
    cudaError_t e = allow_max_dynamic_smem(k_scan_tc<NW, MODE>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_scan_tc<NW, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    k_scan_tc<NW, MODE><<<grid, C::BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NW>
static cudaError_t tc_launch_mode(int mode, int grid, const ScanArgs &a, cudaStream_t s) {
    switch (mode) {
        case TC_FP16: return tc_launch<NW, TC_FP16>(grid, a, s);
        case TC_BF16: return tc_launch<NW, TC_BF16>(grid, a, s);
        case TC_SPLIT: return tc_launch<NW, TC_SPLIT>(grid, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_scan_tc(int nw, int mode, int grid, const ScanArgs &a, cudaStream_t s) {
    if (grid <= 0 || a.kp % 16 || a.kp < 2 * a.n_beams || !a.S16 || !a.beam_scale || !a.win || !a.win_cnt) return cudaErrorInvalidValue;
    switch (nw) {
        case 16: return tc_launch_mode<16>(mode, grid, a, s);
        case 32: return tc_launch_mode<32>(mode, grid, a, s);
        case 64: return tc_launch_mode<64>(mode, grid, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace prism
