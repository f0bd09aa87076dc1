// kernels_scan.cu -- the PRISM probe scan for sm_103a (PRISM Algorithm section, Fig. 1d-f).
//
// One CTA per probe position r0:
//   1. coefficients alpha_b(r0) = A(q_b) e^{-i chi(q_b)} e^{-2 pi i q_b.r0}; the phase q_b.r0 is
//      formed in FP64 and reduced to [-1/2, 1/2) cycles before the FP32 sincos;
//   2. window origin s = floor(r0 / px' + 1/2) - Nw/2 (mod N') on the stored grid (Eq. RegionBounds);
//   3. beam sum psi(u) = sum_b alpha_b S_b(s + u) over the Nw x Nw window, wrapped (Eq. PRISMfinal),
//      each thread accumulating a fixed set of window pixels in registers;
//   4. 2-D FFT of the window in shared memory (row then column two-level FFTs);
//   5. |Psi|^2 and the annular bins: one warp per bin, FP64 sums in a fixed order.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"

namespace prism {

template <int NW>
struct ScanCfg {
    using FS = FftShape<NW>;
    static constexpr int BLOCK = NW <= 8 ? 64 : NW >= 128 ? 512 : 256;
    static constexpr int PIX = NW * NW / BLOCK;       // window pixels per thread
    static constexpr int T = FS::T;
    static constexpr int RSLOTS = BLOCK / T;          // window rows transformed at once
    static constexpr int CW = BLOCK / T;              // window columns transformed at once
    static constexpr int EXR = RSLOTS * FS::N1 * (FS::N2 + 1);
    static constexpr int EXC = NW * CW;
    static constexpr int EX = EXR > EXC ? EXR : EXC;
    static_assert(2 * EX >= NW * NW, "exchange region doubles as the intensity buffer");
    static constexpr size_t SMEM_FIXED = (size_t)(NW * NW + EX) * sizeof(float2);
};

template <int NW>
__global__ void __launch_bounds__(ScanCfg<NW>::BLOCK) k_scan(const __grid_constant__ ScanArgs a) {
    using C = ScanCfg<NW>;
    using FS = FftShape<NW>;
    using Fwd = FwdFft<NW>;
    constexpr int BLOCK = C::BLOCK, PIX = C::PIX, T = C::T, E = FS::E;
    extern __shared__ float2 smem[];
    float2 *win = smem;                 // [NW][NW]
    float2 *ex = win + NW * NW;         // exchange, later |Psi|^2 as float
    float2 *alpha = ex + C::EX;         // [n_beams]
    const int tid = threadIdx.x;
    const int p = a.probe0 + blockIdx.x;
    if (p >= a.n_probes) return;
    const double x0 = a.x0[p], y0 = a.y0[p];

    // 1. coefficients
    for (int b = tid; b < a.n_beams; b += BLOCK) {
        double c = a.qx[b] * x0 + a.qy[b] * y0;
        c -= rint(c);
        float s, co;
        sincospif(-2.0f * (float)c, &s, &co);
        alpha[b] = cmul(__ldg(a.base + b), make_float2(co, s));
    }
    // 2. window origin, FP64 as in the definition
    const int sx = ((int)floor(x0 / a.px_s + 0.5) - NW / 2) & (a.nx_s - 1);
    const int sy = ((int)floor(y0 / a.py_s + 0.5) - NW / 2) & (a.ny_s - 1);
    __syncthreads();

    // 3. gather + beam contraction
    int off[PIX];
    float2 acc[PIX];
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int u = tid + k * BLOCK;
        const int v = u / NW, c = u % NW;
        off[k] = ((sy + v) & (a.ny_s - 1)) * a.nx_s + ((sx + c) & (a.nx_s - 1));
        acc[k] = make_float2(0.f, 0.f);
    }
    const size_t bstride = (size_t)a.ny_s * a.nx_s;
    const float2 *Sb = a.S;
    for (int b = 0; b < a.n_beams; ++b, Sb += bstride) {
        const float2 al = alpha[b];
#pragma unroll
        for (int k = 0; k < PIX; ++k) {
            const float2 s = __ldg(Sb + off[k]);
            acc[k].x = fmaf(al.x, s.x, fmaf(-al.y, s.y, acc[k].x));
            acc[k].y = fmaf(al.x, s.y, fmaf(al.y, s.x, acc[k].y));
        }
    }
#pragma unroll
    for (int k = 0; k < PIX; ++k) win[tid + k * BLOCK] = acc[k];
    __syncthreads();

    // 4a. row FFTs
    {
        const int slot = tid / T, t = tid % T;
        WarpExchange<FS::N1, FS::N2, T> exr{ex + slot * (FS::N1 * (FS::N2 + 1))};
#pragma unroll 1
        for (int r0 = 0; r0 < NW; r0 += C::RSLOTS) {
            const int row = r0 + slot;
            const int rr = row < NW ? row : row % NW;  // surplus lanes repeat a row, no store
            float2 v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = win[rr * NW + Fwd::in_elem(r, t)];
            Fwd::run(v, t, a.tw_fwd, a.tw, exr);
            if (row < NW) {
#pragma unroll
                for (int r = 0; r < E; ++r) win[rr * NW + Fwd::out_elem(r, t)] = v[r];
            }
        }
    }
    __syncthreads();
    // 4b. column FFTs
    {
        const int c = tid % C::CW, t = tid / C::CW;
        ColExchange<FS::N1, FS::N2, C::CW> exc{ex, c};
#pragma unroll 1
        for (int c0 = 0; c0 < NW; c0 += C::CW) {
            const int col = c0 + c;
            const int cc = col < NW ? col : col % NW;
            float2 v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = win[Fwd::in_elem(r, t) * NW + cc];
            Fwd::run(v, t, a.tw_fwd, a.tw, exc);
            __syncthreads();  // all reads of win for this pass done before any write
            if (col < NW) {
#pragma unroll
                for (int r = 0; r < E; ++r) win[Fwd::out_elem(r, t) * NW + cc] = v[r];
            }
        }
    }
    __syncthreads();

    // 5. |Psi|^2 and annular bins
    float *inten = reinterpret_cast<float *>(ex);
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const float2 z = win[tid + k * BLOCK];
        inten[tid + k * BLOCK] = z.x * z.x + z.y * z.y;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int k = warp; k < a.nbins; k += BLOCK / 32) {
        double s = 0.0;
        const int e = __ldg(a.bin_off + k + 1);
        for (int i = __ldg(a.bin_off + k) + lane; i < e; i += 32) s += (double)inten[__ldg(a.bin_idx + i)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) a.out[(size_t)p * a.nbins + k] = (float)(s * a.inv_norm);
    }
}

template <int NW>
static cudaError_t scan_dispatch(const ScanArgs &a, cudaStream_t s) {
    using C = ScanCfg<NW>;
    const int n = a.n_probes - a.probe0;
    if (n <= 0) return cudaSuccess;
    const size_t smem = C::SMEM_FIXED + (size_t)a.n_beams * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_scan<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_scan<NW><<<n, C::BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(int nw, const ScanArgs &a, cudaStream_t s) {
    switch (nw) {
        case 8: return scan_dispatch<8>(a, s);
        case 16: return scan_dispatch<16>(a, s);
        case 32: return scan_dispatch<32>(a, s);
        case 64: return scan_dispatch<64>(a, s);
        case 128: return scan_dispatch<128>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

bool scan_supported(int nw) { return nw == 8 || nw == 16 || nw == 32 || nw == 64 || nw == 128; }

size_t scan_smem_bytes(int nw, int n_beams) {
    size_t fixed = 0;
    switch (nw) {
        case 8: fixed = ScanCfg<8>::SMEM_FIXED; break;
        case 16: fixed = ScanCfg<16>::SMEM_FIXED; break;
        case 32: fixed = ScanCfg<32>::SMEM_FIXED; break;
        case 64: fixed = ScanCfg<64>::SMEM_FIXED; break;
        case 128: fixed = ScanCfg<128>::SMEM_FIXED; break;
        default: return 0;
    }
    return fixed + (size_t)n_beams * sizeof(float2);
}

}  // namespace prism
