// kernels_build.cu -- multislice kernels for sm_103a: slice transmission, the row pass
// (row IFFT, x t_p, row FFT) and the column pass (column FFT, x propagator, column IFFT),
// used both by the compact S-matrix build and by the per-probe multislice baseline.
//
// One multislice step (Eq. Multislice, transmit then propagate) is split into two streaming
// passes over a wave stack [batch][ny][nx] kept in the mixed domain (x-Fourier, y-real):
//   row pass p   : psi_p = IFFT_x(Phi_{p-1});  Z_p = FFT_x(psi_p * t_p)
//   column pass p: Phi_p = IFFT_y( P_p(q) * FFT_y(Z_p) ) / (nx ny)
// so that IFFT_x(Phi_p) is the real-space wave after slice p.  Each pass reads and writes the
// stack once; the 1/(nx ny) of the inverse transform is folded into the propagator table.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"

namespace prism {

// ------------------------------------------------------------------ transmission (t = e^{i sigma V})
// The phase sigma*V is formed in FP64 and reduced to [-1/2, 1/2) cycles before the FP32 sincos.
__global__ void __launch_bounds__(256) k_transmission(const float4 *__restrict__ V, float4 *__restrict__ t,
                                                      size_t n4, double sigma_cycles) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = V[i];
        float vv[4] = {v.x, v.y, v.z, v.w};
        float2 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double c = sigma_cycles * (double)vv[k];
            c -= rint(c);
            float s, co;
            sincospif(2.0f * (float)c, &s, &co);
            o[k] = make_float2(co, s);
        }
        t[2 * i] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        t[2 * i + 1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    }
}

cudaError_t launch_transmission(const float *V, float2 *t, size_t n, double sigma_cycles, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t n4 = n / 4;  // n = H * nx * ny is a multiple of 256
    size_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_transmission<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(V),
                                                     reinterpret_cast<float4 *>(t), n4, sigma_cycles);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ row pass
template <int NX>
struct RowCfg {
    using FS = FftShape<NX>;
    static constexpr int T = FS::T;
    static constexpr int SLOTS = 256 / T;  // rows per CTA
    static constexpr int EXF = FS::N1 * (FS::N2 + 1);
    static constexpr int EXI = FS::N2 * (FS::N1 + 1);
    static constexpr int EX = EXF > EXI ? EXF : EXI;
    static constexpr size_t SMEM = (size_t)SLOTS * EX * sizeof(float2);
};

template <int NX, int MODE>
__global__ void __launch_bounds__(256) k_row(const __grid_constant__ RowArgs a) {
    using C = RowCfg<NX>;
    using FS = FftShape<NX>;
    using Fwd = FwdFft<NX>;
    using Inv = InvFft<NX>;
    constexpr int T = C::T, E = FS::E;
    extern __shared__ float2 smem[];
    const int slot = threadIdx.x / T, t = threadIdx.x % T;
    int row = blockIdx.x * C::SLOTS + slot;
    const bool valid = row < a.n_rows;
    if (!valid) row = a.n_rows - 1;  // lanes of a partial CTA redo a valid row and skip the store
    float2 *exbuf = smem + slot * C::EX;
    WarpExchange<FS::N1, FS::N2, T> exF{exbuf};
    WarpExchange<FS::N2, FS::N1, T> exI{exbuf};

    int b, y;
    if (MODE == ROW_OUT && a.downsample == 2) {
        const int nyh = a.ny >> 1;
        b = row / nyh;
        y = 2 * (row - b * nyh);
    } else {
        b = row / a.ny;
        y = row - b * a.ny;
    }
    float2 *wrow = a.wave + ((size_t)b * a.ny + y) * NX;
    float2 v[E];

    if constexpr (MODE == ROW_PLANE) {
        // psi_b(r) = exp(2 pi i (m f x / nx + n f y / ny)), phase reduced exactly in integers
        const int m = a.beam_mn[2 * (a.beam0 + b)];
        const int n = a.beam_mn[2 * (a.beam0 + b) + 1];
        const long long den = (long long)NX * a.ny;
        long long ky = ((long long)n * a.f * y) % a.ny;
        if (ky < 0) ky += a.ny;
        const long long yterm = ky * NX;
        const float inv_den = 1.0f / (float)den;  // den is a power of two: exact
        const float2 *tp = a.trans + (size_t)y * NX;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int x = Fwd::in_elem(r, t);
            long long kx = ((long long)m * a.f * x) % NX;
            if (kx < 0) kx += NX;
            long long num = kx * a.ny + yterm;
            if (num >= den) num -= den;
            float s, c;
            sincospif(2.0f * ((float)num * inv_den), &s, &c);
            v[r] = cmul(make_float2(c, s), __ldg(tp + x));
        }
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = wrow[Inv::in_elem(r, t)];
        Inv::run(v, t, a.tw_inv, a.tw, exI);
        if constexpr (MODE == ROW_STD) {
            const float2 *tp = a.trans + (size_t)y * NX;
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = cmul(v[r], __ldg(tp + Inv::out_elem(r, t)));
        }
    }

    if constexpr (MODE == ROW_OUT) {
        // real-space exit wave; with downsample 2 the band limit (|k| < n/4) makes every second
        // sample the exact half-resolution wave of the inner Fourier square
        if (!valid) return;
        if (a.downsample == 2) {
            const int nxs = NX / 2, nys = a.ny / 2;
            float2 *srow = a.s_out + ((size_t)(a.beam0 + b) * nys + (y >> 1)) * nxs;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int x = Inv::out_elem(r, t);
                if (!(x & 1)) srow[x >> 1] = v[r];
            }
        } else {
            float2 *srow = a.s_out + ((size_t)(a.beam0 + b) * a.ny + y) * NX;
#pragma unroll
            for (int r = 0; r < E; ++r) srow[Inv::out_elem(r, t)] = v[r];
        }
    } else {
        Fwd::run(v, t, a.tw_fwd, a.tw, exF);
        if (valid) {
#pragma unroll
            for (int r = 0; r < E; ++r) wrow[Fwd::out_elem(r, t)] = v[r];
        }
    }
}

template <class K>
static cudaError_t set_smem(K kernel, size_t smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <int NX>
static cudaError_t row_dispatch(RowMode mode, const RowArgs &a, cudaStream_t s) {
    using C = RowCfg<NX>;
    if (a.n_rows <= 0) return cudaSuccess;
    const dim3 grid((a.n_rows + C::SLOTS - 1) / C::SLOTS);
    cudaError_t e;
    switch (mode) {
        case ROW_STD:
            if ((e = set_smem(k_row<NX, ROW_STD>, C::SMEM)) != cudaSuccess) return e;
            k_row<NX, ROW_STD><<<grid, 256, C::SMEM, s>>>(a);
            break;
        case ROW_PLANE:
            if ((e = set_smem(k_row<NX, ROW_PLANE>, C::SMEM)) != cudaSuccess) return e;
            k_row<NX, ROW_PLANE><<<grid, 256, C::SMEM, s>>>(a);
            break;
        case ROW_OUT:
            if ((e = set_smem(k_row<NX, ROW_OUT>, C::SMEM)) != cudaSuccess) return e;
            k_row<NX, ROW_OUT><<<grid, 256, C::SMEM, s>>>(a);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_row(int nx, RowMode mode, const RowArgs &a, cudaStream_t s) {
    switch (nx) {
        case 16: return row_dispatch<16>(mode, a, s);
        case 32: return row_dispatch<32>(mode, a, s);
        case 64: return row_dispatch<64>(mode, a, s);
        case 128: return row_dispatch<128>(mode, a, s);
        case 256: return row_dispatch<256>(mode, a, s);
        case 512: return row_dispatch<512>(mode, a, s);
        case 1024: return row_dispatch<1024>(mode, a, s);
        case 2048: return row_dispatch<2048>(mode, a, s);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ column pass
template <int NY>
struct ColCfg {
    using FS = FftShape<NY>;
    static constexpr int W = NY >= 2048 ? 4 : NY >= 1024 ? 8 : 16;  // interleaved columns per CTA
    static constexpr int THREADS = FS::T * W;
    static constexpr size_t SMEM = (size_t)NY * W * sizeof(float2);
};

template <int NY, int MODE>
__global__ void __launch_bounds__(ColCfg<NY>::THREADS) k_col(const __grid_constant__ ColArgs a) {
    using C = ColCfg<NY>;
    using FS = FftShape<NY>;
    using Fwd = FwdFft<NY>;
    using Inv = InvFft<NY>;
    constexpr int W = C::W, E = FS::E;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int kx = blockIdx.x * W + c;
    const int b = blockIdx.y;
    float2 *col = a.wave + (size_t)b * NY * a.nx + kx;
    ColExchange<FS::N1, FS::N2, W> exF{smem, c};
    ColExchange<FS::N2, FS::N1, W> exI{smem, c};
    float2 v[E];

    if constexpr (MODE == COL_PROBE) {
        // Psi0(q) = A(q) e^{-i chi(q)} e^{-2 pi i q.r0}, generated in the inverse transform's input layout
        const float2 sx = a.shift_x[(size_t)b * a.nx + kx];
        const float2 *sy = a.shift_y + (size_t)b * NY;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int ky = Inv::in_elem(r, t);
            v[r] = cmul(cmul(__ldg(a.probe_base + (size_t)ky * a.nx + kx), sx), __ldg(sy + ky));
        }
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = col[(size_t)Fwd::in_elem(r, t) * a.nx];
        Fwd::run(v, t, a.tw_fwd, a.tw, exF);
        // Fresnel propagator exp(-i pi lambda t |q|^2) (separable) inside the anti-aliasing aperture
        const int kxs = kx < (a.nx >> 1) ? kx : kx - a.nx;
        const int akx = kxs < 0 ? -kxs : kxs;
        const float2 px = __ldg(a.prop_x + kx);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int ky = Fwd::out_elem(r, t);
            v[r] = (akx <= __ldg(a.aa_kmax + ky)) ? cmul(v[r], cmul(px, __ldg(a.prop_y + ky))) : make_float2(0.f, 0.f);
        }
        if constexpr (MODE == COL_DETECT) {
            float *icol = a.inten + (size_t)b * NY * a.nx + kx;
#pragma unroll
            for (int r = 0; r < E; ++r) icol[(size_t)Fwd::out_elem(r, t) * a.nx] = v[r].x * v[r].x + v[r].y * v[r].y;
            return;
        }
    }
    Inv::run(v, t, a.tw_inv, a.tw, exI);
    if constexpr (MODE == COL_PROBE) {
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = cscale(v[r], a.probe_scale);
    }
#pragma unroll
    for (int r = 0; r < E; ++r) col[(size_t)Inv::out_elem(r, t) * a.nx] = v[r];
}

template <int NY>
static cudaError_t col_dispatch(ColMode mode, const ColArgs &a, cudaStream_t s) {
    using C = ColCfg<NY>;
    if (a.batch <= 0) return cudaSuccess;
    if (a.nx % C::W) return cudaErrorInvalidValue;
    const dim3 grid(a.nx / C::W, a.batch);
    cudaError_t e;
    switch (mode) {
        case COL_STD:
            if ((e = set_smem(k_col<NY, COL_STD>, C::SMEM)) != cudaSuccess) return e;
            k_col<NY, COL_STD><<<grid, C::THREADS, C::SMEM, s>>>(a);
            break;
        case COL_PROBE:
            if ((e = set_smem(k_col<NY, COL_PROBE>, C::SMEM)) != cudaSuccess) return e;
            k_col<NY, COL_PROBE><<<grid, C::THREADS, C::SMEM, s>>>(a);
            break;
        case COL_DETECT:
            if ((e = set_smem(k_col<NY, COL_DETECT>, C::SMEM)) != cudaSuccess) return e;
            k_col<NY, COL_DETECT><<<grid, C::THREADS, C::SMEM, s>>>(a);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_col(int ny, ColMode mode, const ColArgs &a, cudaStream_t s) {
    switch (ny) {
        case 16: return col_dispatch<16>(mode, a, s);
        case 32: return col_dispatch<32>(mode, a, s);
        case 64: return col_dispatch<64>(mode, a, s);
        case 128: return col_dispatch<128>(mode, a, s);
        case 256: return col_dispatch<256>(mode, a, s);
        case 512: return col_dispatch<512>(mode, a, s);
        case 1024: return col_dispatch<1024>(mode, a, s);
        case 2048: return col_dispatch<2048>(mode, a, s);
        default: return cudaErrorInvalidValue;
    }
}

bool row_supported(int n) { return n >= 16 && n <= 2048 && (n & (n - 1)) == 0; }
bool col_supported(int n) { return row_supported(n); }

void fft_split(int n, int *n1, int *n2) {
    int a = 0;
    switch (n) {
        case 8: a = FftShape<8>::N1; break;
        case 16: a = FftShape<16>::N1; break;
        case 32: a = FftShape<32>::N1; break;
        case 64: a = FftShape<64>::N1; break;
        case 128: a = FftShape<128>::N1; break;
        case 256: a = FftShape<256>::N1; break;
        case 512: a = FftShape<512>::N1; break;
        case 1024: a = FftShape<1024>::N1; break;
        case 2048: a = FftShape<2048>::N1; break;
        default: a = 0;
    }
    *n1 = a;
    *n2 = a ? n / a : 0;
}

// ------------------------------------------------------------------ probe shift phases
// shift_x[b][k] = exp(-2 pi i (k/cell_x) x0_b); the phase is reduced in FP64 before FP32 sincos.
__global__ void k_shift(const __grid_constant__ ShiftArgs a) {
    const int b = blockIdx.y;
    const double x0 = a.x0[b], y0 = a.y0[b];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nx + a.ny; i += gridDim.x * blockDim.x) {
        const bool isx = i < a.nx;
        const int k = isx ? i : i - a.nx;
        const int n = isx ? a.nx : a.ny;
        const int ks = k < (n >> 1) ? k : k - n;
        const double q = (double)ks / (isx ? a.cell_x : a.cell_y);
        double c = q * (isx ? x0 : y0);
        c -= rint(c);
        float s, co;
        sincospif(-2.0f * (float)c, &s, &co);
        if (isx)
            a.shift_x[(size_t)b * a.nx + k] = make_float2(co, s);
        else
            a.shift_y[(size_t)b * a.ny + k] = make_float2(co, s);
    }
}

cudaError_t launch_shift(const ShiftArgs &a, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    const dim3 grid((a.nx + a.ny + 255) / 256, a.batch);
    k_shift<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ detector bins
// out[b][k] = scale * sum_{pixels in bin k} inten[b][pixel]: one warp per bin, FP64 lane sums in a
// fixed order and a fixed xor-shuffle tree (bitwise reproducible).
__global__ void __launch_bounds__(256) k_bins(const __grid_constant__ BinArgs a) {
    const int b = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *img = a.inten + (size_t)b * a.npix;
    for (int k = warp; k < a.nbins; k += 8) {
        double s = 0.0;
        const int e = a.bin_off[k + 1];
        for (int i = a.bin_off[k] + lane; i < e; i += 32) s += (double)__ldg(img + __ldg(a.bin_idx + i));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) a.out[(size_t)b * a.nbins + k] = (float)(s * a.scale);
    }
}

cudaError_t launch_bins(const BinArgs &a, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    k_bins<<<a.batch, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace prism
