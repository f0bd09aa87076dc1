// kernels_build.cu -- multislice kernels for sm_103a: slice transmission, the row and column
// passes at their default launch shapes (pass_default.cuh; N >= 512 in kernels_pass_<N>.cu), probe
// shift phases and detector bins; used both by the compact S-matrix build and by the per-probe multislice baseline.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"
#include "pass_default.cuh"
#include "pass_kernels.cuh"

namespace prism {

// ------------------------------------------------------------------ transmission (t = e^{i sigma V})
// The phase sigma*V in cycles is reduced to [-1/2, 1/2) before the FP32 sincos, in float-float
// arithmetic (FP64 runs at a small fraction of the FP32 rate on this GPU): sigma = hi + lo (two
// floats, split on the host), p = V hi rounded and its exact error e = fma(V, hi, -p), so that
// (p - rint(p)) + (e + V lo) is the fractional part to about 2^-24 of a cycle (p - rint(p) is
// exact while |p| < 2^23).
__global__ void __launch_bounds__(256) k_transmission(const float4 *__restrict__ V, float4 *__restrict__ t,
                                                      size_t n4, float sig_hi, float sig_lo) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = V[i];
        float vv[4] = {v.x, v.y, v.z, v.w};
        float2 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float p = vv[k] * sig_hi;
            const float e = fmaf(vv[k], sig_hi, -p);
            const float c = (p - rintf(p)) + fmaf(vv[k], sig_lo, e);
            float s, co;
            sincospif(2.0f * c, &s, &co);
            o[k] = make_float2(co, s);
        }
        t[2 * i] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        t[2 * i + 1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    }
}

// ------------------------------------------------------------------ first slice by the shift theorem
// The first row pass of beam (m, n) transforms psi_b t_0 with psi_b = exp(2 pi i (m f x / nx +
// n f_y y / ny)): row by row that is FFT_x(t_0)[kx - m f] exp(2 pi i n f_y y / ny).  So the row
// transform T0 = FFT_x(t_0) is made once per build (a ROW_PLANE pass of the (0, 0) beam that keeps
// every column) and each beam's first-slice rows are T0 shifted by m f columns times the row's y
// phase -- a gather instead of a transform per row.  One CTA per row at a time, threads over its
// kept columns; nx and ny are powers of two, so the index reductions are masks and ky / ny is exact
// in FP32.
__global__ void __launch_bounds__(256) k_plane(const float2 *__restrict__ T0, float2 *__restrict__ wave,
                                               const int *__restrict__ beam_mn, int beam0, int nb, int nx, int ny,
                                               int f, int f_y, int kx_half) {
    const int kept = kx_half > 0 ? 2 * kx_half - 1 : nx;  // kx = 0 .. kh-1 and nx-kh+1 .. nx-1
    // with f even every beam's shift m f is even and the kept runs start on even columns (kh even,
    // or no pruning), so rows go as 16-byte pixel pairs
    const bool pairs = (f & 1) == 0 && (kx_half & 1) == 0 && (nx & 1) == 0;
    const int npairs = kx_half > 0 ? kx_half : nx / 2;  // kh/2 low + kh/2 high pairs, or all
    for (int row = blockIdx.x; row < nb * ny; row += gridDim.x) {
        const int b = row / ny, y = row - b * ny;
        const int m = __ldg(beam_mn + 2 * (beam0 + b)), n = __ldg(beam_mn + 2 * (beam0 + b) + 1);
        const int ky = (int)(((long long)n * f_y * y) & (ny - 1));
        float sn, cs;
        sincospif(2.0f * ((float)ky / (float)ny), &sn, &cs);
        const float2 e = make_float2(cs, sn);
        const float2 *t0 = T0 + (size_t)y * nx;
        float2 *w = wave + (size_t)row * nx;
        const int shift = m * f;
        if (pairs) {
            // pixel pairs (kx, kx + 1), kx even: the low run [0, kh) and the high run from
            // nx - kh, whose first column lies outside the kept band and is written as zero
            const float4 *t4 = reinterpret_cast<const float4 *>(t0);
            float4 *w4 = reinterpret_cast<float4 *>(w);
            for (int j = threadIdx.x; j < npairs; j += blockDim.x) {
                const int kx = kx_half > 0 && 2 * j >= kx_half ? nx - 2 * kx_half + 2 * j : 2 * j;
                const float4 v = __ldg(t4 + (((kx - shift) & (nx - 1)) >> 1));  // shift even: an aligned pair
                float2 lo = cmul(make_float2(v.x, v.y), e), hi = cmul(make_float2(v.z, v.w), e);
                if (kx_half > 0 && kx == nx - kx_half) lo = make_float2(0.f, 0.f);
                w4[kx >> 1] = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
        } else {
            for (int j = threadIdx.x; j < kept; j += blockDim.x) {
                const int kx = kx_half > 0 && j >= kx_half ? nx - 2 * kx_half + 1 + j : j;
                w[kx] = cmul(__ldg(t0 + ((kx - shift) & (nx - 1))), e);
            }
        }
    }
}

cudaError_t launch_plane(const float2 *T0, float2 *wave, const int *beam_mn, int beam0, int nb, int nx, int ny, int f, int f_y,
                         int kx_half, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    if ((nx & (nx - 1)) || (ny & (ny - 1))) return cudaErrorInvalidValue;  // the masks need powers of two
    const int rows = nb * ny;
    k_plane<<<rows < 152 * 8 ? rows : 152 * 8, 256, 0, s>>>(T0, wave, beam_mn, beam0, nb, nx, ny, f, f_y, kx_half);
    return cudaGetLastError();
}

cudaError_t launch_transmission(const float *V, float2 *t, size_t n, double sigma_cycles, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t n4 = n / 4;  // n = H * nx * ny is a multiple of 256
    size_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const float hi = (float)sigma_cycles, lo = (float)(sigma_cycles - (double)hi);
    k_transmission<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(V),
                                                     reinterpret_cast<float4 *>(t), n4, hi, lo);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ default launch shapes
cudaError_t launch_row(int nx, RowMode mode, const RowArgs &a, cudaStream_t s) {
    switch (nx) {
        case 16: return row_dispatch<16>(mode, a, s);
        case 32: return row_dispatch<32>(mode, a, s);
        case 64: return row_dispatch<64>(mode, a, s);
        case 128: return row_dispatch<128>(mode, a, s);
        case 256: return row_dispatch<256>(mode, a, s);
        case 512: return launch_row_n512(mode, a, s);
        case 1024: return launch_row_n1024(mode, a, s);
        case 2048: return launch_row_n2048(mode, a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col(int ny, ColMode mode, const ColArgs &a, cudaStream_t s) {
    switch (ny) {
        case 16: return col_dispatch<16>(mode, a, s);
        case 32: return col_dispatch<32>(mode, a, s);
        case 64: return col_dispatch<64>(mode, a, s);
        case 128: return col_dispatch<128>(mode, a, s);
        case 256: return col_dispatch<256>(mode, a, s);
        case 512: return launch_col_n512(mode, a, s);
        case 1024: return launch_col_n1024(mode, a, s);
        case 2048: return launch_col_n2048(mode, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int NY>
static bool col_geom(int *lanes, int *regs) {
    using Inv = InvFft<NY>;
    static_assert(Inv::I == 1 && Inv::SPLIT1 == Inv::T && Inv::SPLIT2 == Inv::E, "result row = lane + lanes * register");
    *lanes = Inv::T;
    *regs = Inv::E;
    return true;
}

bool col_fft_geometry(int ny, int *lanes, int *regs) {
    switch (ny) {
        case 16: return col_geom<16>(lanes, regs);
        case 32: return col_geom<32>(lanes, regs);
        case 64: return col_geom<64>(lanes, regs);
        case 128: return col_geom<128>(lanes, regs);
        case 256: return col_geom<256>(lanes, regs);
        case 512: return col_geom<512>(lanes, regs);
        case 1024: return col_geom<1024>(lanes, regs);
        case 2048: return col_geom<2048>(lanes, regs);
        default: return false;
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
        // a pass whose bounded wait ran out left this wave incomplete: the result says so (NaN)
        if (lane == 0) a.out[(size_t)b * a.nbins + k] = (a.err && *a.err) ? __int_as_float(0x7fc00000) : (float)(s * a.scale);
    }
}

cudaError_t launch_bins(const BinArgs &a, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    k_bins<<<a.batch, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace prism
