// scan_common.cuh -- pieces shared by the grouped PRISM scan kernels (FP32 CUDA-core contraction
// and FP16 tensor-core contraction): async copies, probe-group geometry, coefficients and the
// per-window epilogue (window FFT, full diffraction pattern, annular bins).
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"

namespace prism {

// The dynamic shared memory limit of a scan kernel whose launches differ in size (with the beam
// count): the device's opt-in maximum less the kernel's static shared memory.  The attribute
// belongs to the kernel, not to a launch, so plans scanning from several host threads set this same
// value every time instead of their own sizes, which a concurrent smaller setting would undercut
// between another thread's setting and its launch.
template <class K>
static cudaError_t allow_max_dynamic_smem(K kernel) {
    static const int optin = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 0;
        return v;
    }();
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (optin <= (int)fa.sharedSizeBytes) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
// 16-byte copy through L1 (sectors shared by neighbouring copies are fetched once)
__device__ __forceinline__ void cp_async16_ca(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
// 8-byte copy through L1 (one complex64 pixel)
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Sum over one warp of per-lane FP32 partial sums, fixed xor-shuffle tree (every lane gets the
// total).  Pairwise: relative error <= (terms per lane + 5) * 2^-24 for non-negative terms.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Geometry of a group of up to G consecutive probes (thread 0 only), NWX x NWY windows.  Window
// origins follow Eq. RegionBounds in FP64; the union tile of the group's windows, relative to probe
// 0, starts on an even column with an even width (16-byte aligned pixel pairs).  meta layout:
//   [0] sub-groups (1: whole group on one tile, else one per probe)  [1] tile width  [2] tile height
//   [3] tile x origin  [4] tile y origin  [8+p] window x origin  [16+p] window y origin
//   [24+p] window x offset in the tile  [32+p] window y offset in the tile  [40+p] output row (p0 + p)
template <int NWX, int NWY, int G, int D, int MAXTILE>
__device__ void group_geometry(const ScanArgs &a, int p0, int gn, int *meta) {
    int sx[G], sy[G];
    for (int p = 0; p < gn; ++p) {
        sx[p] = ((int)floor(a.x0[p0 + p] / a.px_s + 0.5) - NWX / 2) & (a.nx_s - 1);
        sy[p] = ((int)floor(a.y0[p0 + p] / a.py_s + 0.5) - NWY / 2) & (a.ny_s - 1);
    }
    int dxmin = 0, dxmax = 0, dymin = 0, dymax = 0, dx[G], dy[G];
    for (int p = 0; p < gn; ++p) {
        dx[p] = ((sx[p] - sx[0] + a.nx_s / 2) & (a.nx_s - 1)) - a.nx_s / 2;
        dy[p] = ((sy[p] - sy[0] + a.ny_s / 2) & (a.ny_s - 1)) - a.ny_s / 2;
        dxmin = min(dxmin, dx[p]);
        dxmax = max(dxmax, dx[p]);
        dymin = min(dymin, dy[p]);
        dymax = max(dymax, dy[p]);
    }
    const int tx0 = (sx[0] + dxmin) & (a.nx_s - 1);
    const int shift = tx0 & 1;  // extra leading column to reach an even origin
    const int tw = (dxmax - dxmin + NWX + shift + 1) & ~1;
    const int th = dymax - dymin + NWY;
    const bool fits = tw <= NWX + D && th <= NWY + D && tw * th <= MAXTILE;
    meta[0] = fits ? 1 : gn;
    for (int p = 0; p < G; ++p) {
        meta[8 + p] = sx[p < gn ? p : 0];
        meta[16 + p] = sy[p < gn ? p : 0];
        meta[24 + p] = p < gn ? dx[p] - dxmin + shift : 0;
        meta[32 + p] = p < gn ? dy[p] - dymin : 0;
        meta[40 + p] = p0 + p;
    }
    meta[1] = tw;
    meta[2] = th;
    meta[3] = tx0 - shift;
    meta[4] = (sy[0] + dymin) & (a.ny_s - 1);
}

// Geometry of a GX x GY block of the probe raster (group gx, gy), NWX x NWY windows; executed by
// one warp, lane p = slot j * GX + i for raster row gy*GY + j, column gx*GX + i (GX*GY <= 32).
// Window origins follow Eq. RegionBounds in FP64; the union tile of the slots' windows is used
// when it is no larger than their windows together, else each probe runs on its own window.  The
// union tile starts on an even column and has an even width (a leading column where the windows
// start on an odd one, a trailing one to an even width), so that its rows are 16-byte aligned runs
// of pixel pairs.
// meta (ints): [0] union tile  [1] tile width  [2] tile height  [3] tile x0  [4] tile y0
// [5] probes in the group; per slot p < 32: [8+p] window x0  [40+p] window y0  [72+p] x offset in
// the tile  [104+p] y offset in the tile  [136+p] probe index or -1; [168+e] slot of the e-th
// probe, [200+e] its probe index
template <int NWX, int NWY, int GX, int GY>
__device__ void raster_group_geometry(const ScanArgs &a, int gx, int gy, int *meta, int lane) {
    constexpr int G = GX * GY;
    const int p = lane;
    const int row = gy * GY + p / GX, col = gx * GX + p % GX;
    const bool valid = p < G && row < a.scan_py && col < a.scan_px;
    int sx = 0, sy = 0;
    if (valid) {
        const int pr = row * a.scan_px + col;
        sx = ((int)floor(a.x0[pr] / a.px_s + 0.5) - NWX / 2) & (a.nx_s - 1);
        sy = ((int)floor(a.y0[pr] / a.py_s + 0.5) - NWY / 2) & (a.ny_s - 1);
    }
    const int sx0 = __shfl_sync(0xffffffffu, sx, 0), sy0 = __shfl_sync(0xffffffffu, sy, 0);
    const int dx = valid ? ((sx - sx0 + a.nx_s / 2) & (a.nx_s - 1)) - a.nx_s / 2 : 0;
    const int dy = valid ? ((sy - sy0 + a.ny_s / 2) & (a.ny_s - 1)) - a.ny_s / 2 : 0;
    const int dxmin = __reduce_min_sync(0xffffffffu, dx), dxmax = __reduce_max_sync(0xffffffffu, dx);
    const int dymin = __reduce_min_sync(0xffffffffu, dy), dymax = __reduce_max_sync(0xffffffffu, dy);
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    const int nvalid = __popc(vm);
    const int tx0 = (sx0 + dxmin) & (a.nx_s - 1), shift = tx0 & 1;
    const int tw = (dxmax - dxmin + NWX + shift + 1) & ~1, th = dymax - dymin + NWY;
    if (p < G) {
        meta[8 + p] = sx;
        meta[40 + p] = sy;
        meta[72 + p] = dx - dxmin + shift;
        meta[104 + p] = dy - dymin;
        meta[136 + p] = valid ? row * a.scan_px + col : -1;
    }
    if (valid) {
        const int e = __popc(vm & ((1u << p) - 1u));
        meta[168 + e] = p;
        meta[200 + e] = row * a.scan_px + col;
    }
    if (lane == 0) {
        meta[0] = (long long)(dxmax - dxmin + NWX) * th <= (long long)nvalid * NWX * NWY;  // before the even padding
        meta[1] = tw;
        meta[2] = th;
        meta[3] = tx0 - shift;
        meta[4] = (sy0 + dymin) & (a.ny_s - 1);
        meta[5] = nvalid;
    }
}

// alpha[p][b] = A(q_b - q_t) e^{-i chi} e^{-2 pi i q_b.(r0_p - h tan theta)} for the group's probes
// (phase in FP64, reduced before the FP32 sincos); zero for probes past the end.
template <int G>
__device__ void group_coefficients(const ScanArgs &a, int p0, int gn, float2 *alpha, int tid, int nthreads) {
    for (int i = tid; i < G * a.n_beams; i += nthreads) {
        const int p = i / a.n_beams, b = i - p * a.n_beams;
        float2 v = make_float2(0.f, 0.f);
        if (p < gn) {
            double c = a.qx[b] * (a.x0[p0 + p] - a.shift_x) + a.qy[b] * (a.y0[p0 + p] - a.shift_y);
            c -= rint(c);
            float s, co;
            sincospif(-2.0f * (float)c, &s, &co);
            v = cmul(__ldg(a.base + b), make_float2(co, s));
        }
        alpha[i] = v;
    }
}

// Window epilogue for nwin windows win[p][NWY][PW] (psi in real space on entry, NWX pixels per
// row): 2-D FFT of every window (rows then columns, two-level FFTs; the stage twiddles of the row
// and column lengths in twx and twy), then the full diffraction pattern (if a.cbed) and the
// annular bins (if a.out).  Window p is written to output row oidx[p] (shared memory).  G bounds
// nwin; ex holds ExSize<NWX, NWY, BLOCK>::value float2.
template <int NWX, int NWY, int BLOCK>
struct ExSize {
    using FX = FftShape<NWX>;
    using FY = FftShape<NWY>;
    static constexpr int EXR = (BLOCK / FX::T) * FX::N1 * (FX::N2 + 1);
    static constexpr int EXC = FY::N1 * (FY::N2 + 1) * (BLOCK / FY::T);
    static constexpr int value = EXR > EXC ? EXR : EXC;
};

template <int NWX, int NWY, int BLOCK, int G, int PW>
__device__ void window_epilogue(const ScanArgs &a, float2 *win, float2 *ex, const float2 *twx, const float2 *twy,
                                int nwin, const int *oidx, int tid, const uint16_t *sidx = nullptr) {
    {
        using FS = FftShape<NWX>;
        using Fwd = FwdFft<NWX>;
        constexpr int T = FS::T, E = FS::E, RSLOTS = BLOCK / T;
        const int slot = tid / T, t = tid % T;
        WarpExchange<FS::N1, FS::N2, T> exr{ex + slot * (FS::N1 * (FS::N2 + 1))};
#pragma unroll 1
        for (int r0 = 0; r0 < G * NWY; r0 += RSLOTS) {
            const int row = r0 + slot;
            const bool ok = row < nwin * NWY;
            const int rr = ok ? row : row % NWY;
            float2 v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = win[rr * PW + Fwd::in_elem(r, t)];
            Fwd::run(v, t, twx, a.tw, exr);
            if (ok) {
#pragma unroll
                for (int r = 0; r < E; ++r) win[rr * PW + Fwd::out_elem(r, t)] = v[r];
            }
        }
    }
    __syncthreads();
    {
        // columns like rows: T lanes of one warp per column, warp-local exchange (with the row pitch
        // PW = 4 mod 16 float2, the T x 32/T lane block of a column access covers every bank pair
        // twice: two wavefronts, the minimum for 8-byte accesses)
        using FS = FftShape<NWY>;
        using Fwd = FwdFft<NWY>;
        constexpr int T = FS::T, E = FS::E, CSLOTS = BLOCK / T;
        const int slot = tid / T, t = tid % T;
        WarpExchange<FS::N1, FS::N2, T> exc{ex + slot * (FS::N1 * (FS::N2 + 1))};
#pragma unroll 1
        for (int c0 = 0; c0 < G * NWX; c0 += CSLOTS) {
            const int col = c0 + slot;
            const bool ok = col < nwin * NWX;
            const int cc = ok ? col : col % NWX;
            float2 *w = win + (cc / NWX) * NWY * PW;
            const int x = cc % NWX;
            float2 v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = w[Fwd::in_elem(r, t) * PW + x];
            Fwd::run(v, t, twy, a.tw, exc);
            if (ok) {
#pragma unroll
                for (int r = 0; r < E; ++r) w[Fwd::out_elem(r, t) * PW + x] = v[r];
            }
        }
    }
    __syncthreads();
    // u = ky * NWX + kx: the row is u >> LNW, LNW = log2(NWX)
    constexpr int LNW = NWX == 8 ? 3 : NWX == 16 ? 4 : NWX == 32 ? 5 : NWX == 64 ? 6 : NWX == 128 ? 7 : -1;
    static_assert(LNW > 0 && (1 << LNW) == NWX, "window widths 8 ... 128");
    constexpr int NP = NWX * NWY;
    if (a.cbed) {
        const float fnorm = (float)a.inv_norm;
        for (int i = tid; i < nwin * NP; i += BLOCK) {
            const int p = i / NP, u = i - p * NP;
            const float2 z = win[(p * NWY + (u >> LNW)) * PW + (u & (NWX - 1))];
            a.cbed[(size_t)oidx[p] * NP + u] = (z.x * z.x + z.y * z.y) * fnorm;
        }
    }
    // annular bins: one thread per (window, bin) walks the bin's pixel list with four interleaved
    // FP32 partial sums of the FP32 intensities (fixed order; each partial carries a relative error
    // <= (n/4) 2^-24 for n pixels), then adds the four partials and applies the normalisation in
    // FP64 (the final accumulation of the bin), rounding once to FP32.
    // The lists come from shared memory where the caller staged them (sidx, bin_idx as 16-bit
    // entries), else from global memory by rank (entry i of bin k at bin_idx_t[i * nbins + k], so
    // that the threads of consecutive bins read consecutive words); the same entries either way.
    if (a.out) {
        const int nb = a.nbins;
        for (int j = tid; j < nwin * nb; j += BLOCK) {
            const int p = j / nb, k = j - p * nb;
            const float2 *w = win + p * NWY * PW;
            const int o0 = __ldg(a.bin_off + k), e = __ldg(a.bin_off + k + 1) - o0;
            const int *ix = a.bin_idx_t + k;
            const uint16_t *sx = sidx ? sidx + o0 : nullptr;
            auto entry = [&](int i) { return sx ? (int)sx[i] : __ldg(ix + i * nb); };
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int i = 0;
            for (; i + 4 <= e; i += 4) {
                const int u0 = entry(i), u1 = entry(i + 1);
                const int u2 = entry(i + 2), u3 = entry(i + 3);
                const float2 z0 = w[(u0 >> LNW) * PW + (u0 & (NWX - 1))], z1 = w[(u1 >> LNW) * PW + (u1 & (NWX - 1))];
                const float2 z2 = w[(u2 >> LNW) * PW + (u2 & (NWX - 1))], z3 = w[(u3 >> LNW) * PW + (u3 & (NWX - 1))];
                s0 = fmaf(z0.x, z0.x, fmaf(z0.y, z0.y, s0));
                s1 = fmaf(z1.x, z1.x, fmaf(z1.y, z1.y, s1));
                s2 = fmaf(z2.x, z2.x, fmaf(z2.y, z2.y, s2));
                s3 = fmaf(z3.x, z3.x, fmaf(z3.y, z3.y, s3));
            }
            for (; i < e; ++i) {
                const int u = entry(i);
                const float2 z = w[(u >> LNW) * PW + (u & (NWX - 1))];
                s0 = fmaf(z.x, z.x, fmaf(z.y, z.y, s0));
            }
            const float val = (float)((((double)s0 + (double)s1) + ((double)s2 + (double)s3)) * a.inv_norm);
            float *o = a.out + (size_t)oidx[p] * a.nbins + k;
            *o = a.accumulate ? *o + a.acc_w * val : val;
        }
    }
}

}  // namespace prism
