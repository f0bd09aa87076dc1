// kernels_scan.cu -- the FP32 PRISM probe scan for sm_103a (PRISM Algorithm section, Fig. 1d-f).
//
// Every kernel takes, per probe position r0:
//   1. coefficients alpha_b(r0) = A(q_b) e^{-i chi(q_b)} e^{-2 pi i q_b.r0}; the phase q_b.r0 is
//      formed in FP64 and reduced to [-1/2, 1/2) cycles before the FP32 sincos;
//   2. window origin s = floor(r0 / px' + 1/2) - Nw/2 (mod N') on the stored grid (Eq. RegionBounds);
//   3. beam sum psi(u) = sum_b alpha_b S_b(s + u) over the window, wrapped (Eq. PRISMfinal);
//   4. 2-D FFT of the window in shared memory (row then column two-level FFTs);
//   5. |Psi|^2 and the annular bins, fixed summation order, FP64 scale.
// Three kernels: k_scan_gemm (4 x 8 raster blocks, the beam sum as a register-tiled complex GEMM on
// the union tile of their windows; the default for windows of 16 to 128 pixels), k_scan_grouped (4
// consecutive probes, used when the GEMM's coefficient block does not fit shared memory or for
// 8-pixel windows) and k_scan (one probe per CTA, for very large beam sets).
#include <cuda_runtime.h>

#include <algorithm>

#include "fft.cuh"
#include "params.h"
#include "scan_common.cuh"
#include "scan_gemm.cuh"  // k_scan_gemm: the default contraction shape is instantiated here for every window

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
    static constexpr int EXC = FS::N1 * (FS::N2 + 1) * CW;
    static constexpr int EX = EXR > EXC ? EXR : EXC;
    static_assert(2 * EX >= NW * NW, "exchange region doubles as the intensity buffer");
    static constexpr size_t SMEM_FIXED = (size_t)(NW * NW + EX + NW) * sizeof(float2);
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
    float2 *twf = ex + C::EX;           // window FFT stage twiddles [NW]
    float2 *alpha = twf + NW;           // [n_beams]
    const int tid = threadIdx.x;
    const int p = a.probe0 + blockIdx.x;
    if (p >= a.n_probes) return;
    for (int i = tid; i < NW; i += BLOCK) twf[i] = a.tw_fwd[i];
    const double x0 = a.x0[p], y0 = a.y0[p];

    // 1. coefficients (a tilted probe uses r0 - h tan(theta))
    for (int b = tid; b < a.n_beams; b += BLOCK) {
        double c = a.qx[b] * (x0 - a.shift_x) + a.qy[b] * (y0 - a.shift_y);
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
            Fwd::run(v, t, twf, a.tw, exr);
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
            Fwd::run(v, t, twf, a.tw, exc);
            __syncthreads();  // all reads of win for this pass done before any write
            if (col < NW) {
#pragma unroll
                for (int r = 0; r < E; ++r) win[Fwd::out_elem(r, t) * NW + cc] = v[r];
            }
        }
    }
    __syncthreads();

    // 5. |Psi|^2 (full pattern if requested) and annular bins
    float *inten = reinterpret_cast<float *>(ex);
    const float fnorm = (float)a.inv_norm;
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const float2 z = win[tid + k * BLOCK];
        const float i2 = z.x * z.x + z.y * z.y;
        inten[tid + k * BLOCK] = i2;
        if (a.cbed) a.cbed[(size_t)p * NW * NW + tid + k * BLOCK] = i2 * fnorm;
    }
    __syncthreads();
    if (!a.out) return;
    const int warp = tid >> 5, lane = tid & 31;
    for (int k = warp; k < a.nbins; k += BLOCK / 32) {
        float s = 0.f;
        const int e = __ldg(a.bin_off + k + 1);
        for (int i = __ldg(a.bin_off + k) + lane; i < e; i += 32) s += inten[__ldg(a.bin_idx + i)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const float val = (float)((double)s * a.inv_norm);
            float *o = a.out + (size_t)p * a.nbins + k;
            *o = a.accumulate ? *o + a.acc_w * val : val;
        }
    }
}

template <int NW>
static cudaError_t scan_dispatch(const ScanArgs &a, cudaStream_t s) {
    using C = ScanCfg<NW>;
    const int n = a.n_probes - a.probe0;
    if (n <= 0) return cudaSuccess;
    const size_t smem = C::SMEM_FIXED + (size_t)a.n_beams * sizeof(float2);
    cudaError_t e = allow_max_dynamic_smem(k_scan<NW>);
    if (e != cudaSuccess) return e;
    k_scan<NW><<<n, C::BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}


// ------------------------------------------------------------------ grouped scan
// G consecutive probes share one CTA.  Adjacent probes of a raster are a few stored pixels apart,
// so their windows overlap: per beam, the union tile of the group's windows is staged once in
// shared memory (a STAGES-deep cp.async pipeline of 16-byte pixel pairs keeps the next beams in
// flight while one is summed) and every thread owns tile pixels, so one shared-memory load feeds
// the complex MACs of all G probes.  A group whose windows do not fit the tile is processed one
// probe at a time.
template <int NWX, int NWY>
struct GroupCfg {
    static constexpr int NWM = NWX > NWY ? NWX : NWY;
    static constexpr int G = 4;
    static constexpr int D = 16;                              // tile may exceed a window by D pixels
    static constexpr int BLOCK = NWM >= 64 ? 512 : NWM >= 16 ? 256 : 64;
    static constexpr int MAXTILE = (NWX + D) * NWY;           // tile pixels
    static constexpr int PIX = (MAXTILE + BLOCK - 1) / BLOCK; // tile pixels per thread
    static constexpr int PAIRS = (MAXTILE / 2 + BLOCK - 1) / BLOCK;  // 16-byte copies per thread
    static constexpr int PW = NWX + 4;                        // window row pitch (bank spread)
    static constexpr int EX = ExSize<NWX, NWY, BLOCK>::value;
    static constexpr int STAGES = 4;                          // cp.async pipeline depth (beams in flight)
    static constexpr int BIG = (STAGES * MAXTILE > G * NWY * PW) ? STAGES * MAXTILE : G * NWY * PW;
    static constexpr size_t SMEM_FIXED = (size_t)(BIG + EX + NWX + NWY) * sizeof(float2) + 64 * sizeof(int);
};

template <int NWX, int NWY>
__global__ void __launch_bounds__(GroupCfg<NWX, NWY>::BLOCK) k_scan_grouped(const __grid_constant__ ScanArgs a) {
    using C = GroupCfg<NWX, NWY>;
    constexpr int BLOCK = C::BLOCK, PIX = C::PIX, G = C::G, PW = C::PW;
    extern __shared__ float2 smem[];
    float2 *big = smem;                    // staging tiles [STAGES][MAXTILE], later windows [G][NWY][PW]
    float2 *ex = big + C::BIG;             // FFT exchange
    float2 *twx = ex + C::EX;              // window FFT stage twiddles, rows [NWX] and columns [NWY]
    float2 *twy = twx + NWX;
    int *meta = reinterpret_cast<int *>(twy + NWY);  // group geometry
    float2 *alpha = reinterpret_cast<float2 *>(meta + 64);  // [G][n_beams]
    const int tid = threadIdx.x;
    const int p0 = a.probe0 + blockIdx.x * G;
    if (p0 >= a.n_probes) return;
    const int gn = min(G, a.n_probes - p0);
    for (int i = tid; i < NWX; i += BLOCK) twx[i] = a.tw_fwd[i];
    for (int i = tid; i < NWY; i += BLOCK) twy[i] = a.tw_fwd_y[i];
    group_coefficients<G>(a, p0, gn, alpha, tid, BLOCK);
    if (tid == 0) group_geometry<NWX, NWY, G, C::D, C::MAXTILE>(a, p0, gn, meta);
    __syncthreads();
    const int nsub = meta[0];
    const size_t bstride = (size_t)a.ny_s * a.nx_s;

    for (int sg = 0; sg < nsub; ++sg) {
        // geometry of this sub-group: all gn probes (tile = union), or probe sg alone (its window,
        // widened by one column on the left if it starts on an odd column)
        const bool all = nsub == 1;
        int tw, th, tx0, ty0, ox1 = 0;
        if (all) {
            tw = meta[1];
            th = meta[2];
            tx0 = meta[3];
            ty0 = meta[4];
        } else {
            ox1 = meta[8 + sg] & 1;
            tw = NWX + 2 * ox1;
            th = NWY;
            tx0 = meta[8 + sg] - ox1;
            ty0 = meta[16 + sg];
        }
        const int npx = tw * th;
        const int hw = tw >> 1;  // pixel pairs per tile row
        // global offsets of this thread's pixel pairs (fixed for all beams)
        int off[C::PAIRS];
#pragma unroll
        for (int k = 0; k < C::PAIRS; ++k) {
            const int q = tid + k * BLOCK;
            const int ty = q / hw, tp = q - ty * hw;
            off[k] = q < (npx >> 1) ? ((ty0 + ty) & (a.ny_s - 1)) * a.nx_s + ((tx0 + 2 * tp) & (a.nx_s - 1)) : -1;
        }
        const float2 *al = alpha + (all ? 0 : sg * a.n_beams);
        float2 acc[PIX][G];
#pragma unroll
        for (int k = 0; k < PIX; ++k)
#pragma unroll
            for (int p = 0; p < G; ++p) acc[k][p] = make_float2(0.f, 0.f);

        // beam loop: STAGES-1 beam tiles in flight while one is summed; one barrier per beam
        // (after it every thread is done with the previous tile, whose buffer is then refilled)
        constexpr int S = C::STAGES;
        auto stage = [&](int b) {
            if (b < a.n_beams) {
                const float2 *Sb = a.S + (size_t)b * bstride;
                float2 *buf = big + (b % S) * C::MAXTILE;
#pragma unroll
                for (int k = 0; k < C::PAIRS; ++k)
                    if (off[k] >= 0) cp_async16(buf + 2 * (tid + k * BLOCK), Sb + off[k]);
            }
            cp_async_commit();
        };
#pragma unroll
        for (int b = 0; b < S - 1; ++b) stage(b);
        for (int b = 0; b < a.n_beams; ++b) {
            cp_async_wait<S - 2>();
            __syncthreads();
            stage(b + S - 1);
            const float2 *cur = big + (b % S) * C::MAXTILE;
            float2 av[G];
#pragma unroll
            for (int p = 0; p < G; ++p) av[p] = al[(all ? p : 0) * a.n_beams + b];
            float2 sv[PIX];
#pragma unroll
            for (int k = 0; k < PIX; ++k) sv[k] = cur[tid + k * BLOCK];
#pragma unroll
            for (int k = 0; k < PIX; ++k)
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    acc[k][p].x = fmaf(av[p].x, sv[k].x, fmaf(-av[p].y, sv[k].y, acc[k][p].x));
                    acc[k][p].y = fmaf(av[p].x, sv[k].y, fmaf(av[p].y, sv[k].x, acc[k][p].y));
                }
        }
        cp_async_wait<0>();
        __syncthreads();
        // scatter the accumulators into the windows: tile pixel (ty, tx) is pixel
        // (ty - oy_p, tx - ox_p) of probe p's window
        float2 *win = big;
#pragma unroll
        for (int k = 0; k < PIX; ++k) {
            const int i = tid + k * BLOCK;
            const int ty = i / tw, tx = i - ty * tw;
#pragma unroll
            for (int p = 0; p < G; ++p) {
                const bool act = all ? p < gn : p == 0;
                const int wy = ty - (all ? meta[32 + p] : 0), wx = tx - (all ? meta[24 + p] : ox1);
                if (act && i < npx && wy >= 0 && wy < NWY && wx >= 0 && wx < NWX) win[(p * NWY + wy) * PW + wx] = acc[k][p];
            }
        }
        __syncthreads();
        window_epilogue<NWX, NWY, BLOCK, G, PW>(a, win, ex, twx, twy, all ? gn : 1, meta + 40 + (all ? 0 : sg), tid);
        __syncthreads();  // windows and staging buffers are reused by the next sub-group
    }
}

template <int NWX, int NWY>
static cudaError_t scan_grouped_dispatch(const ScanArgs &a, cudaStream_t s) {
    using C = GroupCfg<NWX, NWY>;
    const int n = a.n_probes - a.probe0;
    if (n <= 0) return cudaSuccess;
    const size_t smem = C::SMEM_FIXED + (size_t)C::G * a.n_beams * sizeof(float2);
    cudaError_t e = allow_max_dynamic_smem(k_scan_grouped<NWX, NWY>);
    if (e != cudaSuccess) return e;
    k_scan_grouped<NWX, NWY><<<(n + C::G - 1) / C::G, C::BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NWX, int NWY>
static bool grouped_fits(int n_beams) {
    return GroupCfg<NWX, NWY>::SMEM_FIXED + (size_t)GroupCfg<NWX, NWY>::G * n_beams * sizeof(float2) <= 227 * 1024;
}

// (128-pixel windows: one CTA per SM, the coefficients of up to about 630 beams in shared memory;
// larger beam sets go to k_scan)
#define PRISM_GEMM_SIDES(X)                                                                                                  \
    X(16, 16) X(16, 32) X(16, 64) X(32, 16) X(32, 32) X(32, 64) X(64, 16) X(64, 32) X(64, 64) X(128, 128)

// shape 0 here; the others (square windows) in kernels_tune_scan.cu
int scan_gemm_grid(int nwx, int nwy, int shape, int n_beams, int scan_px, int scan_py) {
    if (shape != 0) return scan_gemm_grid_tuned(nwx, nwy, shape, n_beams, scan_px, scan_py);
#define PRISM_GEMM_GRID(x, y) \
    if (nwx == x && nwy == y) return gemm_grid<x, y>(n_beams, scan_px, scan_py);
    PRISM_GEMM_SIDES(PRISM_GEMM_GRID)
#undef PRISM_GEMM_GRID
    return 0;
}

cudaError_t launch_scan_gemm(int nwx, int nwy, int shape, int grid, const ScanArgs &a, cudaStream_t s) {
    if (grid <= 0 || !a.win || !a.win_cnt || a.scan_px <= 0 || a.scan_py <= 0) return cudaErrorInvalidValue;
    if (shape != 0) return launch_scan_gemm_tuned(nwx, nwy, shape, grid, a, s);
#define PRISM_GEMM_LAUNCH(x, y) \
    if (nwx == x && nwy == y) return gemm_launch<x, y>(grid, a, s);
    PRISM_GEMM_SIDES(PRISM_GEMM_LAUNCH)
#undef PRISM_GEMM_LAUNCH
    return cudaErrorInvalidValue;
}

size_t scan_gemm_win_bytes(int nwx, int nwy, int shape, int grid, int scan_px, int scan_py) {
    return gemm_win_bytes(shape, nwx, nwy, grid, scan_px, scan_py);
}

int scan_gemm_shapes() { return N_GEMM_SHAPES; }

// the split blocks' completion counters (one per CTA at most), the next work unit, the CTAs done
size_t scan_gemm_cnt_bytes(int grid) { return (size_t)((grid > 0 ? grid : 1) + 2) * sizeof(int); }

// rectangular windows (separate interpolation factors f_x != f_y): grouped kernel only
template <int NWX>
static cudaError_t scan_rect_y(int nwy, const ScanArgs &a, cudaStream_t s) {
    switch (nwy) {
        case 16: return NWX != 16 && grouped_fits<NWX, 16>(a.n_beams) ? scan_grouped_dispatch<NWX, 16>(a, s) : cudaErrorInvalidValue;
        case 32: return NWX != 32 && grouped_fits<NWX, 32>(a.n_beams) ? scan_grouped_dispatch<NWX, 32>(a, s) : cudaErrorInvalidValue;
        case 64: return NWX != 64 && grouped_fits<NWX, 64>(a.n_beams) ? scan_grouped_dispatch<NWX, 64>(a, s) : cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_scan_rect(int nwx, int nwy, const ScanArgs &a, cudaStream_t s) {
    if (nwx == nwy) return launch_scan(nwx, a, s);
    switch (nwx) {
        case 16: return scan_rect_y<16>(nwy, a, s);
        case 32: return scan_rect_y<32>(nwy, a, s);
        case 64: return scan_rect_y<64>(nwy, a, s);
    }
    return cudaErrorInvalidValue;
}

bool scan_rect_supported(int nwx, int nwy, int n_beams) {
    if (nwx == nwy) return scan_supported(nwx);
    auto in = [](int n) { return n == 16 || n == 32 || n == 64; };
    if (!in(nwx) || !in(nwy)) return false;
    const size_t fixed = (nwx == 16 ? (nwy == 32 ? GroupCfg<16, 32>::SMEM_FIXED : GroupCfg<16, 64>::SMEM_FIXED)
                          : nwx == 32 ? (nwy == 16 ? GroupCfg<32, 16>::SMEM_FIXED : GroupCfg<32, 64>::SMEM_FIXED)
                                      : (nwy == 16 ? GroupCfg<64, 16>::SMEM_FIXED : GroupCfg<64, 32>::SMEM_FIXED));
    return fixed + (size_t)4 * n_beams * sizeof(float2) <= 227 * 1024;
}

cudaError_t launch_scan(int nw, const ScanArgs &a, cudaStream_t s) {
    switch (nw) {
        case 8: return grouped_fits<8, 8>(a.n_beams) ? scan_grouped_dispatch<8, 8>(a, s) : scan_dispatch<8>(a, s);
        case 16: return grouped_fits<16, 16>(a.n_beams) ? scan_grouped_dispatch<16, 16>(a, s) : scan_dispatch<16>(a, s);
        case 32: return grouped_fits<32, 32>(a.n_beams) ? scan_grouped_dispatch<32, 32>(a, s) : scan_dispatch<32>(a, s);
        case 64: return grouped_fits<64, 64>(a.n_beams) ? scan_grouped_dispatch<64, 64>(a, s) : scan_dispatch<64>(a, s);
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
