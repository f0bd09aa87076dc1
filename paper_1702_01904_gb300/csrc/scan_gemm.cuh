// scan_gemm.cuh -- the FP32 beam sum of the PRISM scan as a register-tiled complex GEMM
// (k_scan_gemm), templated on the window sides and on the contraction tile shape.  kernels_scan.cu
// instantiates the default shape for every window; kernels_tune_scan.cu the other shapes, which the
// autotuner times, for square windows.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "fft.cuh"
#include "params.h"
#include "scan_common.cuh"

namespace prism {

// ------------------------------------------------------------------ FP32 GEMM scan
// The beam sum of Eq. PRISMfinal for a 4 x 8 block of the probe raster as a complex GEMM on the
// union tile of their windows, on the CUDA cores in FP32: psi_p(r) = sum_b S_b(r) alpha_bp for the
// tile pixels r (M) and the block's 32 probes (N), K = the beams.  The tile is streamed in M tiles
// of 128 pixels; per M tile the beams pass through a 2-stage cp.async ring (KB beams x 128 pixels
// per stage, one 16-byte copy per pixel pair and beam: the union tile starts on an even column and
// has an even width, so a pair never straddles a row or the cell's edge and is 16-byte aligned in
// the S-matrix); thread (lane, warp) accumulates pixels lane +
// 32 i (i < 4) for probes 4 warp + j (j < 4) -- raster row `warp` of the block -- in registers, so
// one 8-byte shared-memory load feeds four complex MACs.  A warp skips the M tiles that lie wholly
// above or below its row's windows (the union tile is NWY + 7 probe steps high, a row's windows
// NWY).  Finished M tiles are scattered to the per-CTA window scratch; the window FFT
// and bins are the shared epilogue.  A block whose union tile is larger than its windows together
// runs probe by probe (only the warp holding that probe computes).
// Work units: the blocks of all full rounds of the persistent grid run whole; the blocks of the
// last, partial round (fewer than the CTAs; all blocks of a scan smaller than the grid) are split
// into up to MAXP parts of their M tiles (or of their probes, when they run probe by probe) so that
// that round keeps every CTA busy.  A split block's windows go to a scratch slot of its own; each
// part counts itself done on an atomic counter, and the part that completes the block runs its
// epilogue.  Every window pixel is still one accumulation in the same beam order, so the split
// changes no result.  Scratch slots: [0, tail) the split blocks, then one per CTA when some block
// runs whole.
// Contraction tile shapes: raster block GX x GY (32 probes, four per warp), beams per ring stage
// and ring depth.  Shape 0 is the default; the autotuner times the others (kernels_tune_scan.cu).
// Every shape accumulates each window pixel over the beams in the same order, so all give bitwise
// the same windows.
struct GemmShape {
    int gx, gy, kb, stages;
};
// The default ring stage holds 33 beams: the 129 beams of a 20 mrad aperture at f = 8 go in 4
// chunks (one block barrier each per M tile) instead of 5 with 32, and two CTAs still share an SM
// (5.47 -> 5.38 ms on the 40 000-probe carbon scan).
constexpr GemmShape GEMM_SHAPES[] = {{4, 8, 33, 2}, {8, 4, 32, 2}, {2, 16, 32, 2}, {4, 8, 16, 3}, {8, 4, 16, 3}, {4, 8, 32, 2}};
constexpr int N_GEMM_SHAPES = sizeof(GEMM_SHAPES) / sizeof(GemmShape);

template <int NWX, int NWY, int SH = 0>
struct GemmCfg {
    static constexpr int GX = GEMM_SHAPES[SH].gx, GY = GEMM_SHAPES[SH].gy, G = GX * GY;  // four probes per warp
    static_assert(G == 32, "a block holds 32 probes");
    static constexpr int BLOCK = 256;
    static constexpr int KB = GEMM_SHAPES[SH].kb;      // beams per ring stage
    static constexpr int STAGES = GEMM_SHAPES[SH].stages;
    static constexpr int MT = 128;                   // tile pixels per M tile
    static constexpr int RING = STAGES * KB * MT;    // float2
    static constexpr int PW = NWX + 4;                        // window row pitch (bank spread)
    static constexpr int NWM = NWX > NWY ? NWX : NWY;
    static constexpr int EW = NWM >= 128 ? 1 : NWM >= 64 ? 2 : NWM == 32 ? 8 : 16;  // windows per epilogue pass
    static constexpr int EX = ExSize<NWX, NWY, BLOCK>::value;
    static constexpr size_t EPI = (size_t)(EW * NWY * PW + EX) * sizeof(float2);
    static constexpr int META = 256;
    static constexpr int META_LAST = META - 1;       // flag: this CTA completed a split block
    static constexpr int META_UNIT = META - 2;       // the work unit this CTA took
    static constexpr int MAXP = 16;                  // parts per split block at most
    __host__ __device__ static constexpr size_t region0(int n_beams) {
        const size_t r = ((size_t)RING + (size_t)n_beams * G) * sizeof(float2);
        return ((r > EPI ? r : EPI) + 127) & ~(size_t)127;
    }
    // region0, the window twiddles, meta, the probes' packed window origins
    __host__ __device__ static constexpr size_t smem(int n_beams) {
        return region0(n_beams) + (size_t)(NWX + NWY) * sizeof(float2) + META * sizeof(int) + G * sizeof(int);
    }
};

template <int NWX, int NWY, int SH = 0>
__global__ void __launch_bounds__(256, 2) k_scan_gemm(const __grid_constant__ ScanArgs a) {
    using C = GemmCfg<NWX, NWY, SH>;
    constexpr int G = C::G, GX = C::GX, GY = C::GY, BLOCK = C::BLOCK, KB = C::KB, MT = C::MT, S = C::STAGES, PW = C::PW;
    extern __shared__ __align__(16) float2 smf[];
    const int nb = a.n_beams;
    float2 *ring = smf;                               // [STAGES][KB][MT]
    float2 *alpha = smf + C::RING;                    // [nb][G]
    float2 *win = smf;                                // epilogue: windows, then exchange
    float2 *ex = win + C::EW * NWY * PW;
    float2 *twx = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(smf) + C::region0(nb));
    float2 *twy = twx + NWX;
    int *meta = reinterpret_cast<int *>(twy + NWY);
    int *wofs = meta + C::META;  // [G], 16-byte aligned
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < NWX; i += BLOCK) twx[i] = a.tw_fwd[i];
    for (int i = tid; i < NWY; i += BLOCK) twy[i] = a.tw_fwd_y[i];
    const int ngx = (a.scan_px + GX - 1) / GX, ngy = (a.scan_py + GY - 1) / GY;
    const size_t npix_s = (size_t)a.ny_s * a.nx_s;
    const int nkc = (nb + KB - 1) / KB, kcs = (nb + nkc - 1) / nkc;  // balanced beam chunks

    const int n_groups = ngx * ngy;
    const int tail = n_groups % gridDim.x, full = n_groups - tail;
    const int parts = tail ? min(C::MAXP, (int)gridDim.x / tail) : 1;

    // Work units come from a counter (after the split counters: the next unit, then the CTAs done),
    // not by a fixed stride: the two CTAs that share an SM are not issued equally, and with fixed
    // shares the favoured one finished its blocks early and left the other to finish alone.  Which
    // CTA computes a unit changes no result.
    int *next_unit = a.win_cnt + gridDim.x, *ctas_done = next_unit + 1;
    const int n_units = full + tail * parts;
    for (;;) {
        if (tid == 0) meta[C::META_UNIT] = atomicAdd(next_unit, 1);
        __syncthreads();  // every thread read the previous unit before the barriers of its body
        const int u = meta[C::META_UNIT];
        if (u >= n_units) break;
        // unit u: block u whole (scratch slot = this CTA), or part `part` of split block full + tg
        int grp = u, part = 0, np = 1, slot = tail + blockIdx.x;
        if (u >= full) {
            const int tg = (u - full) / parts;
            grp = full + tg;
            part = u - full - tg * parts;
            np = parts;
            slot = tg;
        }
        const int gy = grp / ngx, gx = grp - gy * ngx;
        // coefficients alpha[b][p] (zero for slots past the raster)
        for (int i = tid; i < nb * G; i += BLOCK) {
            const int b = i / G, p = i - b * G;
            const int row = gy * GY + p / GX, col = gx * GX + p % GX;
            float2 v = make_float2(0.f, 0.f);
            if (row < a.scan_py && col < a.scan_px) {
                const int pr = row * a.scan_px + col;
                double c = a.qx[b] * (a.x0[pr] - a.shift_x) + a.qy[b] * (a.y0[pr] - a.shift_y);
                c -= rint(c);
                float sn, cs;
                sincospif(-2.0f * (float)c, &sn, &cs);
                v = cmul(__ldg(a.base + b), make_float2(cs, sn));
            }
            alpha[i] = v;
        }
        if (warp == 0) raster_group_geometry<NWX, NWY, GX, GY>(a, gx, gy, meta, lane);
        __syncthreads();
        const bool uni = meta[0] != 0;
        for (int sg = 0; sg < (uni ? 1 : G); ++sg) {
            if (!uni && (meta[136 + sg] < 0 || sg % np != part)) continue;
            // probe by probe: the window widened to start on an even column (ox = its odd start)
            const int ox = uni ? 0 : meta[8 + sg] & 1;
            const int tw = uni ? meta[1] : NWX + 2 * ox, th = uni ? meta[2] : NWY;
            const int tx0 = uni ? meta[3] : meta[8 + sg] - ox, ty0 = uni ? meta[4] : meta[40 + sg];
            const int npx = tw * th, nmt = (npx + MT - 1) / MT;
            // each probe's window origin in the tile, packed (oy << 16 | ox; both >= 0 and small), or
            // one that no tile pixel reaches for the probes not computed here; read by the scatters
            // after a step's barrier (the previous sub-group's ended at a barrier)
            if (tid < G) {
                const bool act = uni ? meta[136 + tid] >= 0 : tid == sg;
                wofs[tid] = !act ? 0x7fff7fff : uni ? (meta[104 + tid] << 16) | meta[72 + tid] : ox;
            }
            // ring steps (M tile, beam chunk) of this unit: all, or a split block's share of M tiles
            const int ls0 = uni ? part * nmt / np * nkc : 0, ls1 = uni ? (part + 1) * nmt / np * nkc : nmt * nkc;
            const bool busy = uni || (sg >> 2) == warp;  // warps whose probes are computed
            // union-tile rows the windows of this warp's probes cover (a warp's four probes share a
            // raster row): M tiles wholly outside them hold none of its window pixels, so the warp
            // skips their products
            int wy0 = 0, wy1 = th - 1;
            if (uni) {
                wy0 = th;
                wy1 = -1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int p = 4 * warp + j;
                    if (meta[136 + p] >= 0) {
                        wy0 = min(wy0, meta[104 + p]);
                        wy1 = max(wy1, meta[104 + p] + NWY - 1);
                    }
                }
            }
            // loader: thread -> tile pixel pair m = 2 (tid % (MT/2)), beams kk = tid / (MT/2), + 4, ...
            // (tw, tx0 and the M tile bounds even: the pair lies in one row, on an even column)
            // (the loader takes the steps in order: it counts its M tile and beam chunk, and finds its
            // pixel pair in the S-matrix only when the tile changes)
            constexpr int PAIRS = MT / 2, KSTEP = BLOCK / PAIRS;
            const int lm = 2 * (tid & (PAIRS - 1)), lk = tid / PAIRS;
            const int mt0 = uni ? part * nmt / np : 0;  // ls0 = mt0 nkc
            int l_step = ls0, l_mt = mt0, l_c = 0, l_tile = -1;
            const float2 *l_pix = nullptr;  // the pair's pixel in beam lk (nullptr: past the union tile)
            auto load = [&]() {
                if (l_step < ls1) {
                    if (l_mt != l_tile) {
                        l_tile = l_mt;
                        const int idx = l_mt * MT + lm;
                        l_pix = nullptr;
                        if (idx < npx) {
                            const int ty = idx / tw, tx = idx - ty * tw;
                            const size_t gp = (size_t)((ty0 + ty) & (a.ny_s - 1)) * a.nx_s + ((tx0 + tx) & (a.nx_s - 1));
                            l_pix = a.S + (size_t)lk * npix_s + gp;
                        }
                    }
                    if (l_pix) {
                        const int b0 = l_c * kcs, bn = min(kcs, nb - b0);
                        float2 *dst = ring + (l_step % S) * (KB * MT) + lm;
                        const float2 *src = l_pix + (size_t)b0 * npix_s;
                        for (int kk = lk; kk < bn; kk += KSTEP, src += (size_t)KSTEP * npix_s) cp_async16(dst + kk * MT, src);
                    }
                    if (++l_c == nkc) {
                        l_c = 0;
                        ++l_mt;
                    }
                }
                ++l_step;
                cp_async_commit();
            };
#pragma unroll
            for (int l = 0; l < S - 1; ++l) load();
            // psi = sum_b S_b Re(alpha_b) + i sum_b S_b Im(alpha_b): two complex accumulators per
            // (pixel, probe), each advanced by one packed FP32x2 FMA of the S value with a real
            // coefficient (accr += S Re a, acci += S Im a), combined when the M tile is done
            float2 accr[4][4], acci[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = make_float2(0.f, 0.f);
            int mt = mt0, c = 0;  // the M tile and beam chunk of step ls
            bool need = false;    // this warp computes M tile mt
            for (int ls = ls0; ls < ls1; ++ls) {
                cp_async_wait<S - 2>();
                __syncthreads();
                load();  // step ls + S - 1: its slot was last read in step ls - 1, which every thread has left
                if (c == 0) need = busy && (mt * MT + MT - 1) / tw >= wy0 && (mt * MT) / tw <= wy1;
                if (need) {
                    const float2 *cur = ring + (ls % S) * (KB * MT);
                    const int b0 = c * kcs, bn = min(kcs, nb - b0);
                    const float4 *al = reinterpret_cast<const float4 *>(alpha + (size_t)b0 * G + 4 * warp);
#pragma unroll 4
                    for (int kk = 0; kk < bn; ++kk) {
                        const float4 a01 = al[(size_t)kk * (G / 2)], a23 = al[(size_t)kk * (G / 2) + 1];
                        const float2 ar[4] = {make_float2(a01.x, a01.x), make_float2(a01.z, a01.z),
                                              make_float2(a23.x, a23.x), make_float2(a23.z, a23.z)};
                        const float2 ai[4] = {make_float2(a01.y, a01.y), make_float2(a01.w, a01.w),
                                              make_float2(a23.y, a23.y), make_float2(a23.w, a23.w)};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float2 sv = cur[kk * MT + lane + 32 * i];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                accr[i][j] = __ffma2_rn(sv, ar[j], accr[i][j]);
                                acci[i][j] = __ffma2_rn(sv, ai[j], acci[i][j]);
                            }
                        }
                    }
                }
                if (c == nkc - 1) {
                    // M tile done: scatter tile pixel (ty, tx) to pixel (ty - oy_p, tx - ox_p) of probe p
                    if (need) {
                        const int4 o4 = *reinterpret_cast<const int4 *>(wofs + 4 * warp);  // this warp's probes
                        const int oo[4] = {o4.x, o4.y, o4.z, o4.w};
                        float2 *wp = a.win + ((size_t)slot * G + 4 * warp) * (NWX * NWY);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int idx = mt * MT + lane + 32 * i;
                            const int ty = idx / tw, tx = idx - ty * tw;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int wy = ty - (oo[j] >> 16), wx = tx - (oo[j] & 0xffff);
                                // psi = accr + i acci
                                const float2 v = make_float2(accr[i][j].x - acci[i][j].y, accr[i][j].y + acci[i][j].x);
                                if (idx < npx && (unsigned)wy < (unsigned)NWY && (unsigned)wx < (unsigned)NWX)
                                    __stcs(wp + j * (NWX * NWY) + wy * NWX + wx, v);
                                accr[i][j] = acci[i][j] = make_float2(0.f, 0.f);
                            }
                        }
                    }
                }
                if (++c == nkc) {
                    c = 0;
                    ++mt;
                }
            }
            cp_async_wait<0>();
            __syncthreads();  // ring reads done before the next sub-group or the epilogue reuses it
        }
        if (np > 1) {
            // split block: count this part done; the part that completes the block goes on to its
            // epilogue (release: every thread's scratch stores before the count; acquire: the count
            // before the scratch loads, which read L2)
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
        // epilogue: EW windows at a time through shared memory (the window scratch written above is
        // visible to the whole CTA after the barrier).  The bins read their pixel lists from global
        // memory: staging them in shared memory (as the tensor-core scan does) cost this kernel, at
        // its register limit, more than it saved (5.09 against 5.03 ms on the carbon scan).
        const int nvalid = meta[5];
        for (int e0 = 0; e0 < nvalid; e0 += C::EW) {
            const int ne = min(C::EW, nvalid - e0);
            // the windows in 16-byte pieces (two pixels of a row), every piece in flight at once
            for (int i = tid; i < ne * (NWX * NWY / 2); i += BLOCK) {
                const int e = i / (NWX * NWY / 2), u = 2 * (i - e * (NWX * NWY / 2));
                cp_async16(win + (e * NWY + u / NWX) * PW + (u % NWX), a.win + ((size_t)slot * G + meta[168 + e0 + e]) * (NWX * NWY) + u);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            window_epilogue<NWX, NWY, BLOCK, C::EW, PW>(a, win, ex, twx, twy, ne, meta + 200 + e0, tid);
            __syncthreads();
        }
    }
    // the last CTA to finish has seen every unit taken: it zeroes both counters for the next launch
    if (tid == 0 && atomicAdd(ctas_done, 1) == (int)gridDim.x - 1) {
        *next_unit = 0;
        *ctas_done = 0;
    }
}

template <int NWX, int NWY, int SH = 0>
static int gemm_grid(int n_beams, int scan_px, int scan_py) {
    using C = GemmCfg<NWX, NWY, SH>;
    const size_t smem = C::smem(n_beams);
    if (smem > 227 * 1024 || scan_px <= 0 || scan_py <= 0) return 0;
    if (allow_max_dynamic_smem(k_scan_gemm<NWX, NWY, SH>) != cudaSuccess)
        return 0;
    if (cudaFuncSetAttribute(k_scan_gemm<NWX, NWY, SH>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_gemm<NWX, NWY, SH>, C::BLOCK, smem) != cudaSuccess || per_sm < 1)
        return 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const long long groups = (long long)((scan_px + C::GX - 1) / C::GX) * ((scan_py + C::GY - 1) / C::GY);
    return (int)std::max<long long>(1, std::min<long long>(groups * C::MAXP, (long long)per_sm * sms));
}

template <int NWX, int NWY, int SH = 0>
static cudaError_t gemm_launch(int grid, const ScanArgs &a, cudaStream_t s) {
    using C = GemmCfg<NWX, NWY, SH>;
    // the ring's 16-byte copies read pixel pairs of the S-matrix
    if (reinterpret_cast<uintptr_t>(a.S) & 15) return cudaErrorMisalignedAddress;
    const size_t smem = C::smem(a.n_beams);
    cudaError_t e = allow_max_dynamic_smem(k_scan_gemm<NWX, NWY, SH>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_scan_gemm<NWX, NWY, SH>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    k_scan_gemm<NWX, NWY, SH><<<grid, C::BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

// window scratch of a launch of contraction shape `shape`: one slot of 32 windows per block split
// over idle CTAs, one per CTA when some block runs whole (0 for an unknown shape or no work)
static inline size_t gemm_win_bytes(int shape, int nwx, int nwy, int grid, int scan_px, int scan_py) {
    if (shape < 0 || shape >= N_GEMM_SHAPES || grid <= 0 || scan_px <= 0 || scan_py <= 0) return 0;
    const int gx = GEMM_SHAPES[shape].gx, gy = GEMM_SHAPES[shape].gy;
    const long long groups = (long long)((scan_px + gx - 1) / gx) * ((scan_py + gy - 1) / gy);
    const long long tail = groups % grid, slots = tail + (groups > tail ? grid : 0);
    return (size_t)slots * (gx * gy) * nwx * nwy * sizeof(float2);
}

}  // namespace prism
