// scan_tc.cuh -- the tensor-core PRISM scan (k_scan_tc) as a template over its window, the 16-bit
// mode and the ring shape of its A operand; kernels_tc.cu instantiates the default ring shape,
// kernels_tc_tune.cu the others, which the scan autotuner times.
#pragma once
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
// Ring shapes of the A operand: stages x K values per stage.  Shape 0 (3 x 96, each chunk issued two
// steps before its MMAs; 272 = 96 + 96 + 80 for the 129-beam set) is the default; the autotuner
// times the others.  Split mode keeps 2 x 32 in every shape (its two operand parts fill the shared
// memory of two CTAs per SM).  Every shape issues the K = 16 MMAs of a pixel tile in the same order
// into the same accumulator, so all give bitwise the same windows.
struct TcShape {
    int stages, kc;
};
constexpr TcShape TC_SHAPES[] = {{3, 96}, {2, 128}, {4, 64}};
constexpr int N_TC_SHAPES = sizeof(TC_SHAPES) / sizeof(TcShape);

template <int NW, bool SPLIT = false, int SH = 0>
struct TcCfg {
    using FS = FftShape<NW>;
    static constexpr int GX = 8, GY = 4, G = GX * GY, N = 2 * G;
    static constexpr int BLOCK = 256;
    static constexpr int PARTS = SPLIT ? 2 : 1;              // hi (and lo) operand parts
    // ring of K chunks (TC_SHAPES; split mode 2 stages of 32)
    static constexpr int STAGES = SPLIT ? 2 : TC_SHAPES[SH].stages;
    static constexpr int KCMAX = SPLIT ? 32 : TC_SHAPES[SH].kc;  // K (16-bit values) per ring stage
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
    static constexpr int META_UNIT = META - 2;              // the work unit this CTA took
    static constexpr int MAXP = 16;                         // parts per split block at most
    // twiddles, meta, the ring's mbarriers, the TMEM address (16 B), the probes' packed window origins
    static constexpr size_t MISC = (size_t)NW * sizeof(float2) + META * sizeof(int) + STAGES * 8 + 16 + G * sizeof(int);
    static constexpr uint32_t TMEM_COLS = 2 * N;            // two accumulators
    __host__ __device__ static constexpr size_t bmat_bytes(int kp) { return (size_t)PARTS * kp * N * 2; }
    __host__ __device__ static constexpr size_t region0(int kp) {
        const size_t r = (size_t)RING + bmat_bytes(kp);
        return ((r > EPI ? r : EPI) + 127) & ~(size_t)127;
    }
    __host__ __device__ static constexpr size_t smem(int kp) { return region0(kp) + MISC; }
};
// meta: the layout of raster_group_geometry (scan_common.cuh)


template <int NW, int MODE, int SH = 0>
__global__ void __maxnreg__(112) k_scan_tc(const __grid_constant__ ScanArgs a) {
    constexpr bool BF = MODE == TC_BF16, SPLIT = MODE == TC_SPLIT;
    using C = TcCfg<NW, SPLIT, SH>;
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
    int *wofs = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(tmem_base) + 16);  // [G]
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
    // work units from a counter, as in the FP32 GEMM scan (the next unit, then the CTAs done, after
    // the split counters)
    int *next_unit = a.win_cnt + gridDim.x, *ctas_done = next_unit + 1;
    const int n_units = full + tail * parts;
    while (!dead) {
        if (tid == 0) meta[C::META_UNIT] = atomicAdd(next_unit, 1);
        __syncthreads();  // every thread read the previous unit before the barriers of its body
        const int u = meta[C::META_UNIT];
        if (u >= n_units) break;
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
            // each probe's window origin in the tile, packed (oy << 16 | ox; both >= 0 and small), or
            // one that no tile pixel reaches for the probes not computed here; the drains read it after
            // the step loop's first barrier, and the previous sub-group's drains ended at a barrier
            if (tid < G) {
                const bool act = uni ? meta[136 + tid] >= 0 : tid == sg;
                wofs[tid] = !act ? 0x7fff7fff : uni ? (meta[104 + tid] << 16) | meta[72 + tid] : 0;
            }
            const uint32_t st0 = st;
            // A chunk of local step ls: thread -> pixel m = 16 warp + lane/2 of the M tile, K cores
            // kc = lane%2, lane%2 + 2, ...  (a lane pair reads one 32-byte sector of a pixel; a warp
            // writes 2 x 256 contiguous shared-memory bytes)
            // The loader takes the steps in order (step ls: M tile m0 + ls / nkc, K chunk ls % nkc), so
            // it counts its tile and chunk, and finds its pixel's row of S16 only when the tile changes.
            const int lm = warp * 16 + (lane >> 1);
            int l_step = 0, l_mt = m0, l_c = 0, l_tile = -1;
            const uint16_t *l_row = nullptr;  // the pixel's K row (nullptr: past the union tile)
            auto load = [&]() {
                if (l_step < nsteps) {
                    if (l_mt != l_tile) {
                        l_tile = l_mt;
                        const int idx = l_mt * 128 + lm;
                        l_row = nullptr;
                        if (idx < npx) {
                            const int ty = idx / tw, tx = idx - ty * tw;
                            const size_t gp = (size_t)((ty0 + ty) & (a.ny_s - 1)) * a.nx_s + ((tx0 + tx) & (a.nx_s - 1));
                            l_row = S16 + gp * (C::PARTS * kp);
                        }
                    }
                    if (l_row) {
                        const int k0 = l_c * kcs, kn = min(kcs, kp - k0);
                        const uint16_t *src = l_row + k0;
                        unsigned char *dst = ring + ((st0 + l_step) % S) * C::STAGE_BYTES + (lm >> 3) * 128 + (lm & 7) * 16;
                        for (int kc = lane & 1; kc < kn / 8; kc += 2) {
                            cp_async16(dst + kc * 2048, src + kc * 8);
                            if constexpr (SPLIT) cp_async16(dst + C::PART_BYTES + kc * 2048, src + kp + kc * 8);
                        }
                    }
                    if (++l_c == nkc) {
                        l_c = 0;
                        ++l_mt;
                    }
                }
                ++l_step;
                cp_async_commit();
            };
            // accumulator of M tile mt -> window scratch of every probe whose window holds the pixel
            auto drain = [&](int mt) {
                tc::fence_after_sync();
                const int q = warp & 3, h = warp >> 2;  // lane quarter, half of the N columns
                const int idx = mt * 128 + 32 * q + lane;
                const int ty = idx / tw, tx = idx - ty * tw;
                float2 *wh = a.win + ((size_t)slot * G + h * (G / 2)) * (NW * NW);  // this half's windows
#pragma unroll
                for (int c16 = 0; c16 < N / 32; ++c16) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((mt & 1) * N + h * (N / 2) + c16 * 16), v);
                    if (idx < npx) {
#pragma unroll
                        for (int pp = 0; pp < 8; ++pp) {
                            const int pl = c16 * 8 + pp;  // probe h G/2 + pl
                            const int o = wofs[h * (G / 2) + pl];
                            const int wy = ty - (o >> 16), wx = tx - (o & 0xffff);
                            if ((unsigned)wy < (unsigned)NW && (unsigned)wx < (unsigned)NW)
                                wh[pl * (NW * NW) + wy * NW + wx] = make_float2(v[2 * pp], v[2 * pp + 1]);
                        }
                    }
                }
                tc::fence_before_sync();
            };
#pragma unroll
            for (int l = 0; l < S - 1; ++l) load();
            int mt = m0, c = 0;  // the M tile and K chunk of step ls
            for (int ls = 0; ls < nsteps; ++ls) {
                const uint32_t s = st0 + ls;
                cp_async_wait<S - 2>();
                tc::fence_proxy_async();
                if (__syncthreads_or(my_fail)) {
                    dead = true;
                    break;
                }
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
                load();  // step ls + S - 1
                if (c == 0 && mt > m0) drain(mt - 1);  // the previous tile of this unit
                if (++c == nkc) {
                    c = 0;
                    ++mt;
                }
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
        // the bins' pixel lists (16-bit) in the shared memory past the windows and the exchange, where
        // the ring and the coefficient operand were, when they fit there: loaded with the first windows,
        // read by every pass of this unit instead of global memory (2.11 -> 2.08 ms on the FP16
        // carbon scan)
        constexpr size_t EPI16 = (C::EPI + 15) & ~(size_t)15;
        const int n16 = a.out && a.bin_idx16 ? (a.n_bin_idx + 7) / 8 : 0;  // 16-byte pieces
        const uint16_t *sidx = n16 > 0 && EPI16 + (size_t)n16 * 16 <= C::region0(kp)
                                   ? reinterpret_cast<const uint16_t *>(sm + EPI16)
                                   : nullptr;
        for (int e0 = 0; e0 < nvalid; e0 += C::EW) {
            const int ne = min(C::EW, nvalid - e0);
            // the windows in 16-byte pieces (two pixels of a row), every piece in flight at once
            for (int i = tid; i < ne * (NW * NW / 2); i += BLOCK) {
                const int e = i / (NW * NW / 2), u = 2 * (i - e * (NW * NW / 2));
                cp_async16(win + (e * NW + u / NW) * PW + (u & (NW - 1)), a.win + ((size_t)slot * G + meta[168 + e0 + e]) * (NW * NW) + u);
            }
            if (sidx && e0 == 0)
                for (int i = tid; i < n16; i += BLOCK) cp_async16(sm + EPI16 + (size_t)i * 16, a.bin_idx16 + (size_t)i * 8);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            window_epilogue<NW, NW, BLOCK, C::EW, PW>(a, win, ex, twf, twf, ne, meta + 200 + e0, tid, sidx);
            __syncthreads();
        }
    }
    // the last CTA to finish has seen every unit taken (or a wait ran out, and the host zeroes the
    // counters): it zeroes both counters for the next launch
    if (tid == 0 && atomicAdd(ctas_done, 1) == (int)gridDim.x - 1) {
        *next_unit = 0;
        *ctas_done = 0;
    }
    cp_async_wait<0>();
    __syncthreads();
    if (dead && tid == 0 && st > 0) tc::mbar_wait_bounded(&mbar[(st - 1) % S], ((st - 1) / S) & 1, TC_WAIT_CYCLES);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}


// persistent grid of a scan launch (0 if the shape does not fit) and the launch itself
template <int NW, int MODE, int SH = 0>
static int tc_grid(int kp, int scan_px, int scan_py) {
    using C = TcCfg<NW, MODE == TC_SPLIT, SH>;
    const size_t smem = C::smem(kp);
    if (smem > 227 * 1024) return 0;
    if (allow_max_dynamic_smem(k_scan_tc<NW, MODE, SH>) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_scan_tc<NW, MODE, SH>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        return 0;
    // Resident CTAs per SM from the kernel's own limits.  The runtime's occupancy query reports one
    // CTA per SM for every kernel that uses tcgen05, but CTAs whose registers, shared memory and
    // TMEM columns fit do run side by side (each allocates TMEM_COLS of the SM's 512 columns; an
    // allocation that does not fit waits for another CTA to free its columns).
    cudaFuncAttributes fa;
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&fa, k_scan_tc<NW, MODE, SH>) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
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

template <int NW, int MODE, int SH = 0>
static cudaError_t tc_launch(int grid, const ScanArgs &a, cudaStream_t s) {
    using C = TcCfg<NW, MODE == TC_SPLIT, SH>;
    const size_t smem = C::smem(a.kp);
    cudaError_t e = allow_max_dynamic_smem(k_scan_tc<NW, MODE, SH>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_scan_tc<NW, MODE, SH>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    k_scan_tc<NW, MODE, SH><<<grid, C::BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace prism
