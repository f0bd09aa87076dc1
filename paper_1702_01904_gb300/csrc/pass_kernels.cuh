// pass_kernels.cuh -- the two streaming passes of one multislice step, as templates over the FFT
// length and the launch shape (threads or columns per CTA, cp.async staging).  kernels_build.cu
// instantiates the default shapes; kernels_tune.cu the alternatives the autotuner times.
//
// One multislice step (Eq. Multislice, transmit then propagate) is split into two streaming
// passes over a wave stack [batch][ny][nx] kept in the mixed domain (x-Fourier, y-real):
//   row pass p   : psi_p = IFFT_x(Phi_{p-1});  Z_p = FFT_x(psi_p * t_p)
//   column pass p: Phi_p = IFFT_y( P_p(q) * FFT_y(Z_p) ) / (nx ny)
// so that IFFT_x(Phi_p) is the real-space wave after slice p.  Each pass reads and writes the
// stack once; the 1/(nx ny) of the inverse transform is folded into the propagator table.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"
#include "tc.cuh"  // mbarrier and TMA helpers

namespace prism {

// ------------------------------------------------------------------ launch geometry
// Persistent launches: as many CTAs as can be resident at once (occupancy x SM count), each
// looping over its share of rows or column tiles.
template <class K>
static cudaError_t set_smem(K kernel, size_t smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

template <class K>
static cudaError_t persistent_grid(K kernel, int threads, size_t smem, long long work, int *grid, bool persist = true) {
    cudaError_t e = set_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    if (!persist) {
        *grid = (int)work;
        return cudaSuccess;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    const long long cap = (long long)(per_sm > 0 ? per_sm : 1) * sm_count();
    *grid = (int)(work < cap ? work : cap);
    return cudaSuccess;
}

// ------------------------------------------------------------------ async copies
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------ row pass
// Each slot (T lanes of one warp) owns one row at a time and walks rows row0, row0 + stride, ...
// The next row streams into the slot's shared-memory staging buffer (cp.async) while the current
// row is transformed; the slice's transmission row is loaded into registers before the inverse
// FFT so that its latency hides behind the transform.
template <int NX>
constexpr int row_default_threads() { return NX >= 512 ? 128 : 256; }

// FFT radix variant (DftSplit, bit 0 forward, bit 1 inverse) of the default launchers: at N = 2048
// both transforms put a radix-4 stage first in their 64- and 32-point register DFTs (row pass 20.0
// -> 8.6 ms per 529-beam launch, column pass 6.4 -> 6.1 ms); elsewhere the default split
__host__ __device__ constexpr int default_fft_variant(int n) { return n >= 2048 ? 3 : 0; }

// THR threads per CTA, STG: cp.async staging of the next row, TM: bulk-copy (TMA) staging of the
// next row's two kept quarters (launch shape only: every variant computes bitwise the same rows)
template <int NX, int THR = row_default_threads<NX>(), bool STG = false, bool TM = false>
struct RowCfg {
    using FS = FftShape<NX>;
    static constexpr int T = FS::T;
    static constexpr int E = FS::E;
    static constexpr bool STAGE = STG;        // cp.async staging of the next row
    static constexpr bool TMA = TM;           // bulk staging of [0, NX/4) and [3NX/4, NX) (one slot = one warp)
    static constexpr bool PERSIST = true;     // grid = resident CTAs, each looping over rows
    static constexpr bool T_EARLY = E <= 32;  // E extra complex registers for t_p
    static constexpr int THREADS = THR;
    static constexpr int SLOTS = THREADS / T;  // rows per CTA in flight
    static constexpr int EXF = FS::N1 * (FS::N2 + 1);
    static constexpr int EXI = FS::N2 * (FS::N1 + 1);
    static constexpr int EX = EXF > EXI ? EXF : EXI;
    static constexpr int SLOT_F2 = (TMA ? NX / 2 : STAGE ? NX : 0) + EX;  // staging row + exchange, float2
    // at N = 2048 the two stage-twiddle tables (32 KB) would hold the CTAs to 2 per SM: there they are
    // read through L1 (read-only path), interleaved with the exchange stores, for 3 CTAs per SM
    static constexpr bool L1TW = NX >= 2048;
    static constexpr int TW_MODE = L1TW ? TW_GLOBAL : TW_SMEM;
    static constexpr int TWF2 = L1TW ? 0 : 2 * NX;  // float2 of twiddles in shared memory
    static constexpr size_t SMEM = (size_t)(TWF2 + SLOTS * SLOT_F2) * sizeof(float2);
};

// bulk-staged rows give up after this many SM cycles (about a second) and report it
constexpr long long ROW_TMA_WAIT_CYCLES = 2000000000LL;

// BL: the kept columns are exactly |kx| < NX/4 (kx_half == NX/4), known at compile time
// RV: split variants of the register DFTs (DftSplit) of the forward (bit 0) and the inverse (bit 1)
// transform: the same transforms, rounded differently
template <int NX, int MODE, int THR = row_default_threads<NX>(), bool STG = false, bool BL = false, bool TM = false, int RV = 0>
__global__ void __launch_bounds__(THR) k_row(const __grid_constant__ RowArgs a) {
    using C = RowCfg<NX, THR, STG, TM>;
    using FS = FftShape<NX>;
    using Fwd = FwdFft<NX, RV & 1>;
    using Inv = InvFft<NX, (RV >> 1) & 1>;
    constexpr int T = C::T, E = FS::E;
    static_assert(!TM || (BL && T == 32 && MODE != ROW_PLANE), "bulk staging: compile-time band, one slot per warp");
    // with the compile-time band the inverse transform's out-of-band inputs are exact zeros
    constexpr unsigned long long ZIN = BL && MODE != ROW_PLANE ? band_zero_mask<Inv, NX>(true) : 0ull;
    extern __shared__ float2 smem[];
    __shared__ __align__(8) uint64_t rbar[C::SLOTS];  // TM: a slot's next row has landed
    uint32_t rphase = 0;
    const int slot = threadIdx.x / T, t = threadIdx.x % T;
    if constexpr (C::TMA) {
        if (t == 0) tc::mbar_init(&rbar[slot], 1);
        tc::fence_mbar_init();
    }
    // FFT stage twiddles (forward, inverse) in shared memory (or read through L1), then one region
    // per slot
    const float2 *twf = a.tw_fwd, *twi = a.tw_inv;
    if constexpr (!C::L1TW) {
        float2 *tf = smem, *ti = smem + NX;
        for (int i = threadIdx.x; i < NX; i += C::THREADS) {
            tf[i] = a.tw_fwd[i];
            ti[i] = a.tw_inv[i];
        }
        __syncthreads();
        twf = tf;
        twi = ti;
    }
    float2 *stg = smem + C::TWF2 + slot * C::SLOT_F2;
    float2 *exbuf = stg + (C::TMA ? NX / 2 : C::STAGE ? NX : 0);
    WarpExchange<FS::N1, FS::N2, T> exF{exbuf};
    WarpExchange<FS::N2, FS::N1, T> exI{exbuf};
    const int stride = gridDim.x * C::SLOTS;
    const int iters = (a.n_rows + stride - 1) / stride;  // uniform over the grid
    const int row0 = blockIdx.x * C::SLOTS + slot;

    // rows past the end are redone on the last row without storing, so every lane of a warp
    // takes part in every exchange
    auto locate = [&](int row, int &b, int &y) {
        row = row < a.n_rows ? row : a.n_rows - 1;
        if (MODE == ROW_OUT && a.downsample == 2) {
            const int nyh = a.ny >> 1;
            b = row / nyh;
            y = 2 * (row - b * nyh);
        } else {
            b = row / a.ny;
            y = row - b * a.ny;
        }
    };
    // kx (FFT order) that can be non-zero in the mixed domain: the column pass zeroes the others
    auto keep = [&](int e) {
        if constexpr (BL) return e < NX / 4 || e > NX - NX / 4;
        else return a.kx_half == 0 || e < a.kx_half || e > NX - a.kx_half;
    };
    // stage a whole row into this slot's buffer: NX*8 bytes in 16-byte pieces, E/2 per lane (pieces
    // of two zero columns are skipped)
    auto stage = [&](int row) {
        int b, y;
        locate(row, b, y);
        const float2 *w = a.wave + ((size_t)b * a.ny + y) * NX;
#pragma unroll
        for (int k = 0; k < E / 2; ++k) {
            const int e = 2 * (t + T * k);
            if (keep(e) || keep(e + 1)) cp_async16(stg + e, w + e);
        }
        cp_async_commit();
    };

    // bulk (TMA) staging of a row's two kept quarters, [0, NX/4) then [3NX/4, NX), into the slot's
    // buffer: lane 0 arms the slot's barrier with the byte count and issues both copies
    auto bulk = [&](int row) {
        if (t == 0) {
            int b, y;
            locate(row, b, y);
            const float2 *w = a.wave + ((size_t)b * a.ny + y) * NX;
            tc::fence_proxy_async();  // the buffer's generic reads (previous row) before the async writes
            tc::mbar_arrive_expect_tx(&rbar[slot], (uint32_t)(NX / 2 * sizeof(float2)));
            tc::bulk_load(stg, w, (uint32_t)(NX / 4 * sizeof(float2)), &rbar[slot]);
            tc::bulk_load(stg + NX / 4, w + 3 * NX / 4, (uint32_t)(NX / 4 * sizeof(float2)), &rbar[slot]);
        }
    };
    if constexpr (C::TMA) bulk(row0);
    if constexpr (MODE != ROW_PLANE && C::STAGE) stage(row0);
    for (int it = 0; it < iters; ++it) {
        const int row = row0 + it * stride;
        const bool valid = row < a.n_rows;
        int b, y;
        locate(row, b, y);
        float2 v[E];
        if constexpr (MODE == ROW_PLANE) {
            // psi_b(r) = exp(2 pi i (m f x / nx + n f y / ny)), phase reduced exactly in integers
            const int m = a.beam_mn[2 * (a.beam0 + b)];
            const int n = a.beam_mn[2 * (a.beam0 + b) + 1];
            const long long den = (long long)NX * a.ny;
            long long ky = ((long long)n * a.f_y * y) % a.ny;
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
                v[r] = cmul(make_float2(c, s), __ldcg(tp + x));
            }
        } else {
            if constexpr (C::TMA) {
                const uint32_t ph = rphase;
                rphase ^= 1;
                const bool ok = tc::mbar_wait_bounded(&rbar[slot], ph, ROW_TMA_WAIT_CYCLES);
                if (__any_sync(0xffffffffu, !ok)) {
                    // report, give the copies in flight one more bounded wait, leave (the whole warp)
                    if (t == 0 && a.err) atomicOr(a.err, 4);
                    tc::mbar_wait_bounded(&rbar[slot], ph, ROW_TMA_WAIT_CYCLES);
                    return;
                }
                static_for<E>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int cls = BandClass<Inv, NX>::of(r, true);
                    // a register's elements lie in one 32-aligned block, so one quarter holds them all
                    constexpr int off = Inv::in_elem(r, 0) < NX / 4 ? 0 : NX / 2;
                    const int e = Inv::in_elem(r, t);
                    if constexpr (cls == BAND_OUT) v[r] = make_float2(0.f, 0.f);
                    else if constexpr (cls == BAND_IN) v[r] = stg[e - off];
                    else v[r] = keep(e) ? stg[e - off] : make_float2(0.f, 0.f);
                });
                __syncwarp();  // the buffer is refilled next
                if (it + 1 < iters) bulk(row + stride);
            } else if constexpr (C::STAGE) {
                cp_async_wait_all();
                __syncwarp();
                static_for<E>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int cls = BL ? BandClass<Inv, NX>::of(r, true) : BAND_MIXED;
                    const int e = Inv::in_elem(r, t);
                    if constexpr (cls == BAND_OUT) v[r] = make_float2(0.f, 0.f);
                    else if constexpr (cls == BAND_IN) v[r] = stg[e];
                    else v[r] = keep(e) ? stg[e] : make_float2(0.f, 0.f);
                });
                __syncwarp();  // the buffer is refilled next
                if (it + 1 < iters) stage(row + stride);
            } else {
                const float2 *w = a.wave + ((size_t)b * a.ny + y) * NX;
                static_for<E>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int cls = BL ? BandClass<Inv, NX>::of(r, true) : BAND_MIXED;
                    const int e = Inv::in_elem(r, t);
                    if constexpr (cls == BAND_OUT) v[r] = make_float2(0.f, 0.f);
                    else if constexpr (cls == BAND_IN) v[r] = __ldcs(w + e);
                    else v[r] = keep(e) ? __ldcs(w + e) : make_float2(0.f, 0.f);
                });
            }
            if constexpr (MODE == ROW_STD) {
                // t_p is shared by all beams: L2-cached, not L1 (keeps L1 for the FFT's traffic)
                const float2 *tp = a.trans + (size_t)y * NX;
                if constexpr (C::T_EARLY) {
                    float2 tv[E];
#pragma unroll
                    for (int r = 0; r < E; ++r) tv[r] = __ldcg(tp + Inv::out_elem(r, t));
                    Inv::template run<decltype(exI), C::TW_MODE, ZIN>(v, t, twi, a.tw, exI);
#pragma unroll
                    for (int r = 0; r < E; ++r) v[r] = cmul(v[r], tv[r]);
                } else {
                    Inv::template run<decltype(exI), C::TW_MODE, ZIN>(v, t, twi, a.tw, exI);
#pragma unroll
                    for (int r = 0; r < E; ++r) v[r] = cmul(v[r], __ldcg(tp + Inv::out_elem(r, t)));
                }
            } else {
                Inv::template run<decltype(exI), C::TW_MODE, ZIN>(v, t, twi, a.tw, exI);
            }
        }
        if constexpr (MODE == ROW_OUT) {
            // real-space exit wave; with downsample 2 the band limit (|k| < n/4) makes every second
            // sample the exact half-resolution wave of the inner Fourier square
            if (valid) {
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
            }
        } else {
            Fwd::template run<decltype(exF), C::TW_MODE>(v, t, twf, a.tw, exF);
            if (valid) {
                float2 *w = a.wave + ((size_t)b * a.ny + y) * NX;
                static_for<E>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int cls = BL ? BandClass<Fwd, NX>::of(r, false) : BAND_MIXED;
                    const int e = Fwd::out_elem(r, t);
                    if constexpr (cls == BAND_IN) __stcs(w + e, v[r]);
                    else if constexpr (cls == BAND_MIXED) {
                        if (keep(e)) __stcs(w + e, v[r]);
                    }
                });
            }
        }
    }
}

template <int NX, int MODE, int THR, bool STG, bool BL, bool TM = false, int RV = 0>
static cudaError_t row_go_bl(const RowArgs &a, cudaStream_t s) {
    using C = RowCfg<NX, THR, STG, TM>;
    int grid = 0;
    cudaError_t e = persistent_grid(k_row<NX, MODE, THR, STG, BL, TM, RV>, C::THREADS, C::SMEM, (a.n_rows + C::SLOTS - 1) / C::SLOTS,
                                    &grid, C::PERSIST);
    if (e != cudaSuccess) return e;
    k_row<NX, MODE, THR, STG, BL, TM, RV><<<grid, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

// TM: bulk staging where it applies (the compile-time band, one slot per warp, rows read from the
// wave); elsewhere the same shape without it, which computes the same rows
template <int NX, int MODE, int THR = row_default_threads<NX>(), bool STG = false, bool TM = false, int RV = 0>
static cudaError_t row_go(const RowArgs &a, cudaStream_t s) {
    using C = RowCfg<NX, THR, STG, TM>;
    if constexpr (C::SMEM > 227 * 1024 || THR % C::T != 0 || THR > 1024) {
        return cudaErrorInvalidConfiguration;
    } else {
        // the compile-time band for the default aperture (aa_frac 1/2 on a square grid: |kx| < NX/4)
        if constexpr (NX >= 64) {
            if (a.kx_half * 4 == NX) {
                if constexpr (TM && C::T == 32 && MODE != ROW_PLANE) return row_go_bl<NX, MODE, THR, STG, true, true, RV>(a, s);
                else return row_go_bl<NX, MODE, THR, STG, true, false, RV>(a, s);
            }
        }
        return row_go_bl<NX, MODE, THR, STG, false, false, RV>(a, s);
    }
}

// ------------------------------------------------------------------ column pass
// A CTA owns W interleaved columns (one tile, NY x W) at a time and walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; the next tile streams into a shared-memory staging buffer
// (cp.async, 16-byte pieces of the W*8-byte row segments) while the current one is transformed.
template <int NY>
constexpr int col_default_w() { return NY >= 1024 ? 8 : 16; }
// the default column launcher stages the next tile by cp.async, except at N = 2048 (8 columns
// unstaged: 6.1 ms per 529-beam launch against 7.5 ms for 4 columns staged)
template <int NY>
constexpr bool col_default_stg() { return NY < 2048; }

// WC interleaved columns per CTA, STG: cp.async staging of the next tile, MB: CTAs per SM the
// register allocation must allow (0: the default rule), TM: the next tile staged by TMA instead
// (NY / BOXR boxes of W = 4 or 8 columns x BOXR rows, one thread issues them) -- launch shape only
template <int NY, int WC = col_default_w<NY>(), bool STG = true, int MB = 0, bool TM = false>
struct ColCfg {
    using FS = FftShape<NY>;
    static constexpr int W = WC;           // interleaved columns per CTA
    static constexpr int THREADS = FS::T * W;
    static constexpr bool TMA = TM;
    static constexpr bool STAGE = STG || TM;  // staging of the next tile (cp.async or TMA)
    static constexpr int BOXR = NY < 256 ? NY : 256;  // rows per TMA box
    // TMA-staged shapes of a square split (forward and inverse use the same table, the inverse its
    // conjugate): one twiddle table in shared memory, read interleaved with the exchange stores;
    // else the tables through L1 (read-only path)
    static constexpr bool SMEM_TW = TM && FS::N1 == FS::N2;
    static constexpr int TW_MODE = SMEM_TW ? TW_SMEM_SEQ : TW_GLOBAL;
    static constexpr bool PERSIST = true;  // grid = resident CTAs, each looping over tiles
    static constexpr int MINB = MB > 0 ? MB : (PERSIST || STAGE) ? 1 : 2;  // CTAs per SM the registers must allow
    static constexpr int EX = ColExSize<NY, W>::value;
    static_assert(EX >= NY * W, "the exchange buffer holds a whole tile (TMA stores)");
    static_assert(!TM || (FS::T % (32 / W) == 0 && FS::T * W >= 32), "TMA stores: whole warps of lanes per column");
    static constexpr size_t SMEM = (size_t)((SMEM_TW ? NY : 0) + (STAGE ? NY * W : 0) + EX) * sizeof(float2);
};

// TMA staging gives up after this many SM cycles (about a second) and reports it in the error word
constexpr long long COL_TMA_WAIT_CYCLES = 2000000000LL;

// BL: every column keeps at most |ky| < NY/4 (band4), known at compile time
// RV: split variants of the register DFTs (DftSplit) of the forward (bit 0) and the inverse (bit 1)
// transform: the same transforms, rounded differently
template <int NY, int MODE, int WC = col_default_w<NY>(), bool STG = true, int MB = 0, bool BL = false, bool TM = false, int RV = 0>
__global__ void __launch_bounds__(ColCfg<NY, WC, STG, MB, TM>::THREADS, ColCfg<NY, WC, STG, MB, TM>::MINB) k_col(const __grid_constant__ ColArgs a) {
    using C = ColCfg<NY, WC, STG, MB, TM>;
    using FS = FftShape<NY>;
    using Fwd = FwdFft<NY, RV & 1>;
    using Inv = InvFft<NY, (RV >> 1) & 1>;
    constexpr int W = C::W, E = FS::E, THREADS = C::THREADS;
    extern __shared__ __align__(128) float2 smem_c[];
    float2 *smem = smem_c;
    __shared__ __align__(8) uint64_t tbar;  // TMA staging: the tile's boxes have landed
    __shared__ int s_next;                  // TMA staging with a tile counter: the next tile
    uint32_t tphase = 0;
    if constexpr (C::TMA) {
        if (threadIdx.x == 0) {
            tc::mbar_init(&tbar, 1);
            tc::fence_mbar_init();
        }
        __syncthreads();
    }
    // FFT stage twiddles (forward, inverse), staging tile [NY][W], exchange
    const float2 *twf = a.tw_fwd, *twi = a.tw_inv;
    if constexpr (C::SMEM_TW) {
        float2 *tws = smem;
        for (int i = threadIdx.x; i < NY; i += THREADS) tws[i] = a.tw_fwd[i];
        __syncthreads();
        twf = tws;
        twi = tws;  // the square split's inverse table holds the same values
    }
    float2 *stg = smem + (C::SMEM_TW ? NY : 0);
    float2 *exb = stg + (C::STAGE ? NY * W : 0);
    const int c = threadIdx.x % W, t = threadIdx.x / W, lane = threadIdx.x & 31;
    ColExchange<FS::N1, FS::N2, W> exF{exb, c};
    ColExchange<FS::N2, FS::N1, W> exI{exb, c};
    // column tiles of W columns: all of them, or (kx_half > 0) only the low ones [0, lo W) and the
    // high ones [hs W, nx), which hold every kx the anti-aliasing aperture lets through
    const int tw_all = a.nx / W;
    int lo = tw_all, hs = tw_all;
    if (a.kx_half > 0) {
        lo = (a.kx_half + W - 1) / W;
        hs = (a.nx - a.kx_half + 1) / W;
        if (lo >= hs) lo = hs = tw_all;
    }
    const int tiles_x = lo + (tw_all - hs);
    const int ntiles = tiles_x * a.batch;
    const int iters = (ntiles + gridDim.x - 1) / gridDim.x;  // uniform over the grid

    // tiles past the end are redone on the last tile without storing (every thread joins every
    // __syncthreads of the exchange)
    auto locate = [&](int tile, int &b, int &kx0) {
        tile = tile < ntiles ? tile : ntiles - 1;
        b = tile / tiles_x;
        const int ti = tile - b * tiles_x;
        kx0 = (ti < lo ? ti : hs + (ti - lo)) * W;
    };
    auto stage = [&](int tile) {
        int b, kx0;
        locate(tile, b, kx0);
        if constexpr (C::TMA) {
            // NY / BOXR boxes of the tile's rows; x = 2 kx0 floats, kx0 a multiple of W (16-byte rule)
            if (threadIdx.x == 0) {
                tc::fence_proxy_async();  // the buffer's generic reads (previous tile) before the async writes
                tc::mbar_arrive_expect_tx(&tbar, (uint32_t)(NY * W * sizeof(float2)));
                const CUtensorMap *map = W == 8 ? &a.wave_map : &a.wave_map4;  // boxes of W columns
                for (int y0 = 0; y0 < NY; y0 += C::BOXR) tc::tma_load_3d(stg + y0 * W, map, 2 * kx0, y0, b, &tbar);
            }
            return;
        }
        const float2 *base = a.wave + (size_t)b * NY * a.nx + kx0;
        constexpr int PIECES = NY * W / 2;  // 16-byte pieces of the tile
#pragma unroll
        for (int k = 0; k < PIECES / THREADS; ++k) {
            const int i = threadIdx.x + THREADS * k;
            const int row = i / (W / 2), cc = 2 * (i % (W / 2));
            cp_async16(stg + row * W + cc, base + (size_t)row * a.nx + cc);
        }
        cp_async_commit();
    };

    if constexpr (C::TMA) {
        // TMA writes 128-byte aligned boxes: a misplaced buffer is reported, never copied into
        if (tc::smem_u32(stg) & 127) {
            if (threadIdx.x == 0 && a.err) atomicOr(a.err, 2);
            return;
        }
    }
    // TMA-staged shapes: the propagator's y factor of every register this thread transforms (rows
    // t + T r, the same in every tile) loaded once into registers
    float2 pyr[E];
    if constexpr (C::TMA && MODE == COL_STD) {
        static_for<E>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            constexpr int cls = BL ? BandClass<Fwd, NY>::of(r, false) : BAND_MIXED;
            if constexpr (cls != BAND_OUT) pyr[r] = __ldg(a.prop_y + Fwd::out_elem(r, t));
        });
    }
    // TMA-staged shapes given a tile counter take their tiles from it, each one tile ahead (the
    // tile the prefetch loads), instead of by a fixed stride: the CTAs sharing an SM are not issued
    // equally, and with fixed shares the favoured ones finished early (per-CTA times of 170 to
    // 204 us in one launch).  Which CTA transforms a tile changes no result.
    const bool dyn = C::TMA && a.tile_ctr != nullptr;
    int cur = blockIdx.x;
    if (dyn) {
        if (threadIdx.x == 0) s_next = atomicAdd(a.tile_ctr, 1);
        __syncthreads();
        cur = s_next;
    }
    if constexpr (MODE != COL_PROBE && C::STAGE) {
        if (cur < ntiles) stage(cur);
    }
    // without persistence every CTA owns exactly one tile and there is no loop (a loop would let
    // the compiler hoist the loop-invariant twiddle loads and hold them in registers)
    const int n_it = C::PERSIST || C::STAGE ? iters : 1;
    for (int it = 0; dyn ? cur < ntiles : it < n_it; ++it) {
        const int tile = dyn ? cur : blockIdx.x + it * gridDim.x;
        const bool valid = tile < ntiles;
        int b, kx0;
        locate(tile, b, kx0);
        const int kx = kx0 + c;
        // TMA-staged shapes store their tile from the exchange buffer, one box per warp: before the
        // exchange is written again (right after the barrier that follows the tile's arrival), every
        // warp's store of the previous tile must have read it
        if constexpr (C::TMA) {
            if (lane == 0) tc::bulk_wait_read_all();
        }

        float2 *col = a.wave + (size_t)b * NY * a.nx + kx;
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
            if constexpr (C::STAGE) {
                if constexpr (C::TMA) {
                    const uint32_t ph = tphase;
                    tphase ^= 1;
                    const bool ok = tc::mbar_wait_bounded(&tbar, ph, COL_TMA_WAIT_CYCLES);
                    if (__syncthreads_or(!ok)) {
                        // report, give the boxes in flight one more bounded wait, let the stores
                        // issued so far finish, leave (every thread)
                        if (threadIdx.x == 0 && a.err) atomicOr(a.err, 2);
                        tc::mbar_wait_bounded(&tbar, ph, COL_TMA_WAIT_CYCLES);
                        if (lane == 0) tc::bulk_wait_all();
                        return;
                    }
                } else {
                    cp_async_wait_all();
                    __syncthreads();
                }
#pragma unroll
                for (int r = 0; r < E; ++r) v[r] = stg[Fwd::in_elem(r, t) * W + c];
                if constexpr (!C::TMA) {
                    __syncthreads();  // the staging buffer is refilled next
                    if (it + 1 < iters) stage(tile + gridDim.x);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) v[r] = col[(size_t)Fwd::in_elem(r, t) * a.nx];
            }
            if constexpr (C::TMA) {
                // the barrier after the tile's arrival ordered every earlier use of the exchange
                // before its writes here (no leading barrier), and the barrier after them is the
                // point where every thread has read the staging buffer: its refill starts there
                Fwd::template run<decltype(exF), C::TW_MODE, 0ull, false>(v, t, twf, a.tw, exF, [&] {
                    if (dyn) {
                        // the next tile, read by every thread after the inverse transform's barriers
                        if (threadIdx.x == 0) {
                            const int nt = atomicAdd(a.tile_ctr, 1);
                            s_next = nt;
                            if (nt < ntiles) stage(nt);
                        }
                    } else if (it + 1 < iters) {
                        stage(tile + gridDim.x);
                    }
                });
            } else {
                Fwd::template run<decltype(exF), C::TW_MODE>(v, t, twf, a.tw, exF);
            }
            // Fresnel propagator exp(-i pi lambda t |q|^2) (separable) inside the anti-aliasing
            // aperture, which on column kx is |ky| <= aa_kmax[kx]
            const float2 px = __ldg(a.prop_x + kx);
            const int kymax = __ldg(a.aa_kmax + kx);
            static_for<E>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr int cls = BL ? BandClass<Fwd, NY>::of(r, false) : BAND_MIXED;
                if constexpr (cls == BAND_OUT) {
                    v[r] = make_float2(0.f, 0.f);  // outside |ky| < NY/4 on every column
                } else {
                    const int ky = Fwd::out_elem(r, t);
                    const int kys = ky < (NY >> 1) ? ky : ky - NY;
                    const int aky = kys < 0 ? -kys : kys;
                    const float2 py = C::TMA && MODE == COL_STD ? pyr[r] : __ldg(a.prop_y + ky);
                    v[r] = aky <= kymax ? cmul(v[r], cmul(px, py)) : make_float2(0.f, 0.f);
                }
            });
            if constexpr (MODE == COL_DETECT) {
                if (valid) {
                    float *icol = a.inten + (size_t)b * NY * a.nx + kx;
#pragma unroll
                    for (int r = 0; r < E; ++r) icol[(size_t)Fwd::out_elem(r, t) * a.nx] = v[r].x * v[r].x + v[r].y * v[r].y;
                }
                continue;
            }
        }
        // after the propagator the out-of-band registers are exact zeros (band4, compile-time band)
        constexpr unsigned long long ZC = BL && MODE != COL_PROBE ? band_zero_mask<Fwd, NY>(false) : 0ull;
        Inv::template run<decltype(exI), C::TW_MODE, ZC>(v, t, twi, a.tw, exI);
        if constexpr (MODE == COL_PROBE) {
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = cscale(v[r], a.probe_scale);
        }
        if constexpr (C::TMA) {
            // result register r of lane t is row t + T r: it goes back to the exchange slot (t, r) that
            // this thread alone read in the inverse transform's second stage, so no barrier is needed
            // before the writes; the slots of a warp's lanes (T / (32 / W) consecutive t) are one
            // contiguous box of the store map, [t][E + 1][W], which lane 0 stores once the warp's
            // writes are visible to the async proxy
            static_assert(Inv::I == 1 && Inv::SPLIT1 == FS::T && Inv::SPLIT2 == E, "result row = t + T r");
            constexpr int TPW = 32 / W;  // lanes t per warp
#pragma unroll
            for (int r = 0; r < E; ++r) exb[(t * (E + 1) + r) * W + c] = v[r];
            tc::fence_proxy_async();  // the generic writes before the async-proxy reads
            __syncwarp();
            if (lane == 0 && valid) {
                const CUtensorMap *map = W == 8 ? &a.out_map : &a.out_map4;
                const int t0 = (threadIdx.x >> 5) * TPW;
                tc::tma_store_4d(map, 2 * kx0, 0, t0, b, exb + t0 * (E + 1) * W);
                tc::bulk_commit();
            }
        } else if (valid) {
#pragma unroll
            for (int r = 0; r < E; ++r) col[(size_t)Inv::out_elem(r, t) * a.nx] = v[r];
        }
        if (dyn) cur = s_next;
    }
    if constexpr (C::TMA) {
        if (lane == 0) tc::bulk_wait_all();  // the last stores complete before the CTA leaves
        // the last CTA to finish has seen every tile taken: it zeroes the counter for the next launch
        if (dyn && threadIdx.x == 0 && atomicAdd(a.tile_ctr + 1, 1) == (int)gridDim.x - 1) {
            a.tile_ctr[0] = 0;
            a.tile_ctr[1] = 0;
        }
    }
}

// column tiles a launch processes (the kernel's tile enumeration)
static inline long long col_tiles(int nx, int w, int kx_half, int batch) {
    int lo = nx / w, hs = nx / w;
    if (kx_half > 0) {
        lo = (kx_half + w - 1) / w;
        hs = (nx - kx_half + 1) / w;
        if (lo >= hs) lo = hs = nx / w;
    }
    return (long long)(lo + (nx / w - hs)) * batch;
}

template <int NY, int MODE, int WC = col_default_w<NY>(), bool STG = true, int MB = 0, bool TM = false, int RV = 0>
static cudaError_t col_go(const ColArgs &a, cudaStream_t s) {
    using C = ColCfg<NY, WC, STG, MB, TM>;
    if constexpr (C::SMEM > 227 * 1024 || C::THREADS > 1024 || (TM && (MODE != COL_STD || (WC != 4 && WC != 8) || NY % C::BOXR))) {
        return cudaErrorInvalidConfiguration;
    } else {
        if (a.nx % C::W) return cudaErrorInvalidValue;
        // the maps must describe this wave stack with boxes of W columns x BOXR rows
        if (TM && !a.wave_map_ok) return cudaErrorInvalidValue;
        int grid = 0;
        const long long work = col_tiles(a.nx, C::W, a.kx_half, a.batch);
        cudaError_t e;
        if constexpr (NY >= 64 && MODE != COL_PROBE) {
            if (a.band4) {
                e = persistent_grid(k_col<NY, MODE, WC, STG, MB, true, TM, RV>, C::THREADS, C::SMEM, work, &grid, C::PERSIST);
                if (e != cudaSuccess) return e;
                k_col<NY, MODE, WC, STG, MB, true, TM, RV><<<grid, C::THREADS, C::SMEM, s>>>(a);
                return cudaGetLastError();
            }
        }
        e = persistent_grid(k_col<NY, MODE, WC, STG, MB, false, TM, RV>, C::THREADS, C::SMEM, work, &grid, C::PERSIST);
        if (e != cudaSuccess) return e;
        k_col<NY, MODE, WC, STG, MB, false, TM, RV><<<grid, C::THREADS, C::SMEM, s>>>(a);
        return cudaGetLastError();
    }
}


}  // namespace prism
