// params.h -- kernel parameter blocks and launcher declarations shared by the host engine
// (engine.cpp, plain C++) and the CUDA translation units.  Parameters travel by value in
// kernel parameter space (__grid_constant__), which keeps the 64 register-DFT twiddles in the
// constant bank.
#pragma once
#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace prism {

struct Tw64 {
    float2 w[64];   // W_64^j = exp(-2 pi i j / 64)
    // tangent form of the same twiddles, W_64^j = s (1 + i k) when |cos| >= |sin| (s = cos, k = tan;
    // (j mod 32) <= 8 or >= 24), else W_64^j = s (k + i) (s = sin, k = cot): sc[j] = (s, s), tk[j] = k
    float2 sc[64];
    float tk[64];
};

enum RowMode { ROW_STD = 0, ROW_PLANE = 1, ROW_OUT = 2 };
enum ColMode { COL_STD = 0, COL_PROBE = 1, COL_DETECT = 2 };

// Row pass over rows of length nx of a wave stack [batch][ny][nx] (x-Fourier between passes).
struct RowArgs {
    float2 *wave;              // [batch][ny][nx]
    const float2 *trans;       // t_p, [ny][nx]   (STD, PLANE)
    const float2 *tw_fwd;      // inter-stage twiddles of the forward split  [N1][N2]
    const float2 *tw_inv;      // inter-stage twiddles of the inverse split  [N2][N1]
    float2 *s_out;             // OUT: S-matrix [B][ny_s][nx_s]
    const int *beam_mn;        // PLANE: [B][2] (m, n)
    int ny;
    int n_rows;                // rows processed by this launch
    int f;                     // PLANE: interpolation factor along x
    int f_y;                   // PLANE: interpolation factor along y
    int beam0;                 // first beam of this batch (PLANE, OUT)
    int downsample;            // OUT
    int kx_half;               // > 0: only kx = -(kx_half-1) ... kx_half-1 of the mixed-domain wave are
                               // non-zero (the propagator's anti-aliasing aperture zeroes the rest):
                               // loads there are replaced by exact zeros and stores are skipped
                               // (STD, PLANE, OUT); 0: every kx
    int *err;                  // device error word: a TMA wait that ran out sets bit 2
    Tw64 tw;
};

// Column pass over columns of length ny.
struct ColArgs {
    CUtensorMap wave_map;      // TMA staging (STD): `wave` as FP32 [batch][ny][2 nx], boxes of 16 floats
                               // (8 columns) x min(ny, 256) rows x 1; valid when wave_map_ok
    CUtensorMap wave_map4;     // the same with boxes of 8 floats (4 columns)
    CUtensorMap out_map;       // TMA stores (STD): `wave` as FP32 [batch][lanes][regs][2 nx] with row
                               // y = lane + lanes * reg (lanes, regs: the column transform's threads
                               // and registers per column, col_fft_geometry), boxes of 16 floats x
                               // (regs + 1) x 32/8 x 1 -- one warp's rows of a finished tile in the
                               // padded exchange layout; the pad entry lies past `regs` and is not stored
    CUtensorMap out_map4;      // the same for 4 columns: boxes of 8 floats x (regs + 1) x 32/4 x 1
    float2 *wave;              // [batch][ny][nx]
    float *inten;              // DETECT: [batch][ny][nx] |Psi|^2 (scaled later)
    const float2 *prop_x;      // [nx]  exp(-i pi lambda dz qx^2)
    const float2 *prop_y;      // [ny]  exp(-i pi lambda dz qy^2) / (nx ny)
    const int *aa_kmax;        // [nx]  largest |ky| inside the AA aperture on column kx, -1 if none
    const float2 *tw_fwd;
    const float2 *tw_inv;
    const float2 *probe_base;  // PROBE: [ny][nx] A(q) exp(-i chi(q))
    const float2 *shift_x;     // PROBE: [batch][nx] exp(-2 pi i qx x0)
    const float2 *shift_y;     // PROBE: [batch][ny] exp(-2 pi i qy y0)
    int nx;
    int batch;
    float probe_scale;         // PROBE: 1 / (nx ny)
    int kx_half;               // > 0: only the column tiles holding kx = -(kx_half-1) ... kx_half-1 are
                               // processed (every other column is zero after the propagator); 0: all
    int band4;                 // 1: the aperture keeps |ky| < ny/4 on every column (aa_kmax < ny/4), so
                               // the column transforms may drop that band's complement at compile
                               // time (STD, DETECT)
    int wave_map_ok;           // 1: the four maps describe `wave` (the TMA-staged shapes may run)
    int *tile_ctr;             // TMA-staged shapes: [2] the next tile and the CTAs done (zero between
                               // launches; the launch that ends last zeroes them), or NULL: tiles by a
                               // fixed stride
    int *err;                  // device error word: a TMA wait that ran out sets bit 1
    Tw64 tw;
};

// PRISM probe scan (coefficients, window gather, beam sum, window FFT, |.|^2, bins).
struct ScanArgs {
    const float2 *S;           // [B][ny_s][nx_s]
    const double *x0;          // [P]
    const double *y0;          // [P]
    const double *qx;          // [B] beam qx = m f / cell_x
    const double *qy;          // [B]
    const float2 *base;        // [B] A(q_b) exp(-i chi(q_b))
    const float2 *tw_fwd;      // window FFT inter-stage twiddles (rows, length nw_x)
    const float2 *tw_fwd_y;    // window FFT inter-stage twiddles (columns, length nw_y)
    const float2 *tw_inv;      // (unused by the forward-only window FFT; kept for symmetry)
    const int *bin_off;        // [nbins+1] CSR offsets into bin_idx
    const int *bin_idx;        // window pixel indices (ky*nw + kx) grouped by bin
    const int *bin_idx_t;      // the same lists by rank: entry i of bin k at [i * nbins + k] (rows of
                               // the longest bin; bin k's list ends at bin_off[k+1] - bin_off[k])
    const uint16_t *bin_idx16; // bin_idx as 16-bit entries, 16-byte aligned and padded to 16 bytes (the
                               // copy a scan stages in shared memory where it fits), or NULL
    int n_bin_idx;             // entries of bin_idx (bin_off[nbins])
    float *out;                // [P][nbins] annular bins, or NULL
    float *cbed;               // [P][nw][nw] full window diffraction patterns (FFT order), or NULL
    float acc_w;               // accumulate: out += acc_w * I (else out = I)
    int accumulate;
    double px_s, py_s;         // stored pixel size
    double shift_x, shift_y;   // h tan(theta): the coefficients use r0 - shift (probe tilt)
    double inv_norm;           // 1 / (nw^4 * sum_b A_b)
    int n_beams;
    int nx_s, ny_s;
    int nbins;
    int n_probes;
    int probe0;
    // 16-bit mode (tensor-core beam sum)
    const void *S16;           // [ny_s * nx_s][kp] 16-bit (re, im) of each beam, zero-padded beams
                               // (split mode: [ny_s * nx_s][2][kp], value row then remainder row)
    const float *beam_scale;   // [B] power of two: S_b = S16_b * beam_scale[b]
    float2 *win;               // window scratch [slots][probes per group][nw][nw]
    int *win_cnt;              // [gridDim.x] parts finished per split block, then the next work unit and
                               // the CTAs done (all zero between launches)
    int *err;                  // device error word (a bounded wait that ran out sets bit 0)
    int kp;                    // K = 2 * roundup(B, 8)
    int scan_px, scan_py;      // probe raster, probe index = row * scan_px + col
    Tw64 tw;
};

// FP32 S of one beam batch -> per-beam scale and pixel-major 16-bit S
struct QuantArgs {
    const float2 *S;           // [nb][npix]
    void *S16;                 // [npix][kp]
    float *scale;              // [B]
    int beam0, nb, npix, kp;
    int mode;                  // 0: FP16, 1: BF16, 2: FP16 value + FP16 remainder (two rows of kp)
};

struct ShiftArgs {
    const double *x0, *y0;     // [batch]
    float2 *shift_x;           // [batch][nx]
    float2 *shift_y;           // [batch][ny]
    int nx, ny, batch;
    double cell_x, cell_y;
};

struct BinArgs {
    const float *inten;        // [batch][npix]
    const int *bin_off;        // [nbins+1]
    const int *bin_idx;
    float *out;                // [batch][nbins]
    double scale;
    int npix, nbins, batch;
    const int *err;            // optional device error word of the passes: non-zero -> the bins are NaN
};

// launchers (kernels_build.cu, kernels_scan.cu); return cudaSuccess or the launch error
cudaError_t launch_transmission(const float *V, float2 *t, size_t n, double sigma_cycles, cudaStream_t s);
// first-slice rows of beams beam0 .. beam0+nb-1 from T0 = FFT_x(t_0) [ny][nx] (kept columns only)
cudaError_t launch_plane(const float2 *T0, float2 *wave, const int *beam_mn, int beam0, int nb, int nx, int ny, int f, int f_y,
                         int kx_half, cudaStream_t s);
cudaError_t launch_row(int nx, RowMode mode, const RowArgs &a, cudaStream_t s);
cudaError_t launch_col(int ny, ColMode mode, const ColArgs &a, cudaStream_t s);
// the column transform of length ny: threads (lanes) per column and registers per thread, whose
// result row is lane + lanes * register (false for an unsupported ny)
bool col_fft_geometry(int ny, int *lanes, int *regs);
cudaError_t launch_scan(int nw, const ScanArgs &a, cudaStream_t s);
// nw_x x nw_y windows (separate f_x, f_y): square ones as launch_scan, rectangular ones (16, 32, 64
// per side) through the grouped kernel; scan_rect_supported says whether a launch can succeed
cudaError_t launch_scan_rect(int nwx, int nwy, const ScanArgs &a, cudaStream_t s);
bool scan_rect_supported(int nwx, int nwy, int n_beams);
// FP32 GEMM scan over raster blocks of 32 probes (window sides 16, 32, 64) in one of the
// contraction tile shapes (0 = default 4 x 8 blocks; the others for square windows): persistent
// grid (0 if it does not fit), launch, and the window scratch it needs
int scan_gemm_grid(int nwx, int nwy, int shape, int n_beams, int scan_px, int scan_py);
cudaError_t launch_scan_gemm(int nwx, int nwy, int shape, int grid, const ScanArgs &a, cudaStream_t s);
// window scratch of the FP32 GEMM scan: one slot per CTA plus one per split group of the last round
size_t scan_gemm_win_bytes(int nwx, int nwy, int shape, int grid, int scan_px, int scan_py);
// the contraction shapes: count, whether one is compiled for a window, its name; the tuned unit
int scan_gemm_shapes();
bool scan_gemm_shape_valid(int nwx, int nwy, int shape);
const char *scan_gemm_shape_name(int shape);
int scan_gemm_grid_tuned(int nwx, int nwy, int shape, int n_beams, int scan_px, int scan_py);
cudaError_t launch_scan_gemm_tuned(int nwx, int nwy, int shape, int grid, const ScanArgs &a, cudaStream_t s);
// scan counters: completion counters of the split groups (int[grid]), the next work unit and the
// CTAs done (int[2]); zeroed once, each launch leaves them zero
size_t scan_gemm_cnt_bytes(int grid);
cudaError_t launch_shift(const ShiftArgs &a, cudaStream_t s);
cudaError_t launch_bins(const BinArgs &a, cudaStream_t s);
cudaError_t launch_tc_selftest(float *out, int *status, cudaStream_t s);
cudaError_t launch_wait_selftest(int *status, long long limit_cycles, int arrive, cudaStream_t s);
// 16-bit mode (kernels_tc.cu)
cudaError_t launch_quantize(const QuantArgs &a, cudaStream_t s);
cudaError_t launch_dequantize(const void *S16, const float *scale, float2 *out, int n_beams, int npix, int kp,
                              int mode, cudaStream_t s);
cudaError_t launch_scan_tc(int nw, int mode, int shape, int grid, const ScanArgs &a, cudaStream_t s);
bool scan_tc_supported(int nw);
// persistent grid of the tensor-core scan (resident CTAs, at most the probe groups), 0 if it does
// not fit; window scratch bytes for that grid
int scan_tc_grid(int nw, int kp, int mode, int shape, int scan_px, int scan_py);
// ring shapes of the tensor-core scan's A operand (scan_tc.cuh): count for a mode, name; the
// non-default shapes (kernels_tc_tune.cu)
int scan_tc_shapes(int mode);
const char *scan_tc_shape_name(int shape);
int scan_tc_grid_tuned(int nw, int kp, int mode, int shape, int scan_px, int scan_py);
cudaError_t launch_scan_tc_tuned(int nw, int mode, int shape, int grid, const ScanArgs &a, cudaStream_t s);
// window scratch of the tensor-core scan: one slot per CTA plus one per split block of the last round
size_t scan_tc_win_bytes(int nw, int grid, int scan_px, int scan_py);
// autotuner launch shapes of ROW_STD (kind 0) and COL_STD (kind 1), N = 256 ... 2048 (kernels_tune.cu)
int tune_shapes(int kind);
const char *tune_shape_name(int kind, int v);
int tune_default_shape(int kind, int n);
bool tune_shape_valid(int kind, int n, int v);
bool tune_shape_needs_map(int kind, int v);  // the shape stages through TMA (ColArgs::wave_map)
int tune_shape_fft_variant(int kind, int v);  // its FFT radix variant (DftSplit), -1 if unknown
int tune_default_fft_variant(int n);          // the radix variant of the default launchers at N
int tune_col_tma_shape(int w);                // the TMA-staged column shape of w columns per CTA, or -1
int tune_row_find(int thr, bool stg, bool tma);  // the row shape of thr threads per CTA and that staging, or -1
bool tune_shape_fills_sm(int kind, int v);    // 3 or more CTAs per SM, each with a third of its resources
cudaError_t launch_row_shape(int nx, int v, const RowArgs &a, cudaStream_t s);
// the standard row pass of a multislice scan: at nx = 1024 the 384-thread shape with the next row's
// kept quarters staged by bulk TMA copies (the fastest there), elsewhere the default launcher; every
// shape computes the same rows
cudaError_t launch_row_std(int nx, const RowArgs &a, cudaStream_t s);
cudaError_t launch_col_shape(int ny, int v, const ColArgs &a, cudaStream_t s);
// smallest scan-window / FFT sizes the kernels are instantiated for
bool row_supported(int n);
bool col_supported(int n);
bool scan_supported(int nw);
// FFT split used by the kernels for length n: forward (n1, n2)
void fft_split(int n, int *n1, int *n2);

}  // namespace prism
