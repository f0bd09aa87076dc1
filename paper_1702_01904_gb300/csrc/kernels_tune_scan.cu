// kernels_tune_scan.cu -- the alternative contraction tile shapes of the FP32 GEMM scan (raster blocks
// 8 x 4 and 2 x 16 besides the default 4 x 8; rings of 3 stages of 16 beams besides 2 of 32) for
// square windows of 16, 32 and 64 pixels, which the scan autotuner times.  A separate unit so that
// it compiles in parallel with kernels_scan.cu.  Every shape accumulates each window pixel over the
// beams in the same order: the windows, and so the detector stacks, are bitwise the same.
#include <cuda_runtime.h>

#include "params.h"
#include "scan_gemm.cuh"

namespace prism {

namespace {

const char *GEMM_NAMES[N_GEMM_SHAPES] = {"4x8 blocks, 2 x 33 beams", "8x4 blocks, 2 x 32 beams", "2x16 blocks, 2 x 32 beams",
                                         "4x8 blocks, 3 x 16 beams", "8x4 blocks, 3 x 16 beams", "4x8 blocks, 2 x 32 beams"};

template <int NW>
int grid_nw(int shape, int n_beams, int px, int py) {
    switch (shape) {
        case 1: return gemm_grid<NW, NW, 1>(n_beams, px, py);
        case 2: return gemm_grid<NW, NW, 2>(n_beams, px, py);
        case 3: return gemm_grid<NW, NW, 3>(n_beams, px, py);
        case 4: return gemm_grid<NW, NW, 4>(n_beams, px, py);
        case 5: return gemm_grid<NW, NW, 5>(n_beams, px, py);
    }
    return 0;
}

template <int NW>
cudaError_t launch_nw(int shape, int grid, const ScanArgs &a, cudaStream_t s) {
    switch (shape) {
        case 1: return gemm_launch<NW, NW, 1>(grid, a, s);
        case 2: return gemm_launch<NW, NW, 2>(grid, a, s);
        case 3: return gemm_launch<NW, NW, 3>(grid, a, s);
        case 4: return gemm_launch<NW, NW, 4>(grid, a, s);
        case 5: return gemm_launch<NW, NW, 5>(grid, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool scan_gemm_shape_valid(int nwx, int nwy, int shape) {
    if (shape == 0) return true;
    return shape > 0 && shape < N_GEMM_SHAPES && nwx == nwy && (nwx == 16 || nwx == 32 || nwx == 64);
}

const char *scan_gemm_shape_name(int shape) { return shape >= 0 && shape < N_GEMM_SHAPES ? GEMM_NAMES[shape] : "?"; }

int scan_gemm_grid_tuned(int nwx, int nwy, int shape, int n_beams, int scan_px, int scan_py) {
    if (!scan_gemm_shape_valid(nwx, nwy, shape)) return 0;
    switch (nwx) {
        case 16: return grid_nw<16>(shape, n_beams, scan_px, scan_py);
        case 32: return grid_nw<32>(shape, n_beams, scan_px, scan_py);
        case 64: return grid_nw<64>(shape, n_beams, scan_px, scan_py);
    }
    return 0;
}

cudaError_t launch_scan_gemm_tuned(int nwx, int nwy, int shape, int grid, const ScanArgs &a, cudaStream_t s) {
    if (!scan_gemm_shape_valid(nwx, nwy, shape)) return cudaErrorInvalidValue;
    switch (nwx) {
        case 16: return launch_nw<16>(shape, grid, a, s);
        case 32: return launch_nw<32>(shape, grid, a, s);
        case 64: return launch_nw<64>(shape, grid, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace prism
