// kernels_tc_tune.cu -- the tensor-core scan's ring shapes other than the default (scan_tc.cuh), which
// the scan autotuner times (FP16 and BF16; split mode has one shape).  A separate unit so that it
// compiles beside kernels_tc.cu.
#include "scan_tc.cuh"

namespace prism {

namespace {
template <int NW>
int grid_nw(int mode, int shape, int kp, int px, int py) {
    if (mode == TC_FP16) {
        if (shape == 1) return tc_grid<NW, TC_FP16, 1>(kp, px, py);
        if (shape == 2) return tc_grid<NW, TC_FP16, 2>(kp, px, py);
    } else if (mode == TC_BF16) {
        if (shape == 1) return tc_grid<NW, TC_BF16, 1>(kp, px, py);
        if (shape == 2) return tc_grid<NW, TC_BF16, 2>(kp, px, py);
    }
    return 0;
}
template <int NW>
cudaError_t launch_nw(int mode, int shape, int grid, const ScanArgs &a, cudaStream_t s) {
    if (mode == TC_FP16) {
        if (shape == 1) return tc_launch<NW, TC_FP16, 1>(grid, a, s);
        if (shape == 2) return tc_launch<NW, TC_FP16, 2>(grid, a, s);
    } else if (mode == TC_BF16) {
        if (shape == 1) return tc_launch<NW, TC_BF16, 1>(grid, a, s);
        if (shape == 2) return tc_launch<NW, TC_BF16, 2>(grid, a, s);
    }
    return cudaErrorInvalidValue;
}
static_assert(N_TC_SHAPES == 3, "one branch per shape above");
}  // namespace

int scan_tc_grid_tuned(int nw, int kp, int mode, int shape, int scan_px, int scan_py) {
    switch (nw) {
        case 16: return grid_nw<16>(mode, shape, kp, scan_px, scan_py);
        case 32: return grid_nw<32>(mode, shape, kp, scan_px, scan_py);
        case 64: return grid_nw<64>(mode, shape, kp, scan_px, scan_py);
    }
    return 0;
}

cudaError_t launch_scan_tc_tuned(int nw, int mode, int shape, int grid, const ScanArgs &a, cudaStream_t s) {
    switch (nw) {
        case 16: return launch_nw<16>(mode, shape, grid, a, s);
        case 32: return launch_nw<32>(mode, shape, grid, a, s);
        case 64: return launch_nw<64>(mode, shape, grid, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace prism
