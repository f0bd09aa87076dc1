// kernels_tune.cu -- the autotuner's launch shapes of the two multislice passes (ROW_STD and
// COL_STD, N = 256 ... 2048): names, lookups and the dispatch on N to the kernels_tune_<N>.cu units,
// which instantiate the shapes (tune_pass.cuh).  A shape changes only how rows or columns are spread
// over threads, whether the next row/tile is staged through shared memory (with cp.async, by bulk or
// tiled TMA copies completing on an mbarrier), and the FFT radix: the split of the 32- and 64-point
// register DFTs (DftSplit) of the pass's forward and inverse transform.  Shapes of one radix variant
// compute bitwise the same transform; the variants round differently.
#include <cuda_runtime.h>

#include "params.h"
#include "tune_pass.cuh"

namespace prism {

namespace {

using tune::COL_SHAPES;
using tune::N_COL;
using tune::N_ROW;
using tune::ROW_SHAPES;
const char *ROW_NAMES[N_ROW] = {"128 thr",
                                "256 thr",
                                "128 thr, staged",
                                "256 thr, staged",
                                "128 thr, TMA",
                                "256 thr, TMA",
                                "384 thr, staged",
                                "384 thr, TMA",
                                "384 thr, TMA, radix-4 first: forward",
                                "384 thr, TMA, radix-4 first: inverse",
                                "384 thr, TMA, radix-4 first: both",
                                "128 thr, radix-4 first: both",
                                "128 thr, staged, radix-4 first: both"};
const char *COL_NAMES[N_COL] = {"W4, staged",
                                "W8, staged",
                                "W16, staged",
                                "W4, TMA, 3/SM",
                                "W8",
                                "W8, TMA",
                                "W8, 2/SM",
                                "W4, staged, 3/SM",
                                "W4, TMA, 3/SM, radix-4 first: forward",
                                "W4, TMA, 3/SM, radix-4 first: inverse",
                                "W4, TMA, 3/SM, radix-4 first: both",
                                "W8, staged, radix-4 first: both",
                                "W8, radix-4 first: both",
                                "W4, staged, radix-4 first: both"};
static_assert(sizeof(ROW_NAMES) / sizeof(ROW_NAMES[0]) == N_ROW && sizeof(COL_NAMES) / sizeof(COL_NAMES[0]) == N_COL, "one name per shape");

}  // namespace

int tune_shapes(int kind) { return kind == 0 ? N_ROW : kind == 1 ? N_COL : 0; }

const char *tune_shape_name(int kind, int v) {
    if (kind == 0 && v >= 0 && v < N_ROW) return ROW_NAMES[v];
    if (kind == 1 && v >= 0 && v < N_COL) return COL_NAMES[v];
    return "?";
}

int tune_default_shape(int kind, int n) {
    const int rv = default_fft_variant(n);
    if (kind == 0) {
        const int thr = n >= 512 ? 128 : 256;  // row_default_threads, unstaged
        for (int v = 0; v < N_ROW; ++v)
            if (ROW_SHAPES[v].a == thr && !ROW_SHAPES[v].stg && !ROW_SHAPES[v].tma && ROW_SHAPES[v].rv == rv) return v;
    } else if (kind == 1) {
        const int w = n >= 1024 ? 8 : 16;  // col_default_w
        const bool stg = n < 2048;         // col_default_stg
        for (int v = 0; v < N_COL; ++v)
            if (COL_SHAPES[v].a == w && COL_SHAPES[v].stg == stg && COL_SHAPES[v].mb == 0 && !COL_SHAPES[v].tma &&
                COL_SHAPES[v].rv == rv)
                return v;
    }
    return -1;
}

int tune_default_fft_variant(int n) { return default_fft_variant(n); }

int tune_shape_fft_variant(int kind, int v) {
    if (kind == 0 && v >= 0 && v < N_ROW) return ROW_SHAPES[v].rv;
    if (kind == 1 && v >= 0 && v < N_COL) return COL_SHAPES[v].rv;
    return -1;
}

bool tune_shape_needs_map(int kind, int v) { return kind == 1 && v >= 0 && v < N_COL && COL_SHAPES[v].tma; }

bool tune_shape_fills_sm(int kind, int v) { return kind == 1 && v >= 0 && v < N_COL && COL_SHAPES[v].mb >= 3; }

int tune_row_find(int thr, bool stg, bool tma) {
    for (int v = 0; v < N_ROW; ++v)
        if (ROW_SHAPES[v].a == thr && ROW_SHAPES[v].stg == stg && ROW_SHAPES[v].tma == tma && ROW_SHAPES[v].rv == 0) return v;
    return -1;
}

cudaError_t launch_row_std(int nx, const RowArgs &a, cudaStream_t s) {
    if (nx == 1024) {
        const int v = tune_row_find(384, false, true);
        if (v >= 0 && tune_row_valid(1024, v)) return tune_row_launch(1024, v, a, s);
    }
    return launch_row(nx, ROW_STD, a, s);
}

int tune_col_tma_shape(int w) {
    for (int v = 0; v < N_COL; ++v)
        if (COL_SHAPES[v].tma && COL_SHAPES[v].a == w && COL_SHAPES[v].rv == 0) return v;
    return -1;
}

bool tune_row_valid(int n, int v) {
    switch (n) {
        case 256: return tune::row_valid<256>(v, tune::RowSeq{});
        case 512: return tune::row_valid<512>(v, tune::RowSeq{});
        case 1024: return tune::row_valid<1024>(v, tune::RowSeq{});
        case 2048: return tune::row_valid<2048>(v, tune::RowSeq{});
    }
    return false;
}

cudaError_t tune_row_launch(int nx, int v, const RowArgs &a, cudaStream_t s) {
    switch (nx) {
        case 256: return tune::row_launch_n256(v, a, s);
        case 512: return tune::row_launch_n512(v, a, s);
        case 1024: return tune::row_launch_n1024(v, a, s);
        case 2048: return tune::row_launch_n2048(v, a, s);
    }
    return cudaErrorInvalidValue;
}

bool tune_shape_valid(int kind, int n, int v) {
    if (kind == 0) {
        return tune_row_valid(n, v);
    } else if (kind == 1) {
        switch (n) {
            case 256: return tune::col_valid<256>(v, tune::ColSeq{});
            case 512: return tune::col_valid<512>(v, tune::ColSeq{});
            case 1024: return tune::col_valid<1024>(v, tune::ColSeq{});
            case 2048: return tune::col_valid<2048>(v, tune::ColSeq{});
        }
    }
    return false;
}

cudaError_t launch_row_shape(int nx, int v, const RowArgs &a, cudaStream_t s) {
    if (!tune_shape_valid(0, nx, v)) return cudaErrorInvalidValue;
    return tune_row_launch(nx, v, a, s);
}

cudaError_t launch_col_shape(int ny, int v, const ColArgs &a, cudaStream_t s) {
    if (!tune_shape_valid(1, ny, v)) return cudaErrorInvalidValue;
    switch (ny) {
        case 256: return tune::col_launch_n256(v, a, s);
        case 512: return tune::col_launch_n512(v, a, s);
        case 1024: return tune::col_launch_n1024(v, a, s);
        case 2048: return tune::col_launch_n2048(v, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace prism
