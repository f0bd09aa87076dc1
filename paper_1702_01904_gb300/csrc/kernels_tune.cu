// kernels_tune.cu -- the alternative launch shapes of the two multislice passes that the autotuner
// times (ROW_STD and COL_STD, N = 256 ... 2048): the column shapes and the shape tables here, the
// row shapes in kernels_tune_row.cu (a separate unit so that both compile in parallel).  A shape
// changes only how rows or columns are spread over threads and whether the next row/tile is staged
// through shared memory (with cp.async, or for "W8, TMA" with tiled TMA loads completing on an
// mbarrier); every shape computes bitwise the same transform.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"
#include "pass_kernels.cuh"
#include "tune_shapes.cuh"

namespace prism {

namespace {

using tune::COL_SHAPES;
using tune::N_COL;
using tune::N_ROW;
using tune::ROW_SHAPES;
const char *ROW_NAMES[N_ROW] = {"128 thr", "256 thr", "128 thr, staged", "256 thr, staged", "128 thr, TMA",
                                "256 thr, TMA", "384 thr, staged", "384 thr, TMA"};
const char *COL_NAMES[N_COL] = {"W4, staged", "W8, staged", "W16, staged", "W4, TMA, 3/SM", "W8", "W8, TMA", "W8, 2/SM", "W4, staged, 3/SM"};

template <int N, int I>
constexpr bool col_ok() {
    using C = ColCfg<N, COL_SHAPES[I].a, COL_SHAPES[I].stg, COL_SHAPES[I].mb, COL_SHAPES[I].tma>;
    return C::SMEM <= 227 * 1024 && C::THREADS <= 1024 && (size_t)C::MINB * (C::SMEM + 1024) <= 228 * 1024 &&
           (!C::TMA || ((C::W == 4 || C::W == 8) && N % C::BOXR == 0));
}

template <int N, int I>
cudaError_t col_shape(const ColArgs &a, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    return col_go<N, COL_STD, COL_SHAPES[I].a, COL_SHAPES[I].stg, COL_SHAPES[I].mb, COL_SHAPES[I].tma>(a, s);
}

template <int N>
cudaError_t col_n(int v, const ColArgs &a, cudaStream_t s) {
    switch (v) {
        case 0: return col_shape<N, 0>(a, s);
        case 1: return col_shape<N, 1>(a, s);
        case 2: return col_shape<N, 2>(a, s);
        case 3: return col_shape<N, 3>(a, s);
        case 4: return col_shape<N, 4>(a, s);
        case 5: return col_shape<N, 5>(a, s);
        case 6: return col_shape<N, 6>(a, s);
        case 7: return col_shape<N, 7>(a, s);
    }
    return cudaErrorInvalidValue;
}
template <int N>
bool col_valid_n(int v) {
    constexpr bool ok[N_COL] = {col_ok<N, 0>(), col_ok<N, 1>(), col_ok<N, 2>(), col_ok<N, 3>(),
                                col_ok<N, 4>(), col_ok<N, 5>(), col_ok<N, 6>(), col_ok<N, 7>()};
    return v >= 0 && v < N_COL && ok[v];
}

}  // namespace

int tune_shapes(int kind) { return kind == 0 ? N_ROW : kind == 1 ? N_COL : 0; }

const char *tune_shape_name(int kind, int v) {
    if (kind == 0 && v >= 0 && v < N_ROW) return ROW_NAMES[v];
    if (kind == 1 && v >= 0 && v < N_COL) return COL_NAMES[v];
    return "?";
}

int tune_default_shape(int kind, int n) {
    if (kind == 0) {
        const int thr = n >= 512 ? 128 : 256;  // row_default_threads, unstaged
        for (int v = 0; v < N_ROW; ++v)
            if (ROW_SHAPES[v].a == thr && !ROW_SHAPES[v].stg && !ROW_SHAPES[v].tma) return v;
    } else if (kind == 1) {
        const int w = n >= 2048 ? 4 : n >= 1024 ? 8 : 16;  // col_default_w, staged
        for (int v = 0; v < N_COL; ++v)
            if (COL_SHAPES[v].a == w && COL_SHAPES[v].stg && COL_SHAPES[v].mb == 0 && !COL_SHAPES[v].tma) return v;
    }
    return -1;
}

bool tune_shape_needs_map(int kind, int v) { return kind == 1 && v >= 0 && v < N_COL && COL_SHAPES[v].tma; }

bool tune_shape_fills_sm(int kind, int v) { return kind == 1 && v >= 0 && v < N_COL && COL_SHAPES[v].mb >= 3; }

int tune_row_find(int thr, bool stg, bool tma) {
    for (int v = 0; v < N_ROW; ++v)
        if (ROW_SHAPES[v].a == thr && ROW_SHAPES[v].stg == stg && ROW_SHAPES[v].tma == tma) return v;
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
        if (COL_SHAPES[v].tma && COL_SHAPES[v].a == w) return v;
    return -1;
}

bool tune_shape_valid(int kind, int n, int v) {
    if (kind == 0) {
        return tune_row_valid(n, v);
    } else if (kind == 1) {
        switch (n) {
            case 256: return col_valid_n<256>(v);
            case 512: return col_valid_n<512>(v);
            case 1024: return col_valid_n<1024>(v);
            case 2048: return col_valid_n<2048>(v);
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
        case 256: return col_n<256>(v, a, s);
        case 512: return col_n<512>(v, a, s);
        case 1024: return col_n<1024>(v, a, s);
        case 2048: return col_n<2048>(v, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace prism
