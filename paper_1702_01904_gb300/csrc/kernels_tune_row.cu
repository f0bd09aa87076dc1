// kernels_tune_row.cu -- the row-pass launch shapes the autotuner times (N = 256 ... 2048); every
// shape computes bitwise the same transform.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"
#include "pass_kernels.cuh"
#include "tune_shapes.cuh"

namespace prism {

namespace {
using tune::N_ROW;
using tune::ROW_SHAPES;

template <int N, int I>
constexpr bool row_ok() {
    using C = RowCfg<N, ROW_SHAPES[I].a, ROW_SHAPES[I].stg, ROW_SHAPES[I].tma>;
    return C::SMEM <= 227 * 1024 && ROW_SHAPES[I].a % C::T == 0 && ROW_SHAPES[I].a <= 1024 && (!C::TMA || C::T == 32);
}

template <int N, int I>
cudaError_t row_shape(const RowArgs &a, cudaStream_t s) {
    if (a.n_rows <= 0) return cudaSuccess;
    return row_go<N, ROW_STD, ROW_SHAPES[I].a, ROW_SHAPES[I].stg, ROW_SHAPES[I].tma>(a, s);
}

template <int N>
cudaError_t row_n(int v, const RowArgs &a, cudaStream_t s) {
    switch (v) {
        case 0: return row_shape<N, 0>(a, s);
        case 1: return row_shape<N, 1>(a, s);
        case 2: return row_shape<N, 2>(a, s);
        case 3: return row_shape<N, 3>(a, s);
        case 4: return row_shape<N, 4>(a, s);
        case 5: return row_shape<N, 5>(a, s);
        case 6: return row_shape<N, 6>(a, s);
        case 7: return row_shape<N, 7>(a, s);
    }
    return cudaErrorInvalidValue;
}
template <int N>
bool row_valid_n(int v) {
    constexpr bool ok[N_ROW] = {row_ok<N, 0>(), row_ok<N, 1>(), row_ok<N, 2>(), row_ok<N, 3>(),
                                row_ok<N, 4>(), row_ok<N, 5>(), row_ok<N, 6>(), row_ok<N, 7>()};
    return v >= 0 && v < N_ROW && ok[v];
}
}  // namespace

bool tune_row_valid(int n, int v) {
    switch (n) {
        case 256: return row_valid_n<256>(v);
        case 512: return row_valid_n<512>(v);
        case 1024: return row_valid_n<1024>(v);
        case 2048: return row_valid_n<2048>(v);
    }
    return false;
}

cudaError_t tune_row_launch(int nx, int v, const RowArgs &a, cudaStream_t s) {
    switch (nx) {
        case 256: return row_n<256>(v, a, s);
        case 512: return row_n<512>(v, a, s);
        case 1024: return row_n<1024>(v, a, s);
        case 2048: return row_n<2048>(v, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace prism
