// pass_default.cuh -- the row and column passes at their default launch shapes (the launchers
// behind launch_row / launch_col): templates over N, instantiated for N <= 256 in kernels_build.cu
// and for the larger N in units of their own (kernels_pass_<N>.cu), so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"
#include "params.h"
#include "pass_kernels.cuh"

namespace prism {

template <int NX>
static cudaError_t row_dispatch(RowMode mode, const RowArgs &a, cudaStream_t s) {
    if (a.n_rows <= 0) return cudaSuccess;
    constexpr int T = row_default_threads<NX>(), RV = default_fft_variant(NX);
    switch (mode) {
        case ROW_STD: return row_go<NX, ROW_STD, T, false, false, RV>(a, s);
        case ROW_PLANE: return row_go<NX, ROW_PLANE, T, false, false, RV>(a, s);
        case ROW_OUT: return row_go<NX, ROW_OUT, T, false, false, RV>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <int NY>
static cudaError_t col_dispatch(ColMode mode, const ColArgs &a, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    constexpr int W = col_default_w<NY>(), RV = default_fft_variant(NY);
    constexpr bool STG = col_default_stg<NY>();
    switch (mode) {
        case COL_STD: return col_go<NY, COL_STD, W, STG, 0, false, RV>(a, s);
        case COL_PROBE: return col_go<NY, COL_PROBE, W, STG, 0, false, RV>(a, s);
        case COL_DETECT: return col_go<NY, COL_DETECT, W, STG, 0, false, RV>(a, s);
    }
    return cudaErrorInvalidValue;
}

// the launchers of one N, defined by its kernels_pass_<N>.cu unit
cudaError_t launch_row_n512(RowMode mode, const RowArgs &a, cudaStream_t s);
cudaError_t launch_row_n1024(RowMode mode, const RowArgs &a, cudaStream_t s);
cudaError_t launch_row_n2048(RowMode mode, const RowArgs &a, cudaStream_t s);
cudaError_t launch_col_n512(ColMode mode, const ColArgs &a, cudaStream_t s);
cudaError_t launch_col_n1024(ColMode mode, const ColArgs &a, cudaStream_t s);
cudaError_t launch_col_n2048(ColMode mode, const ColArgs &a, cudaStream_t s);

}  // namespace prism

// body of a kernels_pass_<N>.cu unit
#define PRISM_PASS_UNIT(N)                                                                                     \
    namespace prism {                                                                                          \
    cudaError_t launch_row_n##N(RowMode mode, const RowArgs &a, cudaStream_t s) { return row_dispatch<N>(mode, a, s); } \
    cudaError_t launch_col_n##N(ColMode mode, const ColArgs &a, cudaStream_t s) { return col_dispatch<N>(mode, a, s); } \
    }
