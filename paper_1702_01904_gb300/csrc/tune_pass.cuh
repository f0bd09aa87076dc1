// tune_pass.cuh -- the autotuner's shapes of the two multislice passes (tune_shapes.cuh) as kernel
// instantiations for one N: validity (compile-time, from the launch configuration alone) and the
// launch of shape v.  Each kernels_tune_<N>.cu unit instantiates one N (from N = 512 on, the row and
// the column shapes in units of their own, kernels_tune_<N>_row.cu and _col.cu), so that the units
// compile in parallel; kernels_tune.cu holds the tables and dispatches on N.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "fft.cuh"
#include "params.h"
#include "pass_kernels.cuh"
#include "tune_shapes.cuh"

namespace prism {
namespace tune {

template <int N, int I>
constexpr bool row_ok() {
    using C = RowCfg<N, ROW_SHAPES[I].a, ROW_SHAPES[I].stg, ROW_SHAPES[I].tma>;
    return C::SMEM <= 227 * 1024 && ROW_SHAPES[I].a % C::T == 0 && ROW_SHAPES[I].a <= 1024 && (!C::TMA || C::T == 32) &&
           (ROW_SHAPES[I].rv == 0 || N >= 512);
}

template <int N, int I>
constexpr bool col_ok() {
    using C = ColCfg<N, COL_SHAPES[I].a, COL_SHAPES[I].stg, COL_SHAPES[I].mb, COL_SHAPES[I].tma>;
    return C::SMEM <= 227 * 1024 && C::THREADS <= 1024 && (size_t)C::MINB * (C::SMEM + 1024) <= 228 * 1024 &&
           (!C::TMA || ((C::W == 4 || C::W == 8) && N % C::BOXR == 0)) && (COL_SHAPES[I].rv == 0 || N >= 512);
}

template <int N, int... I>
bool row_valid(int v, std::integer_sequence<int, I...>) {
    constexpr bool ok[N_ROW] = {row_ok<N, I>()...};
    return v >= 0 && v < N_ROW && ok[v];
}
template <int N, int... I>
bool col_valid(int v, std::integer_sequence<int, I...>) {
    constexpr bool ok[N_COL] = {col_ok<N, I>()...};
    return v >= 0 && v < N_COL && ok[v];
}
using RowSeq = std::make_integer_sequence<int, N_ROW>;
using ColSeq = std::make_integer_sequence<int, N_COL>;

template <int N, int I>
cudaError_t row_shape(const RowArgs &a, cudaStream_t s) {
    if (a.n_rows <= 0) return cudaSuccess;
    if constexpr (!row_ok<N, I>()) {
        return cudaErrorInvalidValue;
    } else {
        return row_go<N, ROW_STD, ROW_SHAPES[I].a, ROW_SHAPES[I].stg, ROW_SHAPES[I].tma, ROW_SHAPES[I].rv>(a, s);
    }
}
template <int N, int I>
cudaError_t col_shape(const ColArgs &a, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    if constexpr (!col_ok<N, I>()) {
        return cudaErrorInvalidValue;
    } else {
        return col_go<N, COL_STD, COL_SHAPES[I].a, COL_SHAPES[I].stg, COL_SHAPES[I].mb, COL_SHAPES[I].tma, COL_SHAPES[I].rv>(a, s);
    }
}

template <int N, int... I>
cudaError_t row_launch(int v, const RowArgs &a, cudaStream_t s, std::integer_sequence<int, I...>) {
    cudaError_t e = cudaErrorInvalidValue;
    ((v == I ? (e = row_shape<N, I>(a, s), true) : false) || ...);
    return e;
}
template <int N, int... I>
cudaError_t col_launch(int v, const ColArgs &a, cudaStream_t s, std::integer_sequence<int, I...>) {
    cudaError_t e = cudaErrorInvalidValue;
    ((v == I ? (e = col_shape<N, I>(a, s), true) : false) || ...);
    return e;
}

// launchers of every row and column shape for one N (defined by the kernels_tune_<N>.cu units)
cudaError_t row_launch_n256(int v, const RowArgs &a, cudaStream_t s);
cudaError_t row_launch_n512(int v, const RowArgs &a, cudaStream_t s);
cudaError_t row_launch_n1024(int v, const RowArgs &a, cudaStream_t s);
cudaError_t row_launch_n2048(int v, const RowArgs &a, cudaStream_t s);
cudaError_t col_launch_n256(int v, const ColArgs &a, cudaStream_t s);
cudaError_t col_launch_n512(int v, const ColArgs &a, cudaStream_t s);
cudaError_t col_launch_n1024(int v, const ColArgs &a, cudaStream_t s);
cudaError_t col_launch_n2048(int v, const ColArgs &a, cudaStream_t s);

}  // namespace tune
}  // namespace prism

// bodies of the kernels_tune_<N>*.cu units: the row shapes, the column shapes, or both of one N
#define PRISM_TUNE_ROW_UNIT(N)                                                                             \
    namespace prism {                                                                                      \
    namespace tune {                                                                                       \
    cudaError_t row_launch_n##N(int v, const RowArgs &a, cudaStream_t s) { return row_launch<N>(v, a, s, RowSeq{}); } \
    }                                                                                                      \
    }
#define PRISM_TUNE_COL_UNIT(N)                                                                             \
    namespace prism {                                                                                      \
    namespace tune {                                                                                       \
    cudaError_t col_launch_n##N(int v, const ColArgs &a, cudaStream_t s) { return col_launch<N>(v, a, s, ColSeq{}); } \
    }                                                                                                      \
    }
#define PRISM_TUNE_UNIT(N) PRISM_TUNE_ROW_UNIT(N) PRISM_TUNE_COL_UNIT(N)
