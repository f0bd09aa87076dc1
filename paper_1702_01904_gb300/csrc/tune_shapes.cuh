// tune_shapes.cuh -- launch shapes of the row and column passes that the autotuner times
// (kernels_tune.cu: names, lookups, dispatch; tune_pass.cuh and kernels_tune_<N>.cu: the kernels).
#pragma once

namespace prism {
namespace tune {

struct Shape {
    int a;      // row pass: threads per CTA; column pass: interleaved columns per CTA
    bool stg;   // cp.async staging of the next row / tile
    int mb;     // column pass: CTAs per SM the registers must allow (0: default rule)
    bool tma;   // the next tile (column pass, needs the plan's tensor map of the wave) or row (row
                // pass, bulk copies of its kept quarters) staged by TMA
    int rv;     // FFT radix: split variants of the 32- and 64-point register DFTs (DftSplit) of the
                // forward (bit 0) and inverse (bit 1) transform; non-zero only for N >= 512, where
                // the transforms use those DFTs
};
constexpr Shape ROW_SHAPES[] = {{128, false, 0, false, 0}, {256, false, 0, false, 0}, {128, true, 0, false, 0},
                                {256, true, 0, false, 0},  {128, false, 0, true, 0},  {256, false, 0, true, 0},
                                {384, true, 0, false, 0},  {384, false, 0, true, 0},  {384, false, 0, true, 1},
                                {384, false, 0, true, 2},  {384, false, 0, true, 3},  {128, false, 0, false, 3},
                                {128, true, 0, false, 3}};
constexpr Shape COL_SHAPES[] = {{4, true, 0, false, 0},  {8, true, 0, false, 0}, {16, true, 0, false, 0}, {4, false, 3, true, 0},
                                {8, false, 0, false, 0}, {8, false, 0, true, 0}, {8, false, 2, false, 0}, {4, true, 3, false, 0},
                                {4, false, 3, true, 1},  {4, false, 3, true, 2}, {4, false, 3, true, 3},  {8, true, 0, false, 3},
                                {8, false, 0, false, 3}, {4, true, 0, false, 3}};
constexpr int N_ROW = sizeof(ROW_SHAPES) / sizeof(Shape);
constexpr int N_COL = sizeof(COL_SHAPES) / sizeof(Shape);

}  // namespace tune

// row shapes (kernels_tune.cu)
bool tune_row_valid(int n, int v);
cudaError_t tune_row_launch(int nx, int v, const RowArgs &a, cudaStream_t s);

}  // namespace prism
