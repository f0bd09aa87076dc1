// tune_shapes.cuh -- launch shapes of the row and column passes that the autotuner times
// (kernels_tune.cu: column shapes and the tables; kernels_tune_row.cu: row shapes).
#pragma once

namespace prism {
namespace tune {

struct Shape {
    int a;      // row pass: threads per CTA; column pass: interleaved columns per CTA
    bool stg;   // cp.async staging of the next row / tile
    int mb;     // column pass: CTAs per SM the registers must allow (0: default rule)
    bool tma;   // the next tile (column pass, needs the plan's tensor map of the wave) or row (row
                // pass, bulk copies of its kept quarters) staged by TMA
};
constexpr Shape ROW_SHAPES[] = {{128, false, 0, false}, {256, false, 0, false}, {128, true, 0, false}, {256, true, 0, false},
                                {128, false, 0, true},  {256, false, 0, true},  {384, true, 0, false}, {384, false, 0, true}};
constexpr Shape COL_SHAPES[] = {{4, true, 0, false},  {8, true, 0, false},  {16, true, 0, false}, {4, false, 3, true},
                                {8, false, 0, false}, {8, false, 0, true},  {8, false, 2, false}, {4, true, 3, false}};
constexpr int N_ROW = sizeof(ROW_SHAPES) / sizeof(Shape);
constexpr int N_COL = sizeof(COL_SHAPES) / sizeof(Shape);

}  // namespace tune

// row shapes (kernels_tune_row.cu)
bool tune_row_valid(int n, int v);
cudaError_t tune_row_launch(int nx, int v, const RowArgs &a, cudaStream_t s);

}  // namespace prism
