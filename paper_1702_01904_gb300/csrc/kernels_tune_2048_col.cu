// kernels_tune_2048_col.cu -- every column-pass shape of the autotuner for N = 2048 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_COL_UNIT(2048)
