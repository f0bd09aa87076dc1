// kernels_tune_1024_col.cu -- every column-pass shape of the autotuner for N = 1024 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_COL_UNIT(1024)
