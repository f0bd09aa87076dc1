// kernels_tune_1024_row.cu -- every row-pass shape of the autotuner for N = 1024 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_ROW_UNIT(1024)
