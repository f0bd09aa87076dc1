// kernels_tune_2048_row.cu -- every row-pass shape of the autotuner for N = 2048 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_ROW_UNIT(2048)
