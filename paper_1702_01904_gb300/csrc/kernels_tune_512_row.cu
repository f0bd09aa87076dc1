// kernels_tune_512_row.cu -- every row-pass shape of the autotuner for N = 512 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_ROW_UNIT(512)
