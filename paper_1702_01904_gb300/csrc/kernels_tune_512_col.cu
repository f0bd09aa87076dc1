// kernels_tune_512_col.cu -- every column-pass shape of the autotuner for N = 512 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_COL_UNIT(512)
