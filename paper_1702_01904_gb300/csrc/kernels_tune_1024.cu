// kernels_tune_1024.cu -- every row- and column-pass shape of the autotuner for N = 1024 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_UNIT(1024)
