// kernels_tune_2048.cu -- every row- and column-pass shape of the autotuner for N = 2048 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_UNIT(2048)
