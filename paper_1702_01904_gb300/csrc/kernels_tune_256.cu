// kernels_tune_256.cu -- every row- and column-pass shape of the autotuner for N = 256 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_UNIT(256)
