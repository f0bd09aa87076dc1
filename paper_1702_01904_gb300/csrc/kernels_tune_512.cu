// kernels_tune_512.cu -- every row- and column-pass shape of the autotuner for N = 512 (tune_pass.cuh).
#include "tune_pass.cuh"

PRISM_TUNE_UNIT(512)
