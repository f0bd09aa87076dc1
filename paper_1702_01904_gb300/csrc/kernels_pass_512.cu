// kernels_pass_512.cu -- the row and column passes at their default launch shapes for N = 512
// (pass_default.cuh).
#include "pass_default.cuh"

PRISM_PASS_UNIT(512)
