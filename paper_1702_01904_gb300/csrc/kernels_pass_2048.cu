// kernels_pass_2048.cu -- the row and column passes at their default launch shapes for N = 2048
// (pass_default.cuh).
#include "pass_default.cuh"

PRISM_PASS_UNIT(2048)
