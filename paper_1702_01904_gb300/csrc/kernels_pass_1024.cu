// kernels_pass_1024.cu -- the row and column passes at their default launch shapes for N = 1024
// (pass_default.cuh).
#include "pass_default.cuh"

PRISM_PASS_UNIT(1024)
