// internal.h -- host helpers shared between the engine and the fixed-scratch multislice entry point.
#pragma once
#include <stddef.h>

#include <vector>

#include "params.h"
#include "prism.h"

namespace prism {

// Host tables of one multislice scan: everything the kernels read besides V, as host vectors.
struct MsHostTables {
    int nx = 0, ny = 0, H = 0;
    double lam = 0, sigma = 0, count = 0;
    std::vector<int> slice_prop;
    std::vector<float2> prop_x, prop_y, twr_f, twr_i, twc_f, twc_i, pbase;
    std::vector<int> aa_kmax, bin_off, bin_idx;
    std::vector<double> pos;  // x0[P] then y0[P]
    int kx_half = 0;          // row/column passes: kept columns |kx| < kx_half (0: all), as multislice_scan_run
    int band4 = 0;            // column passes: the aperture keeps |ky| < ny/4 on every column
    Tw64 tw;
};

// Validate the arguments of a multislice scan and build its host tables (same checks and FP64
// decisions as multislice_scan_run).  Returns a PRISM status; fills the thread-local error on failure.
int internal_multislice_tables(const prism_grid *grid, const prism_probe *probe, const prism_scan *scan,
                               const prism_detector *det, MsHostTables *out);
// Device-pointer validation as used by the entry points (NULL, alignment, memory type, device).
int internal_check_dev_ptr(const void *p, size_t align, const char *what);
// Record a failure in the thread-local error string and return `code`.
int internal_fail(int code, const char *msg);

}  // namespace prism
