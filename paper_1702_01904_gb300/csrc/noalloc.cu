// noalloc.cu -- multislice STEM scan that allocates no device memory.
//
// Some callers cannot allocate device memory themselves: a host application that hands out the
// whole device-memory budget through its own pool and forbids other allocators, or a
// latency-critical loop in which cudaMalloc / cudaFree (which may synchronise the device) are not
// allowed.  multislice_scan_run_noalloc serves them: it computes exactly what multislice_scan_run
// computes, with the same kernels, but every buffer it needs besides the caller's input and output
// lives in one fixed, file-scope device array of PRISM_NOALLOC_SCRATCH_BYTES.  Every GPU that
// loads this library holds that array until the process exits.
//
// Host code must not take the array's symbol as a device address (on the host it is only a
// stand-in), so the device address is looked up once per device with cudaGetSymbolAddress, with
// that device current, on the first call made on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "params.h"
#include "prism.h"

using namespace prism;

static __device__ __align__(256) unsigned char g_noalloc_scratch[PRISM_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
std::vector<void *> g_scratch_ptr;  // device address of g_noalloc_scratch, per device ordinal

// Device address of the scratch array on the current device (looked up on first use).
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return internal_fail(PRISM_ERR_CUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if ((int)g_scratch_ptr.size() <= dev) g_scratch_ptr.resize(dev + 1, nullptr);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return internal_fail(PRISM_ERR_CUDA, (std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)).c_str());
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PRISM_OK;
}

// Sub-allocation of the fixed array: 256-byte aligned segments, bump pointer.
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t count) {
        used = (used + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + used);
        used += count * sizeof(T);
        return p;
    }
    static size_t need(size_t bytes) { return ((bytes + 255) & ~(size_t)255); }
};

template <class T>
int put(T *dst, const std::vector<T> &src, cudaStream_t st) {
    if (src.empty()) return PRISM_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return internal_fail(PRISM_ERR_CUDA, (std::string("table upload: ") + cudaGetErrorString(e)).c_str());
    return PRISM_OK;
}

}  // namespace

extern "C" int multislice_scan_run_noalloc(const prism_grid *grid, const float *V_dev, const prism_probe *probe,
                                           const prism_scan *scan, const prism_detector *det, float *out_dev,
                                           void *cuda_stream) {
    MsHostTables M;
    int rc = internal_multislice_tables(grid, probe, scan, det, &M);
    if (rc) return rc;
    const long long Pn = (long long)scan->px * scan->py;
    if (Pn == 0) return PRISM_OK;
    if ((rc = internal_check_dev_ptr(V_dev, 16, "V_dev"))) return rc;
    if ((rc = internal_check_dev_ptr(out_dev, 4, "out_dev"))) return rc;
    const int nx = M.nx, ny = M.ny, H = M.H;
    const size_t px = (size_t)nx * ny;

    // sizes of the fixed segments and of one probe in flight
    const size_t fixed = Carve::need(H * px * 8) + Carve::need(px * 8) + Carve::need(M.prop_x.size() * 8) +
                         Carve::need(M.prop_y.size() * 8) + Carve::need(M.aa_kmax.size() * 4) + 2 * Carve::need(nx * 8) +
                         2 * Carve::need(ny * 8) + Carve::need(M.bin_off.size() * 4) + Carve::need(M.bin_idx.size() * 4) +
                         Carve::need(M.pos.size() * 8);
    const size_t per_probe = px * 8 + px * 4 + (size_t)(nx + ny) * 8;
    const size_t slack = 4 * 256;
    if (fixed + slack + per_probe > (size_t)PRISM_NOALLOC_SCRATCH_BYTES) {
        const std::string msg = "multislice_scan_run_noalloc: this grid needs " + std::to_string(fixed + slack + per_probe) +
                                " bytes of scratch, more than the fixed " + std::to_string((size_t)PRISM_NOALLOC_SCRATCH_BYTES) +
                                " (use multislice_scan_run)";
        return internal_fail(PRISM_ERR_BUDGET, msg.c_str());
    }
    const int Pb = (int)std::min<long long>(Pn, (long long)(((size_t)PRISM_NOALLOC_SCRATCH_BYTES - fixed - slack) / per_probe));

    void *sp = nullptr;
    if ((rc = scratch_address(&sp))) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Carve C{static_cast<unsigned char *>(sp)};
    float2 *t = C.take<float2>(H * px);
    float2 *pbase = C.take<float2>(px);
    float2 *prop_x = C.take<float2>(M.prop_x.size());
    float2 *prop_y = C.take<float2>(M.prop_y.size());
    int *aa = C.take<int>(M.aa_kmax.size());
    float2 *twr_f = C.take<float2>(nx), *twr_i = C.take<float2>(nx);
    float2 *twc_f = C.take<float2>(ny), *twc_i = C.take<float2>(ny);
    int *d_off = C.take<int>(M.bin_off.size());
    int *d_idx = C.take<int>(M.bin_idx.size());
    double *pos = C.take<double>(M.pos.size());
    float2 *wave = C.take<float2>((size_t)Pb * px);
    float *inten = C.take<float>((size_t)Pb * px);
    float2 *shx = C.take<float2>((size_t)Pb * nx);
    float2 *shy = C.take<float2>((size_t)Pb * ny);
    if (C.used > (size_t)PRISM_NOALLOC_SCRATCH_BYTES) return internal_fail(PRISM_ERR_BUDGET, "scratch layout overflow");

    // Every region below is fully written before it is read in this call, so nothing has to be
    // cleared; the previous call's contents are simply overwritten.
    if ((rc = put(pbase, M.pbase, st)) || (rc = put(prop_x, M.prop_x, st)) || (rc = put(prop_y, M.prop_y, st)) ||
        (rc = put(aa, M.aa_kmax, st)) || (rc = put(twr_f, M.twr_f, st)) || (rc = put(twr_i, M.twr_i, st)) ||
        (rc = put(twc_f, M.twc_f, st)) || (rc = put(twc_i, M.twc_i, st)) || (rc = put(d_off, M.bin_off, st)) ||
        (rc = put(d_idx, M.bin_idx, st)) || (rc = put(pos, M.pos, st)))
        return rc;

    auto check = [&](cudaError_t err, const char *what) {
        if (err != cudaSuccess) return internal_fail(PRISM_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(err)).c_str());
        return PRISM_OK;
    };
    if ((rc = check(launch_transmission(V_dev, t, (size_t)H * px, M.sigma / (2.0 * 3.141592653589793), st), "transmission")))
        return rc;
    for (long long p0 = 0; p0 < Pn; p0 += Pb) {
        const int nb = (int)std::min<long long>(Pb, Pn - p0);
        ShiftArgs sa;
        sa.x0 = pos + p0;
        sa.y0 = pos + Pn + p0;
        sa.shift_x = shx;
        sa.shift_y = shy;
        sa.nx = nx;
        sa.ny = ny;
        sa.batch = nb;
        sa.cell_x = grid->cell_x;
        sa.cell_y = grid->cell_y;
        if ((rc = check(launch_shift(sa, st), "shift phases"))) return rc;
        ColArgs ci;
        std::memset(&ci, 0, sizeof(ci));
        ci.wave = wave;
        ci.aa_kmax = aa;
        ci.tw_fwd = twc_f;
        ci.tw_inv = twc_i;
        ci.nx = nx;
        ci.tw = M.tw;
        ci.batch = nb;
        ci.probe_base = pbase;
        ci.shift_x = shx;
        ci.shift_y = shy;
        ci.probe_scale = (float)(1.0 / ((double)nx * ny));
        if ((rc = check(launch_col(ny, COL_PROBE, ci, st), "probe init"))) return rc;
        for (int p = 0; p < H; ++p) {
            RowArgs ra;
            std::memset(&ra, 0, sizeof(ra));
            ra.wave = wave;
            ra.trans = t + (size_t)p * px;
            ra.tw_fwd = twr_f;
            ra.tw_inv = twr_i;
            ra.ny = ny;
            ra.n_rows = nb * ny;
            ra.kx_half = M.kx_half;
            ra.tw = M.tw;
            if ((rc = check(launch_row_std(nx, ra, st), "row pass"))) return rc;
            const int pi = M.slice_prop[p];
            ColArgs ca = ci;
            ca.prop_x = prop_x + (size_t)pi * nx;
            ca.prop_y = prop_y + (size_t)pi * ny;
            ca.inten = inten;
            ca.probe_base = nullptr;
            // the detecting pass reads and writes every column, as in multislice_scan_run
            ca.kx_half = p + 1 == H ? 0 : M.kx_half;
            ca.band4 = M.band4;
            if ((rc = check(launch_col(ny, p + 1 == H ? COL_DETECT : COL_STD, ca, st), "column pass"))) return rc;
        }
        BinArgs ba;
        std::memset(&ba, 0, sizeof(ba));
        ba.inten = inten;
        ba.bin_off = d_off;
        ba.bin_idx = d_idx;
        ba.out = out_dev + (size_t)p0 * det->nbins;
        const double nn = (double)nx * ny;
        ba.scale = M.count > 0 ? nn * nn / M.count : 0.0;
        ba.npix = (int)px;
        ba.nbins = det->nbins;
        ba.batch = nb;
        if ((rc = check(launch_bins(ba, st), "bins"))) return rc;
    }
    return PRISM_OK;
}
