// engine.cpp -- host side of libprism: the C ABI declared in include/prism.h.
//
// Plans, validation, FP64 tables (beam set, propagators, anti-aliasing bounds, FFT twiddles,
// detector bin maps), stream-ordered device memory and kernel launch sequencing.  Compiled with
// -ffp-contract=off: every FP64 decision made here (beam membership, anti-aliasing mask, aperture,
// detector bin of a pixel) is evaluated with the same operations, in the same order, as its
// definition, so the integer outcome does not depend on the compiler fusing multiply-adds.
#include "prism.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"
#include "params.h"

namespace prism {
size_t scan_smem_bytes(int nw, int n_beams);
}

using namespace prism;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail(PRISM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char *prism_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ physics (CODATA 2018)
static const double H_PLANCK = 6.62607015e-34;
static const double M_ELECTRON = 9.1093837015e-31;
static const double Q_ELECTRON = 1.602176634e-19;
static const double C_LIGHT = 299792458.0;
static const double BEAM_SLACK = 1e-12;
static const double PI = 3.141592653589793;

// lambda = h / sqrt(2 m0 e V (1 + e V / (2 m0 c^2))), Angstrom
extern "C" double prism_wavelength(double kv) {
    const double ev = Q_ELECTRON * (kv * 1e3);
    const double p2 = 2.0 * M_ELECTRON * ev * (1.0 + ev / (2.0 * M_ELECTRON * C_LIGHT * C_LIGHT));
    return H_PLANCK / std::sqrt(p2) * 1e10;
}

// sigma = 2 pi m e lambda / h^2 with the relativistic mass m, rad/(V*Angstrom)
extern "C" double prism_interaction_constant(double kv) {
    const double ev = Q_ELECTRON * (kv * 1e3);
    const double m = M_ELECTRON + ev / (C_LIGHT * C_LIGHT);
    const double lam_m = prism_wavelength(kv) * 1e-10;
    return 2.0 * PI * m * Q_ELECTRON * lam_m / (H_PLANCK * H_PLANCK) * 1e-10;
}

// alpha_max = largest probe semi-angle + f lambda dq (PRISM Algorithm section), plus the tilt of the
// aperture's centre; dq on the coarser beam-lattice axis
extern "C" int prism_recommended_alpha_max(const prism_grid *g, const prism_probe *probe, double *out) {
    if (!g || !probe || !out) return fail(PRISM_ERR_INVALID, "NULL argument");
    if (!(g->kv > 0) || g->f < 1 || g->f_y < 0 || !(g->cell_x > 0) || !(g->cell_y > 0) || !(probe->alpha_mrad >= 0))
        return fail(PRISM_ERR_INVALID, "prism_recommended_alpha_max: kv, f, f_y, cells or alpha out of range");
    const int fy = g->f_y ? g->f_y : g->f;
    const double step = std::max((double)g->f / g->cell_x, (double)fy / g->cell_y);
    *out = probe->alpha_mrad + 1000.0 * std::hypot(probe->tilt_x, probe->tilt_y) + 1000.0 * prism_wavelength(g->kv) * step;
    return PRISM_OK;
}

static inline int signed_index(int k, int n) { return k < n / 2 ? k : k - n; }
static inline bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// W_N^m = exp(-2 pi i m / N)
static float2 wN(long long m, int N) {
    m %= N;
    if (m < 0) m += N;
    const double a = 2.0 * PI * (double)m / (double)N;
    return make_float2((float)std::cos(a), (float)-std::sin(a));
}

// exp(-2 pi i c) for a phase in cycles, reduced before the trigonometric call
static float2 phase_cycles(double c) {
    c -= std::floor(c);
    const double a = 2.0 * PI * c;
    return make_float2((float)std::cos(a), (float)-std::sin(a));
}

static Tw64 make_tw64() {
    Tw64 t;
    for (int j = 0; j < 64; ++j) {
        t.w[j] = wN(j, 64);
        // tangent form (the kernels pick the same form from j at compile time)
        const double a = -2.0 * PI * (double)j / 64.0, c = std::cos(a), s = std::sin(a);
        const bool tan_form = (j & 31) <= 8 || (j & 31) >= 24;
        const float sc = (float)(tan_form ? c : s);
        t.sc[j] = make_float2(sc, sc);
        t.tk[j] = (float)(tan_form ? s / c : c / s);
    }
    return t;
}

// inter-stage twiddles of a two-level FFT with split (A, B): table[k1 * B + n2] = W_N^{n2 k1}
static std::vector<float2> stage_table(int N, int A, int B) {
    std::vector<float2> t((size_t)A * B);
    for (int k1 = 0; k1 < A; ++k1)
        for (int n2 = 0; n2 < B; ++n2) t[(size_t)k1 * B + n2] = wN((long long)n2 * k1, N);
    return t;
}

// A caller's device pointer must be device (or managed) memory of the current device; V is read
// with 16-byte vector loads, so it must also be 16-byte aligned.
static int check_dev_ptr(const void *p, size_t align, const char *what) {
    if (!p) return fail(PRISM_ERR_INVALID, std::string(what) + " is NULL");
    if (((uintptr_t)p) % align) return fail(PRISM_ERR_INVALID, std::string(what) + " is not " + std::to_string(align) + "-byte aligned");
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PRISM_ERR_INVALID, std::string(what) + " is not a CUDA pointer");
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (!(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) || at.device != dev)
        return fail(PRISM_ERR_INVALID, std::string(what) + " is not device memory of the current device");
    return PRISM_OK;
}

// ------------------------------------------------------------------ device memory helpers
struct DevArena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    int alloc(void **p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 16;
        cudaError_t e = cudaMallocAsync(p, n, stream);
        if (e != cudaSuccess) {
            *p = nullptr;
            return fail(PRISM_ERR_CUDA, std::string("cudaMallocAsync(") + std::to_string(n) + "): " + cudaGetErrorString(e));
        }
        ptrs.push_back(*p);
        bytes += n;
        return PRISM_OK;
    }
    template <class T>
    int upload(T **p, const std::vector<T> &h) {
        int rc = alloc((void **)p, h.size() * sizeof(T));
        if (rc) return rc;
        if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, stream));
        return PRISM_OK;
    }
    void release() {
        for (void *p : ptrs) cudaFreeAsync(p, stream);
        ptrs.clear();
        bytes = 0;
    }
    void forget(void *p, size_t n) {
        auto it = std::find(ptrs.begin(), ptrs.end(), p);
        if (it != ptrs.end()) {
            cudaFreeAsync(p, stream);
            ptrs.erase(it);
            bytes -= n;
        }
    }
};

// ------------------------------------------------------------------ grid validation and tables
struct GridTables {
    int nx, ny, H;
    double lam, sigma;
    std::vector<double> dz;           // per slice
    std::vector<int> slice_prop;      // slice -> propagator table index
    std::vector<double> prop_dz;      // distinct thicknesses
    std::vector<float2> prop_x, prop_y;
    std::vector<int> aa_kmax;
    int kx_half = 0;                  // columns |kx| < kx_half pass the aperture (0: all columns)
    int band4 = 0;                    // every column passes at most |ky| < ny/4
    double q_aa;
    std::vector<float2> twr_f, twr_i, twc_f, twc_i;
};

static int check_grid_common(const prism_grid *g) {
    if (!g) return fail(PRISM_ERR_INVALID, "grid is NULL");
    if (g->nx <= 0 || g->ny <= 0 || g->n_slices <= 0) return fail(PRISM_ERR_INVALID, "nx, ny and n_slices must be positive");
    if (!(g->cell_x > 0) || !(g->cell_y > 0) || !std::isfinite(g->cell_x) || !std::isfinite(g->cell_y))
        return fail(PRISM_ERR_INVALID, "cell sizes must be positive and finite");
    if (!(g->kv > 0) || !std::isfinite(g->kv)) return fail(PRISM_ERR_INVALID, "kv must be positive");
    if (!(g->aa_frac > 0) || g->aa_frac > 1.0) return fail(PRISM_ERR_INVALID, "aa_frac must be in (0, 1]");
    if (!g->slice_dz && (!(g->dz >= 0) || !std::isfinite(g->dz))) return fail(PRISM_ERR_INVALID, "dz must be >= 0");
    if (g->slice_dz)
        for (int p = 0; p < g->n_slices; ++p)
            if (!(g->slice_dz[p] >= 0) || !std::isfinite(g->slice_dz[p])) return fail(PRISM_ERR_INVALID, "slice_dz must be >= 0");
    if (!pow2(g->nx) || !pow2(g->ny) || g->nx < 16 || g->ny < 16 || g->nx > 2048 || g->ny > 2048)
        return fail(PRISM_ERR_UNSUPPORTED, "nx and ny must be powers of two in [16, 2048]");
    return PRISM_OK;
}

static int build_grid_tables(const prism_grid *g, GridTables &T) {
    T.nx = g->nx;
    T.ny = g->ny;
    T.H = g->n_slices;
    T.lam = prism_wavelength(g->kv);
    T.sigma = prism_interaction_constant(g->kv);
    T.dz.resize(T.H);
    for (int p = 0; p < T.H; ++p) T.dz[p] = g->slice_dz ? g->slice_dz[p] : g->dz;
    T.slice_prop.resize(T.H);
    for (int p = 0; p < T.H; ++p) {
        int idx = -1;
        for (size_t i = 0; i < T.prop_dz.size(); ++i)
            if (T.prop_dz[i] == T.dz[p]) idx = (int)i;
        if (idx < 0) {
            idx = (int)T.prop_dz.size();
            T.prop_dz.push_back(T.dz[p]);
        }
        T.slice_prop[p] = idx;
    }
    // Fresnel propagator exp(-i pi lambda t q^2) factored per axis; 1/(nx ny) of the inverse FFT
    // folded into the y factor
    const double inv = 1.0 / ((double)T.nx * (double)T.ny);
    for (double dzv : T.prop_dz) {
        for (int k = 0; k < T.nx; ++k) {
            const double q = (double)signed_index(k, T.nx) / g->cell_x;
            T.prop_x.push_back(phase_cycles(0.5 * T.lam * dzv * q * q));
        }
        for (int k = 0; k < T.ny; ++k) {
            const double q = (double)signed_index(k, T.ny) / g->cell_y;
            float2 w = phase_cycles(0.5 * T.lam * dzv * q * q);
            T.prop_y.push_back(make_float2((float)(w.x * inv), (float)(w.y * inv)));
        }
    }
    // anti-aliasing aperture |q| < aa_frac * q_nyquist, as a per-column bound on |ky| (the column
    // pass applies it along each column kx)
    const double q_nyq = std::min(0.5 * T.nx / g->cell_x, 0.5 * T.ny / g->cell_y);
    T.q_aa = g->aa_frac * q_nyq;
    const double qaa2 = T.q_aa * T.q_aa;
    T.aa_kmax.assign(T.nx, -1);
    for (int kx = 0; kx < T.nx; ++kx) {
        const double qx = (double)signed_index(kx, T.nx) / g->cell_x;
        int kmax = -1;
        for (int ky = 0; ky < T.ny; ++ky) {
            const int ks = signed_index(ky, T.ny);
            const double qy = (double)ks / g->cell_y;
            const bool in = qx * qx + qy * qy < qaa2;
            if (in) kmax = std::max(kmax, std::abs(ks));
        }
        // the mask must be the symmetric interval |ky| <= kmax
        for (int ky = 0; ky < T.ny; ++ky) {
            const int ks = signed_index(ky, T.ny);
            const double qy = (double)ks / g->cell_y;
            const bool in = qx * qx + qy * qy < qaa2;
            if (in != (std::abs(ks) <= kmax)) return fail(PRISM_ERR_INVALID, "anti-aliasing mask is not a symmetric interval");
        }
        T.aa_kmax[kx] = kmax;
    }
    // columns that pass the aperture: |kx| <= K, a symmetric interval (else no pruning)
    int K = -1;
    for (int kx = 0; kx < T.nx; ++kx)
        if (T.aa_kmax[kx] >= 0) K = std::max(K, std::abs(signed_index(kx, T.nx)));
    bool interval = K >= 0;
    for (int kx = 0; kx < T.nx && interval; ++kx)
        interval = (T.aa_kmax[kx] >= 0) == (std::abs(signed_index(kx, T.nx)) <= K);
    T.kx_half = interval && K + 1 < T.nx / 2 ? K + 1 : 0;
    T.band4 = *std::max_element(T.aa_kmax.begin(), T.aa_kmax.end()) < T.ny / 4;
    int a1, a2;
    fft_split(T.nx, &a1, &a2);
    T.twr_f = stage_table(T.nx, a1, a2);
    T.twr_i = stage_table(T.nx, a2, a1);
    fft_split(T.ny, &a1, &a2);
    T.twc_f = stage_table(T.ny, a1, a2);
    T.twc_i = stage_table(T.ny, a2, a1);
    return PRISM_OK;
}

// CSR of pixels grouped by detector bin: bin = floor((1000 lambda |q| - start) / step), q =
// (k_x mult_x / cell_x, k_y mult_y / cell_y), pixel index ky * nx + kx in FFT order.
static void detector_csr(int nx, int ny, double cell_x, double cell_y, int mult_x, int mult_y, double lam,
                         const prism_detector *det, std::vector<int> &off, std::vector<int> &idx) {
    std::vector<int> bin((size_t)nx * ny);
    off.assign(det->nbins + 1, 0);
    for (int ky = 0; ky < ny; ++ky) {
        const double qy = ((double)signed_index(ky, ny) * mult_y) / cell_y;
        for (int kx = 0; kx < nx; ++kx) {
            const double qx = ((double)signed_index(kx, nx) * mult_x) / cell_x;
            const double theta = 1000.0 * lam * std::sqrt(qx * qx + qy * qy);
            const double bf = std::floor((theta - det->start_mrad) / det->step_mrad);
            int b = -1;
            if (bf >= 0 && bf < det->nbins) b = (int)bf;
            bin[(size_t)ky * nx + kx] = b;
            if (b >= 0) off[b + 1]++;
        }
    }
    for (int b = 0; b < det->nbins; ++b) off[b + 1] += off[b];
    idx.assign(off[det->nbins], 0);
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (size_t i = 0; i < bin.size(); ++i)
        if (bin[i] >= 0) idx[fill[bin[i]]++] = (int)i;
}

static int check_det(const prism_detector *det) {
    if (!det) return fail(PRISM_ERR_INVALID, "detector is NULL");
    if (det->nbins < 1 || det->nbins > 4096) return fail(PRISM_ERR_INVALID, "nbins must be in [1, 4096]");
    if (!(det->step_mrad > 0) || !std::isfinite(det->step_mrad) || !std::isfinite(det->start_mrad))
        return fail(PRISM_ERR_INVALID, "detector step must be positive and finite");
    return PRISM_OK;
}

static int check_probe(const prism_probe *pr) {
    if (!pr) return fail(PRISM_ERR_INVALID, "probe is NULL");
    if (!(pr->alpha_mrad >= 0) || !std::isfinite(pr->alpha_mrad) || !std::isfinite(pr->c1) || !std::isfinite(pr->c3))
        return fail(PRISM_ERR_INVALID, "probe parameters must be finite, alpha >= 0");
    if (!std::isfinite(pr->tilt_x) || !std::isfinite(pr->tilt_y) || std::fabs(pr->tilt_x) > 0.5 || std::fabs(pr->tilt_y) > 0.5)
        return fail(PRISM_ERR_INVALID, "probe tilt must be finite and below 0.5 rad");
    return PRISM_OK;
}

static int check_scan(const prism_scan *sc, double lim_x, double lim_y) {
    if (!sc) return fail(PRISM_ERR_INVALID, "scan is NULL");
    if (sc->px < 0 || sc->py < 0) return fail(PRISM_ERR_INVALID, "scan sizes must be >= 0");
    const long long P = (long long)sc->px * sc->py;
    if (P > (1LL << 30)) return fail(PRISM_ERR_INVALID, "too many probe positions");
    if (P > 0 && (!sc->x0 || !sc->y0)) return fail(PRISM_ERR_INVALID, "scan positions are NULL");
    for (long long i = 0; i < P; ++i)
        if (!std::isfinite(sc->x0[i]) || !std::isfinite(sc->y0[i]) || std::fabs(sc->x0[i]) > lim_x || std::fabs(sc->y0[i]) > lim_y)
            return fail(PRISM_ERR_INVALID, "probe position not finite or beyond 2^28 pixels");
    return PRISM_OK;
}

// aperture A(q): lambda |q| <= alpha (inclusive, 1e-12 relative slack)
static bool inside_aperture(double qx, double qy, double lam, double alpha_rad) {
    const double ax = lam * qx;
    const double ay = lam * qy;
    return ax * ax + ay * ay <= alpha_rad * alpha_rad * (1.0 + BEAM_SLACK);
}

// chi(q) = pi lambda q^2 C1 + (pi/2) lambda^3 q^4 C3, returned in cycles (chi / 2 pi)
static double chi_cycles(double q2, double lam, double c1, double c3) {
    const double chi = PI * lam * q2 * c1 + 0.5 * PI * lam * lam * lam * q2 * q2 * c3;
    return chi / (2.0 * PI);
}

// Probe tilt (PRISM Algorithm section): aperture and chi centred on q_t = theta / lambda, and the
// coefficients evaluated at r0 - h tan(theta) with h the cell thickness.
struct Tilt {
    double qtx, qty, sx, sy;
};
static Tilt tilt_terms(const prism_probe *pr, double lam, const std::vector<double> &dz) {
    double h = 0;
    for (double d : dz) h += d;
    return {pr->tilt_x / lam, pr->tilt_y / lam, h * std::tan(pr->tilt_x), h * std::tan(pr->tilt_y)};
}

// ------------------------------------------------------------------ plan
struct PendingEv {
    int kind;
    cudaEvent_t a, b;
};

struct prism_plan {
    prism_grid g;
    GridTables T;
    cudaStream_t stream = nullptr;
    int device = 0;
    int nxs = 0, nys = 0, nw = 0, nwy = 0, fy = 1, nbeams = 0, batch = 0;  // nw: window x side
    std::vector<int> bm, bn;
    bool built = false;
    size_t budget = 0;
    DevArena arena;
    // device tables / buffers
    float2 *t = nullptr, *wave = nullptr, *S = nullptr;  // S: all beams (FP32 mode) or one beam batch (16-bit)
    float2 *t0f = nullptr;     // FFT_x(t_0) [ny][nx]: the first slice of every beam by the shift theorem
    int *zero_mn = nullptr;    // the (0, 0) beam that makes it
    int prec = PRISM_PRECISION_FP32;
    void *S16 = nullptr;       // 16-bit mode: [ny_s * nx_s][kp]
    float *scale = nullptr;    // 16-bit mode: [kp / 2] per-beam power-of-two scales
    int kp = 0;
    float2 *win = nullptr;     // scan window scratch (GEMM and tensor-core scans)
    size_t win_cap = 0;
    int *win_cnt = nullptr;    // scans: completion counters of split groups, work-unit counters
    size_t cnt_cap = 0;
    CUtensorMap wave_map, wave_map4;  // the wave stack for the TMA-staged column pass (8 / 4 columns per box)
    CUtensorMap out_map, out_map4;    // its stores (ColArgs::out_map)
    bool shared_sms = false;   // a batch runs this plan's kernels beside other cells' (see col_default_shape)
    bool wave_map_ok = false;
    int *dev_err = nullptr;    // device error word
    int *col_ctr = nullptr;    // the TMA-staged column pass's tile counter and CTAs done (int[2])
    int tune_shape[2] = {-1, -1};  // autotuned launch shape of ROW_STD / COL_STD (-1: default launcher)
    double tune_ms[2][PRISM_TUNE_MAX_SHAPES];
    bool tuned[2] = {false, false};
    int scan_shape = 0;            // contraction tile shape of the FP32 GEMM scan (0: default)
    double scan_ms[PRISM_TUNE_MAX_SHAPES];
    bool scan_tuned = false;
    int tc_shape = 0;              // ring shape of the tensor-core scan (16-bit modes; 0: default)
    double tc_ms[PRISM_TUNE_MAX_SHAPES];
    bool tc_tuned = false;
    float2 *prop_x = nullptr, *prop_y = nullptr;
    int *aa_kmax = nullptr;
    float2 *twr_f = nullptr, *twr_i = nullptr, *twc_f = nullptr, *twc_i = nullptr, *tww_f = nullptr, *tww_fy = nullptr;
    int *beam_mn = nullptr;
    double *beam_q = nullptr;  // qx[B] then qy[B]
    // grown on demand
    double *pos = nullptr;
    size_t pos_cap = 0;
    float2 *base = nullptr;
    int *bin_buf = nullptr;    // window detector: CSR offsets, CSR indices, indices by rank
    size_t bin_cap = 0;
    size_t bin_t_off = 0;      // element offset of the by-rank table in bin_buf
    size_t bin_16_off = 0;     // element offset of the 16-bit lists in bin_buf (a multiple of 4)
    size_t bin_n = 0;          // entries of the lists
    float *out_stage = nullptr;
    size_t out_cap = 0;
    float *v_stage = nullptr;
    size_t v_cap = 0;
    // host-buffer builds: potential chunks copied on their own stream, each chunk's transmission
    // launched once its copy is done (the copy of later chunks overlaps the first slices' passes)
    cudaStream_t copy = nullptr;
    cudaEvent_t copy_start = nullptr;
    std::vector<cudaEvent_t> copy_done;
    Tw64 tw64;
    // cached detector map
    double det_key[2] = {0, 0};
    int det_nbins = -1;
    // statistics
    long launches = 0;
    bool profiling = false;
    std::vector<PendingEv> pending;
    std::vector<cudaEvent_t> ev_pool;
    double kms[PRISM_K_COUNT] = {0};
    long kl[PRISM_K_COUNT] = {0};
};

template <class F>
static int plan_launch(prism_plan *P, int kind, F &&fn) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (P->profiling) {
        for (cudaEvent_t *e : {&a, &b}) {
            if (!P->ev_pool.empty()) {
                *e = P->ev_pool.back();
                P->ev_pool.pop_back();
            } else {
                CUDA_TRY(cudaEventCreate(e));
            }
        }
        CUDA_TRY(cudaEventRecord(a, P->stream));
    }
    cudaError_t e = fn();
    if (e != cudaSuccess) return fail(PRISM_ERR_CUDA, std::string("kernel launch (") + prism_kernel_name(kind) + "): " + cudaGetErrorString(e));
    if (P->profiling) {
        CUDA_TRY(cudaEventRecord(b, P->stream));
        P->pending.push_back({kind, a, b});
    }
    P->kl[kind]++;
    P->launches++;
    return PRISM_OK;
}

static int grow(DevArena &A, void **p, size_t *cap, size_t need) {
    if (need <= *cap && *p) return PRISM_OK;
    if (*p) A.forget(*p, *cap);
    *p = nullptr;
    *cap = 0;
    int rc = A.alloc(p, need);
    if (rc) return rc;
    *cap = need;
    return PRISM_OK;
}

// tensor-core scan mode of a 16-bit precision (kernels_tc.cu: 0 FP16, 1 BF16, 2 FP16 value + remainder)
static int tc_mode(int prec) { return prec == PRISM_PRECISION_BF16 ? 1 : prec == PRISM_PRECISION_FP16X2 ? 2 : 0; }
// 16-bit rows stored per pixel
static int tc_parts(int prec) { return prec == PRISM_PRECISION_FP16X2 ? 2 : 1; }

// The driver's tensor-map encoder through the runtime's entry-point query (null if unavailable)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    return encode;
}

// Tensor map of a wave stack [batch][ny][nx] complex64 for the TMA-staged column pass: FP32 view
// [batch][ny][2 nx], boxes of 2 w floats (w = 4 or 8 columns) x min(ny, 256) rows x 1.  The encoder comes from
// the driver through the runtime's entry-point query; false (shape not used) if it is unavailable
// or the stack breaks a rule of the map (16-byte aligned base, strides multiples of 16 bytes).
static bool encode_wave_map(CUtensorMap &map, const float2 *wave, int nx, int ny, int batch, int w) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    std::memset(&map, 0, sizeof(map));
    if (!encode || !wave || ((uintptr_t)wave & 15) || nx < 8 || nx % 8 || ny < 1 || batch < 1) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * nx, (cuuint64_t)ny, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * nx * sizeof(float), (cuuint64_t)2 * nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * w), (cuuint32_t)std::min(ny, 256), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(wave), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map for the TMA stores of the column pass: the same stack as FP32 [batch][lanes][regs][2 nx]
// with row y = lane + lanes * reg (the column transform's result layout, col_fft_geometry), boxes of
// 2 w floats x (regs + 1) x 32 / w x 1: one warp's lanes of a finished tile in the exchange layout,
// whose pad entry (reg = regs) lies outside the map and is not stored.
static bool encode_out_map(CUtensorMap &map, const float2 *wave, int nx, int ny, int batch, int w) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    std::memset(&map, 0, sizeof(map));
    int lanes = 0, regs = 0;
    if (!encode || !wave || ((uintptr_t)wave & 15) || nx < 8 || nx % 8 || batch < 1 || (w != 4 && w != 8) ||
        !col_fft_geometry(ny, &lanes, &regs) || lanes * regs != ny || lanes % (32 / w) || regs + 1 > 256)
        return false;
    const cuuint64_t row = (cuuint64_t)2 * nx * sizeof(float);
    const cuuint64_t dims[4] = {(cuuint64_t)2 * nx, (cuuint64_t)regs, (cuuint64_t)lanes, (cuuint64_t)batch};
    const cuuint64_t strides[3] = {row * lanes, row, row * ny};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * w), (cuuint32_t)(regs + 1), (cuuint32_t)(32 / w), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2 *>(wave), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the load and store maps of a wave stack for both column counts; false if any cannot be encoded
static bool encode_wave_maps(CUtensorMap &m8, CUtensorMap &m4, CUtensorMap &o8, CUtensorMap &o4, const float2 *wave, int nx,
                             int ny, int batch) {
    return encode_wave_map(m8, wave, nx, ny, batch, 8) && encode_wave_map(m4, wave, nx, ny, batch, 4) &&
           encode_out_map(o8, wave, nx, ny, batch, 8) && encode_out_map(o4, wave, nx, ny, batch, 4);
}

extern "C" int prism_plan_create(const prism_grid *grid, size_t hbm_budget_bytes, void *cuda_stream, prism_plan **out) {
    if (!out) return fail(PRISM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int rc = check_grid_common(grid);
    if (rc) return rc;
    const prism_grid &g = *grid;
    if (g.f < 1) return fail(PRISM_ERR_INVALID, "f must be >= 1");
    if (g.f_y < 0) return fail(PRISM_ERR_INVALID, "f_y must be >= 0 (0: f_y = f)");
    const int fy = g.f_y > 0 ? g.f_y : g.f;
    if (g.downsample != 1 && g.downsample != 2) return fail(PRISM_ERR_INVALID, "downsample must be 1 or 2");
    if (g.downsample == 2 && g.aa_frac > 0.5) return fail(PRISM_ERR_INVALID, "downsample 2 needs aa_frac <= 0.5");
    if (!(g.alpha_max_mrad > 0) || !std::isfinite(g.alpha_max_mrad)) return fail(PRISM_ERR_INVALID, "alpha_max_mrad must be positive");
    if ((g.nx % (g.downsample * g.f)) || (g.ny % (g.downsample * fy)))
        return fail(PRISM_ERR_INVALID, "nx must be divisible by downsample * f and ny by downsample * f_y");
    const int nxs = g.nx / g.downsample, nys = g.ny / g.downsample;
    const int nwx = nxs / g.f, nwy = nys / fy;
    const auto side_ok = [](int n) { return n == 16 || n == 32 || n == 64; };
    if (nwx == nwy ? !scan_supported(nwx) : !(side_ok(nwx) && side_ok(nwy)))
        return fail(PRISM_ERR_UNSUPPORTED, "scan window must be square with 8, 16, 32, 64 or 128 pixels, or have sides of 16, 32 or 64");
    if (g.precision != PRISM_PRECISION_FP32 && g.precision != PRISM_PRECISION_FP16 && g.precision != PRISM_PRECISION_BF16 &&
        g.precision != PRISM_PRECISION_FP16X2)
        return fail(PRISM_ERR_INVALID, "precision must be PRISM_PRECISION_FP32, _FP16, _BF16 or _FP16X2");
    const bool half = g.precision != PRISM_PRECISION_FP32;
    if (half && nwx != nwy) return fail(PRISM_ERR_UNSUPPORTED, "16-bit precision needs a square scan window (f_y = f on a square grid)");
    if (half && !scan_tc_supported(nwx))
        return fail(PRISM_ERR_UNSUPPORTED, "16-bit precision needs a scan window of 16, 32 or 64 pixels");

    int device = 0;
    CUDA_TRY(cudaGetDevice(&device));
    prism_plan *P = new prism_plan();
    P->device = device;
    P->g = g;
    P->g.slice_dz = nullptr;
    P->stream = (cudaStream_t)cuda_stream;
    P->arena.stream = P->stream;
    P->budget = hbm_budget_bytes;
    P->nxs = nxs;
    P->nys = nys;
    P->nw = nwx;
    P->nwy = nwy;
    P->fy = fy;
    P->prec = g.precision;
    rc = build_grid_tables(&g, P->T);
    if (rc) {
        delete P;
        return rc;
    }
    // plane-wave set (PRISM Algorithm section): q_mn = (m f / cx, n f / cy), lambda |q| <= alpha_max
    const double lam = P->T.lam;
    const double alpha = g.alpha_max_mrad * 1e-3;
    const int mmax = (int)std::floor(alpha / (lam * g.f / g.cell_x)) + 1;
    const int nmax = (int)std::floor(alpha / (lam * fy / g.cell_y)) + 1;
    std::vector<double> bq;
    for (int n = -nmax; n <= nmax; ++n)
        for (int m = -mmax; m <= mmax; ++m) {
            const double qx = (double)(m * g.f) / g.cell_x;
            const double qy = (double)(n * fy) / g.cell_y;
            if (inside_aperture(qx, qy, lam, alpha)) {
                if (!(qx * qx + qy * qy < P->T.q_aa * P->T.q_aa)) {
                    delete P;
                    return fail(PRISM_ERR_INVALID, "beam outside the anti-aliasing aperture: alpha_max too large for the grid");
                }
                P->bm.push_back(m);
                P->bn.push_back(n);
            }
        }
    P->nbeams = (int)P->bm.size();
    if (P->nbeams == 0) {
        delete P;
        return fail(PRISM_ERR_INVALID, "empty beam set");
    }
    P->kp = 2 * ((P->nbeams + 7) / 8 * 8);
    if (half ? scan_tc_grid(P->nw, P->kp, tc_mode(P->prec), 0, 1, 1) <= 0
             : nwx == nwy ? scan_smem_bytes(P->nw, P->nbeams) > 227 * 1024 : !scan_rect_supported(nwx, nwy, P->nbeams)) {
        delete P;
        return fail(PRISM_ERR_UNSUPPORTED, "too many beams for the scan kernel's shared memory");
    }
    std::vector<int> mn(2 * P->nbeams);
    std::vector<double> q(2 * P->nbeams);
    for (int b = 0; b < P->nbeams; ++b) {
        mn[2 * b] = P->bm[b];
        mn[2 * b + 1] = P->bn[b];
        q[b] = (double)(P->bm[b] * g.f) / g.cell_x;
        q[P->nbeams + b] = (double)(P->bn[b] * fy) / g.cell_y;
    }
    // memory plan
    const size_t px = (size_t)g.nx * g.ny;
    const size_t t_bytes = (size_t)g.n_slices * px * 8;
    // FP32 mode keeps S for all beams; 16-bit mode keeps the pixel-major 16-bit S plus one FP32
    // beam batch that the quantiser reads
    const size_t sbeam = (size_t)nxs * nys * 8;
    const size_t s16_bytes = half ? (size_t)nxs * nys * P->kp * 2 * tc_parts(g.precision) + (size_t)P->kp / 2 * sizeof(float) : 0;
    const size_t w_bytes = px * 8;
    const size_t per_beam = w_bytes + (half ? sbeam : 0);
    const size_t fixed = t_bytes + px * 8 + (half ? s16_bytes : (size_t)P->nbeams * sbeam) + (1 << 20);
    int batch = P->nbeams;
    if (hbm_budget_bytes) {
        if (fixed + per_beam > hbm_budget_bytes) {
            delete P;
            return fail(PRISM_ERR_BUDGET, "plan needs " + std::to_string(fixed + per_beam) + " bytes, budget " + std::to_string(hbm_budget_bytes));
        }
        batch = (int)std::min<size_t>(P->nbeams, (hbm_budget_bytes - fixed) / per_beam);
    }
    P->batch = batch;
    const size_t s_bytes = (half ? (size_t)batch : (size_t)P->nbeams) * sbeam;
    P->tw64 = make_tw64();
    std::vector<float2> tww_f, tww_fy;
    {
        int a1, a2;
        fft_split(P->nw, &a1, &a2);
        tww_f = stage_table(P->nw, a1, a2);
        fft_split(P->nwy, &a1, &a2);
        tww_fy = stage_table(P->nwy, a1, a2);
    }
    DevArena &A = P->arena;
    auto bail = [&](int code) {
        A.release();
        cudaStreamSynchronize(P->stream);
        delete P;
        return code;
    };
    if ((rc = A.alloc((void **)&P->t, t_bytes))) return bail(rc);
    if ((rc = A.alloc((void **)&P->S, s_bytes))) return bail(rc);
    if (half) {
        if ((rc = A.alloc(&P->S16, (size_t)nxs * nys * P->kp * 2 * tc_parts(P->prec)))) return bail(rc);
        if ((rc = A.alloc((void **)&P->scale, (size_t)P->kp / 2 * sizeof(float)))) return bail(rc);
        // padded beams stay zero in S16 (their coefficients are zero too, and 0 * 0 must not be NaN)
        CUDA_TRY(cudaMemsetAsync(P->S16, 0, (size_t)nxs * nys * P->kp * 2 * tc_parts(P->prec), P->stream));
        CUDA_TRY(cudaMemsetAsync(P->scale, 0, (size_t)P->kp / 2 * sizeof(float), P->stream));
    }
    if ((rc = A.alloc((void **)&P->dev_err, sizeof(int)))) return bail(rc);
    CUDA_TRY(cudaMemsetAsync(P->dev_err, 0, sizeof(int), P->stream));
    if ((rc = A.alloc((void **)&P->col_ctr, 2 * sizeof(int)))) return bail(rc);
    CUDA_TRY(cudaMemsetAsync(P->col_ctr, 0, 2 * sizeof(int), P->stream));
    if ((rc = A.alloc((void **)&P->wave, (size_t)batch * w_bytes))) return bail(rc);
    if ((rc = A.alloc((void **)&P->t0f, px * 8))) return bail(rc);
    if ((rc = A.alloc((void **)&P->zero_mn, 2 * sizeof(int)))) return bail(rc);
    CUDA_TRY(cudaMemsetAsync(P->zero_mn, 0, 2 * sizeof(int), P->stream));
    P->wave_map_ok = encode_wave_maps(P->wave_map, P->wave_map4, P->out_map, P->out_map4, P->wave, g.nx, g.ny, batch);
    if ((rc = A.upload(&P->prop_x, P->T.prop_x))) return bail(rc);
    if ((rc = A.upload(&P->prop_y, P->T.prop_y))) return bail(rc);
    if ((rc = A.upload(&P->aa_kmax, P->T.aa_kmax))) return bail(rc);
    if ((rc = A.upload(&P->twr_f, P->T.twr_f))) return bail(rc);
    if ((rc = A.upload(&P->twr_i, P->T.twr_i))) return bail(rc);
    if ((rc = A.upload(&P->twc_f, P->T.twc_f))) return bail(rc);
    if ((rc = A.upload(&P->twc_i, P->T.twc_i))) return bail(rc);
    if ((rc = A.upload(&P->tww_f, tww_f))) return bail(rc);
    if ((rc = A.upload(&P->tww_fy, tww_fy))) return bail(rc);
    if ((rc = A.upload(&P->beam_mn, mn))) return bail(rc);
    if ((rc = A.upload(&P->beam_q, q))) return bail(rc);
    if ((rc = A.alloc((void **)&P->base, (size_t)P->nbeams * sizeof(float2)))) return bail(rc);
    // the uploads above read host vectors that die with this scope
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        fail(PRISM_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e));
        return bail(PRISM_ERR_CUDA);
    }
    *out = P;
    return PRISM_OK;
}

extern "C" void prism_plan_destroy(prism_plan *P) {
    if (!P) return;
    cudaStreamSynchronize(P->stream);
    for (auto &pe : P->pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (auto e : P->ev_pool) cudaEventDestroy(e);
    if (P->copy) {
        cudaStreamSynchronize(P->copy);
        cudaStreamDestroy(P->copy);
    }
    if (P->copy_start) cudaEventDestroy(P->copy_start);
    for (auto e : P->copy_done) cudaEventDestroy(e);
    P->arena.release();
    cudaStreamSynchronize(P->stream);
    delete P;
}

extern "C" int prism_sync(prism_plan *P) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    CUDA_TRY(cudaGetLastError());
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CUDA_TRY(cudaMemset(P->dev_err, 0, sizeof(int)));
        // a scan or column pass whose wait ran out may have left its counters mid-count
        if (P->win_cnt) CUDA_TRY(cudaMemset(P->win_cnt, 0, P->cnt_cap));
        CUDA_TRY(cudaMemset(P->col_ctr, 0, 2 * sizeof(int)));
        return fail(PRISM_ERR_DEVICE, "a kernel's bounded wait ran out (device error word " + std::to_string(err) + ")");
    }
    return PRISM_OK;
}

// ------------------------------------------------------------------ S-matrix build
static RowArgs row_args(prism_plan *P) {
    RowArgs a;
    std::memset(&a, 0, sizeof(a));
    a.wave = P->wave;
    a.tw_fwd = P->twr_f;
    a.tw_inv = P->twr_i;
    a.s_out = P->S;
    a.beam_mn = P->beam_mn;
    a.ny = P->g.ny;
    a.f = P->g.f;
    a.f_y = P->fy;
    a.downsample = P->g.downsample;
    a.kx_half = P->T.kx_half;
    a.err = P->dev_err;
    a.tw = P->tw64;
    return a;
}

static ColArgs col_args(const GridTables &T, float2 *wave, const float2 *prop_x, const float2 *prop_y,
                        const int *aa_kmax, const float2 *tf, const float2 *ti, const Tw64 &tw) {
    ColArgs a;
    std::memset(&a, 0, sizeof(a));
    a.wave = wave;
    a.prop_x = prop_x;
    a.prop_y = prop_y;
    a.aa_kmax = aa_kmax;
    a.tw_fwd = tf;
    a.tw_inv = ti;
    a.nx = T.nx;
    a.tw = tw;
    (void)T;
    return a;
}

static int build_launches(prism_plan *P, const float *V_dev, int per = 0);

// the column pass's launch shape when none is tuned or pinned: at N = 1024 the TMA-staged shape of
// 4 columns per CTA, 3 CTAs per SM (the fastest there: 0.275 ms per launch on the 1024^2 carbon
// workload, against 0.293 with 8 columns and 0.320 for cp.async staging), when the plan holds the
// tensor maps of its wave; otherwise the default launcher (-1)
// In a batch graph with parallel branches the passes of different cells share the SMs, and a shape
// that fills an SM by itself (3 CTAs of 66 KB and 168 x 128 registers) leaves no room for the
// other branches' kernels: there the 8-column TMA shape (one 131 KB CTA per SM) is the default, and
// the autotuner skips the SM-filling shapes (64 uneven cells, 4 branches: 2.78 s per run with them,
// 2.25 s without).
static int col_default_shape(const prism_plan *P) {
    if (P->g.ny != 1024 || !P->wave_map_ok) return -1;
    const int v = tune_col_tma_shape(P->shared_sms ? 8 : 4);
    return v >= 0 && tune_shape_valid(PRISM_TUNE_COL, 1024, v) ? v : -1;
}

// the row pass's launch shape when none is tuned or pinned: at N = 1024, 384 threads (12 warps per
// SM) with the next row's two kept quarters staged by bulk TMA copies (0.292 ms per launch on the
// 1024^2 carbon workload, against 0.315 for 256 threads staged by cp.async and 0.333 for 128 threads
// unstaged); in a batch graph, whose branches share the SMs, the default launcher's smaller CTAs
// (this shape holds 163 KB of shared memory per CTA)
static int row_default_shape(const prism_plan *P) {
    if (P->g.nx != 1024 || P->shared_sms) return -1;
    const int v = tune_row_find(384, false, true);
    return v >= 0 && tune_shape_valid(PRISM_TUNE_ROW, 1024, v) ? v : -1;
}

// the plan's wave stack in the column arguments of its build and autotuner launches
static void col_wave_map(const prism_plan *P, ColArgs &ca) {
    ca.wave_map = P->wave_map;
    ca.wave_map4 = P->wave_map4;
    ca.out_map = P->out_map;
    ca.out_map4 = P->out_map4;
    ca.wave_map_ok = P->wave_map_ok ? 1 : 0;
    ca.tile_ctr = P->col_ctr;
    ca.err = P->dev_err;
}

extern "C" int prism_build_smatrix(prism_plan *P, const float *V_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    int rc;
    if ((rc = check_dev_ptr(V_dev, 16, "V_dev"))) return rc;
    return build_launches(P, V_dev);
}

// transmission, every slice's row and column passes, ROW_OUT (and the 16-bit quantiser) of every
// beam batch: kernel launches only (also captured into batch graphs).  per > 0: the transmission
// functions are made `per` slices at a time, each chunk after P->copy_done[chunk] (host-buffer
// builds); otherwise all slices in one launch.
static int build_launches(prism_plan *P, const float *V_dev, int per) {
    int rc;
    const prism_grid &g = P->g;
    const size_t px = (size_t)g.nx * g.ny;
    const double sigma_cycles = P->T.sigma / (2.0 * PI);
    const bool chunked = per > 0;
    if (!chunked) per = g.n_slices;
    for (int b0 = 0; b0 < P->nbeams; b0 += P->batch) {
        const int nb = std::min(P->batch, P->nbeams - b0);
        for (int p = 0; p < g.n_slices; ++p) {
            if (b0 == 0 && p % per == 0) {
                // transmission functions t_p = exp(i sigma V_p) of slices p ... p + per - 1
                if (chunked) CUDA_TRY(cudaStreamWaitEvent(P->stream, P->copy_done[p / per], 0));
                const int ns = std::min(per, g.n_slices - p);
                rc = plan_launch(P, PRISM_K_TRANSMIT, [&] {
                    return launch_transmission(V_dev + (size_t)p * px, P->t + (size_t)p * px, (size_t)ns * px, sigma_cycles, P->stream);
                });
                if (rc) return rc;
            }
            if (p == 0) {
                // first slice (shift theorem): T0 = FFT_x(t_0) once per build, every column -- the
                // first row pass of the (0, 0) beam -- then every beam's rows as T0 shifted by m f
                // columns times the y phase exp(2 pi i n f_y y / ny)
                if (b0 == 0) {
                    RowArgs r0 = row_args(P);
                    r0.wave = P->t0f;
                    r0.trans = P->t;
                    r0.n_rows = g.ny;
                    r0.beam_mn = P->zero_mn;
                    r0.beam0 = 0;
                    r0.kx_half = 0;
                    rc = plan_launch(P, PRISM_K_ROW_PLANE, [&] { return launch_row(g.nx, ROW_PLANE, r0, P->stream); });
                    if (rc) return rc;
                }
                rc = plan_launch(P, PRISM_K_PLANE, [&] {
                    return launch_plane(P->t0f, P->wave, P->beam_mn, b0, nb, g.nx, g.ny, g.f, P->fy, P->T.kx_half, P->stream);
                });
            } else {
                RowArgs ra = row_args(P);
                ra.trans = P->t + (size_t)p * px;
                ra.n_rows = nb * g.ny;
                ra.beam0 = b0;
                const int rs = P->tune_shape[0] >= 0 ? P->tune_shape[0] : row_default_shape(P);
                rc = plan_launch(P, PRISM_K_ROW, [&] {
                    return rs >= 0 ? launch_row_shape(g.nx, rs, ra, P->stream) : launch_row(g.nx, ROW_STD, ra, P->stream);
                });
            }
            if (rc) return rc;
            const int pi = P->T.slice_prop[p];
            ColArgs ca = col_args(P->T, P->wave, P->prop_x + (size_t)pi * g.nx, P->prop_y + (size_t)pi * g.ny,
                                  P->aa_kmax, P->twc_f, P->twc_i, P->tw64);
            ca.batch = nb;
            ca.kx_half = P->T.kx_half;
            ca.band4 = P->T.band4;
            col_wave_map(P, ca);
            const int cs = P->tune_shape[1] >= 0 ? P->tune_shape[1] : col_default_shape(P);
            rc = plan_launch(P, PRISM_K_COL, [&] {
                return cs >= 0 ? launch_col_shape(g.ny, cs, ca, P->stream) : launch_col(g.ny, COL_STD, ca, P->stream);
            });
            if (rc) return rc;
        }
        RowArgs ro = row_args(P);
        ro.n_rows = nb * (g.downsample == 2 ? g.ny / 2 : g.ny);
        ro.beam0 = P->prec == PRISM_PRECISION_FP32 ? b0 : 0;  // 16-bit mode: S holds this batch only
        rc = plan_launch(P, PRISM_K_ROW_OUT, [&] { return launch_row(g.nx, ROW_OUT, ro, P->stream); });
        if (rc) return rc;
        if (P->prec != PRISM_PRECISION_FP32) {
            QuantArgs q;
            q.S = P->S;
            q.S16 = P->S16;
            q.scale = P->scale;
            q.beam0 = b0;
            q.nb = nb;
            q.npix = P->nxs * P->nys;
            q.kp = P->kp;
            q.mode = tc_mode(P->prec);
            rc = plan_launch(P, PRISM_K_QUANT, [&] { return launch_quantize(q, P->stream); });
            if (rc) return rc;
        }
    }
    P->built = true;
    return PRISM_OK;
}

extern "C" int prism_build_smatrix_host(prism_plan *P, const float *V_host) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    if (!V_host) return fail(PRISM_ERR_INVALID, "V_host is NULL");
    const size_t bytes = (size_t)P->g.n_slices * P->g.nx * P->g.ny * sizeof(float);
    int rc = grow(P->arena, (void **)&P->v_stage, &P->v_cap, bytes);
    if (rc) return rc;
    // the potential in up to 8 chunks of slices on the copy stream, after every earlier use of the
    // staging buffer on the plan's stream
    const int H = P->g.n_slices, per = (H + 7) / 8, nch = (H + per - 1) / per;
    const size_t slice = (size_t)P->g.nx * P->g.ny;
    if (!P->copy) {
        CUDA_TRY(cudaStreamCreateWithFlags(&P->copy, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&P->copy_start, cudaEventDisableTiming));
    }
    while ((int)P->copy_done.size() < nch) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        P->copy_done.push_back(e);
    }
    CUDA_TRY(cudaEventRecord(P->copy_start, P->stream));
    CUDA_TRY(cudaStreamWaitEvent(P->copy, P->copy_start, 0));
    for (int c = 0; c < nch; ++c) {
        const size_t off = (size_t)c * per * slice, n = (size_t)std::min(per, H - c * per) * slice;
        CUDA_TRY(cudaMemcpyAsync(P->v_stage + off, V_host + off, n * sizeof(float), cudaMemcpyHostToDevice, P->copy));
        CUDA_TRY(cudaEventRecord(P->copy_done[c], P->copy));
    }
    return build_launches(P, P->v_stage, per);
}

// ------------------------------------------------------------------ scan
static int scan_prepare(prism_plan *P, const prism_probe *probe, const prism_scan *sc, const prism_detector *det,
                        ScanArgs &a, bool need_built = true) {
    int rc;
    if ((rc = check_probe(probe))) return rc;
    if (det && (rc = check_det(det))) return rc;
    const double pxs = P->g.cell_x / P->nxs, pys = P->g.cell_y / P->nys;
    if ((rc = check_scan(sc, pxs * (double)(1 << 28), pys * (double)(1 << 28)))) return rc;
    if (need_built && !P->built) return fail(PRISM_ERR_INVALID, "S-matrix not built");
    const int B = P->nbeams;
    const double lam = P->T.lam;
    const Tilt tl = tilt_terms(probe, lam, P->T.dz);
    // A(q_b - q_t) exp(-i chi(q_b - q_t)) and sum_b A_b
    std::vector<float2> base(B);
    double count = 0;
    for (int b = 0; b < B; ++b) {
        const double qx = (double)(P->bm[b] * P->g.f) / P->g.cell_x;
        const double qy = (double)(P->bn[b] * P->fy) / P->g.cell_y;
        const double dqx = qx - tl.qtx;
        const double dqy = qy - tl.qty;
        if (inside_aperture(dqx, dqy, lam, probe->alpha_mrad * 1e-3)) {
            base[b] = phase_cycles(chi_cycles(dqx * dqx + dqy * dqy, lam, probe->c1, probe->c3));
            count += 1.0;
        } else {
            base[b] = make_float2(0.f, 0.f);
        }
    }
    const long long Pn = (long long)sc->px * sc->py;
    if ((rc = grow(P->arena, (void **)&P->pos, &P->pos_cap, std::max<size_t>(16, (size_t)Pn * 2 * sizeof(double))))) return rc;
    if (Pn > 0) {
        // pageable copy of the caller's arrays: cudaMemcpyAsync stages pageable memory before it returns
        std::vector<double> xy((size_t)Pn * 2);
        std::memcpy(xy.data(), sc->x0, Pn * sizeof(double));
        std::memcpy(xy.data() + Pn, sc->y0, Pn * sizeof(double));
        CUDA_TRY(cudaMemcpyAsync(P->pos, xy.data(), xy.size() * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(P->base, base.data(), B * sizeof(float2), cudaMemcpyHostToDevice, P->stream));
    // window bin map (q = k f / cell on the window grid), cached per detector
    if (det && (P->det_nbins != det->nbins || P->det_key[0] != det->start_mrad || P->det_key[1] != det->step_mrad)) {
        std::vector<int> off, idx;
        detector_csr(P->nw, P->nwy, P->g.cell_x, P->g.cell_y, P->g.f, P->fy, lam, det, off, idx);
        // the lists again by rank within the bin, so that threads summing consecutive bins read
        // consecutive words
        int maxlen = 0;
        for (int k = 0; k < det->nbins; ++k) maxlen = std::max(maxlen, off[k + 1] - off[k]);
        std::vector<int> idx_t((size_t)maxlen * det->nbins, 0);
        for (int k = 0; k < det->nbins; ++k)
            for (int i = 0; i < off[k + 1] - off[k]; ++i) idx_t[(size_t)i * det->nbins + k] = idx[off[k] + i];
        P->bin_t_off = off.size() + idx.size();
        std::vector<int> all(off);
        all.insert(all.end(), idx.begin(), idx.end());
        all.insert(all.end(), idx_t.begin(), idx_t.end());
        // the lists once more as 16-bit entries (window pixels < 2^16), from a 16-byte boundary and
        // padded to 16 bytes, for the scans that stage them in shared memory
        while (all.size() % 4) all.push_back(0);
        P->bin_16_off = all.size();
        P->bin_n = idx.size();
        std::vector<uint16_t> i16((idx.size() + 7) / 8 * 8, 0);
        for (size_t i = 0; i < idx.size(); ++i) i16[i] = (uint16_t)idx[i];
        const size_t w16 = i16.size() / 2;
        all.resize(all.size() + w16);
        std::memcpy(all.data() + P->bin_16_off, i16.data(), i16.size() * sizeof(uint16_t));
        if ((rc = grow(P->arena, (void **)&P->bin_buf, &P->bin_cap, all.size() * sizeof(int)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(P->bin_buf, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, P->stream));
        P->det_nbins = det->nbins;
        P->det_key[0] = det->start_mrad;
        P->det_key[1] = det->step_mrad;
    }
    std::memset(&a, 0, sizeof(a));
    a.S = P->S;
    a.x0 = P->pos;
    a.y0 = P->pos + Pn;
    a.qx = P->beam_q;
    a.qy = P->beam_q + B;
    a.base = P->base;
    a.tw_fwd = P->tww_f;
    a.tw_fwd_y = P->tww_fy;
    a.bin_off = det ? P->bin_buf : nullptr;
    a.bin_idx = det ? P->bin_buf + det->nbins + 1 : nullptr;
    a.bin_idx_t = det ? P->bin_buf + P->bin_t_off : nullptr;
    a.bin_idx16 = det ? reinterpret_cast<const uint16_t *>(P->bin_buf + P->bin_16_off) : nullptr;
    a.n_bin_idx = det ? (int)P->bin_n : 0;
    a.px_s = pxs;
    a.py_s = pys;
    a.shift_x = tl.sx;
    a.shift_y = tl.sy;
    const double nw2 = (double)P->nw * (double)P->nwy;
    a.inv_norm = count > 0 ? 1.0 / (nw2 * nw2 * count) : 0.0;
    a.n_beams = B;
    a.nx_s = P->nxs;
    a.ny_s = P->nys;
    a.nbins = det ? det->nbins : 0;
    a.n_probes = (int)Pn;
    a.probe0 = 0;
    a.S16 = P->S16;
    a.beam_scale = P->scale;
    a.kp = P->kp;
    a.scan_px = sc->px;
    a.scan_py = sc->py;
    a.err = P->dev_err;
    a.tw = P->tw64;
    return PRISM_OK;
}

// the scan's counters (completion counters of the blocks it splits over idle CTAs, int[grid], then its
// work-unit counters, int[2]), zeroed when allocated; every launch leaves them at zero
static int split_counters(prism_plan *P, ScanArgs &a, int grid) {
    const size_t cb = scan_gemm_cnt_bytes(grid);
    const bool fresh = !P->win_cnt || cb > P->cnt_cap;
    int rc = grow(P->arena, (void **)&P->win_cnt, &P->cnt_cap, cb);
    if (rc) return rc;
    if (fresh) CUDA_TRY(cudaMemsetAsync(P->win_cnt, 0, P->cnt_cap, P->stream));
    a.win = P->win;
    a.win_cnt = P->win_cnt;
    return PRISM_OK;
}

// FP32 mode: the CUDA-core scan kernels; 16-bit mode: the tensor-core kernel (persistent grid, its
// window scratch grown on demand)
// FP32: the GEMM scan over 8 x 4 raster blocks when its shared memory fits (grid > 0), else the
// grouped / per-probe kernels (grid 0); 16-bit: the tensor-core scan
// the GEMM scan's contraction shape in use: the tuned or pinned one where it is compiled for the
// plan's window, else the default
static int gemm_shape(const prism_plan *P) {
    return P->scan_shape > 0 && scan_gemm_shape_valid(P->nw, P->nwy, P->scan_shape) ? P->scan_shape : 0;
}

// the tensor-core scan's ring shape in use: the tuned or pinned one, else the default
static int tc_shape(const prism_plan *P) {
    return P->tc_shape > 0 && P->tc_shape < scan_tc_shapes(tc_mode(P->prec)) ? P->tc_shape : 0;
}

static int scan_setup(prism_plan *P, ScanArgs &a, int *grid) {
    *grid = 0;
    if (P->prec == PRISM_PRECISION_FP32) {
        const int sh = gemm_shape(P);
        *grid = scan_gemm_grid(P->nw, P->nwy, sh, P->nbeams, a.scan_px, a.scan_py);
        if (*grid <= 0) {
            *grid = 0;
            return PRISM_OK;
        }
        const size_t wb = scan_gemm_win_bytes(P->nw, P->nwy, sh, *grid, a.scan_px, a.scan_py);
        if (!wb) return fail(PRISM_ERR_CUDA, "FP32 scan: no window scratch size for contraction shape " + std::to_string(sh));
        int rc = grow(P->arena, (void **)&P->win, &P->win_cap, wb);
        if (rc) return rc;
        return split_counters(P, a, *grid);
    }
    *grid = scan_tc_grid(P->nw, P->kp, tc_mode(P->prec), tc_shape(P), a.scan_px, a.scan_py);
    if (*grid <= 0) return fail(PRISM_ERR_CUDA, "tensor-core scan: no resident launch configuration");
    int rc = grow(P->arena, (void **)&P->win, &P->win_cap, scan_tc_win_bytes(P->nw, *grid, a.scan_px, a.scan_py));
    if (rc) return rc;
    return split_counters(P, a, *grid);
}

static int scan_go(prism_plan *P, const ScanArgs &a, int grid) {
    if (P->prec == PRISM_PRECISION_FP32)
        return plan_launch(P, PRISM_K_SCAN, [&] {
            return grid > 0 ? launch_scan_gemm(P->nw, P->nwy, gemm_shape(P), grid, a, P->stream)
                            : launch_scan_rect(P->nw, P->nwy, a, P->stream);
        });
    return plan_launch(P, PRISM_K_SCAN, [&] { return launch_scan_tc(P->nw, tc_mode(P->prec), tc_shape(P), grid, a, P->stream); });
}

static int scan_launch(prism_plan *P, ScanArgs &a) {
    int grid = 0;
    int rc = scan_setup(P, a, &grid);
    if (rc) return rc;
    return scan_go(P, a, grid);
}

extern "C" int prism_scan_run(prism_plan *P, const prism_probe *probe, const prism_scan *sc,
                              const prism_detector *det, float *out_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    ScanArgs a;
    int rc = scan_prepare(P, probe, sc, det, a);
    if (rc) return rc;
    if (a.n_probes == 0) return PRISM_OK;
    if ((rc = check_dev_ptr(out_dev, 4, "out_dev"))) return rc;
    a.out = out_dev;
    return scan_launch(P, a);
}

extern "C" int prism_scan_run_host(prism_plan *P, const prism_probe *probe, const prism_scan *sc,
                                   const prism_detector *det, float *out_host) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    ScanArgs a;
    int rc = scan_prepare(P, probe, sc, det, a);
    if (rc) return rc;
    if (a.n_probes == 0) return PRISM_OK;
    if (!out_host) return fail(PRISM_ERR_INVALID, "out_host is NULL");
    const size_t bytes = (size_t)a.n_probes * det->nbins * sizeof(float);
    if ((rc = grow(P->arena, (void **)&P->out_stage, &P->out_cap, bytes))) return rc;
    a.out = P->out_stage;
    rc = scan_launch(P, a);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(out_host, P->out_stage, bytes, cudaMemcpyDeviceToHost, P->stream));
    return PRISM_OK;
}

extern "C" int prism_scan_run_cbed(prism_plan *P, const prism_probe *probe, const prism_scan *sc, float *out_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    ScanArgs a;
    int rc = scan_prepare(P, probe, sc, nullptr, a);
    if (rc) return rc;
    if (a.n_probes == 0) return PRISM_OK;
    if ((rc = check_dev_ptr(out_dev, 4, "out_dev"))) return rc;
    a.out = nullptr;
    a.cbed = out_dev;
    return scan_launch(P, a);
}

extern "C" int prism_scan_run_accumulate(prism_plan *P, const prism_probe *probe, const prism_scan *sc,
                                         const prism_detector *det, float weight, float *out_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    if (!std::isfinite(weight)) return fail(PRISM_ERR_INVALID, "weight must be finite");
    ScanArgs a;
    int rc = scan_prepare(P, probe, sc, det, a);
    if (rc) return rc;
    if (a.n_probes == 0) return PRISM_OK;
    if ((rc = check_dev_ptr(out_dev, 4, "out_dev"))) return rc;
    a.out = out_dev;
    a.accumulate = 1;
    a.acc_w = weight;
    return scan_launch(P, a);
}

// ------------------------------------------------------------------ multislice baseline
// The row passes may skip the columns the anti-aliasing aperture zeroes (|kx| >= kx_half) only if
// the initial probe is zero there too: a probe aperture wider than the anti-aliasing aperture keeps
// every column (returns 0).
static int probe_kx_half(int kx_half, const std::vector<float2> &pbase, int nx, int ny) {
    for (int ky = 0; ky < ny && kx_half; ++ky)
        for (int kx = kx_half; kx <= nx - kx_half; ++kx) {
            const float2 v = pbase[(size_t)ky * nx + kx];
            if (v.x != 0.f || v.y != 0.f) return 0;
        }
    return kx_half;
}

extern "C" int multislice_scan_run(const prism_grid *grid, const float *V_dev, const prism_probe *probe,
                                   const prism_scan *sc, const prism_detector *det, float *out_dev,
                                   void *cuda_stream, size_t scratch_bytes) {
    int rc;
    if ((rc = check_grid_common(grid))) return rc;
    if ((rc = check_probe(probe))) return rc;
    if ((rc = check_det(det))) return rc;
    const prism_grid &g = *grid;
    if ((rc = check_scan(sc, g.cell_x / g.nx * (double)(1 << 28), g.cell_y / g.ny * (double)(1 << 28)))) return rc;
    const long long Pn = (long long)sc->px * sc->py;
    if (Pn == 0) return PRISM_OK;
    if ((rc = check_dev_ptr(V_dev, 16, "V_dev"))) return rc;
    if ((rc = check_dev_ptr(out_dev, 4, "out_dev"))) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GridTables T;
    if ((rc = build_grid_tables(&g, T))) return rc;
    const int nx = g.nx, ny = g.ny;
    const size_t px = (size_t)nx * ny;
    // probe A(q - q_t) exp(-i chi(q - q_t)) on the full grid, sum |Psi0|^2 = aperture pixel count
    const Tilt tl = tilt_terms(probe, T.lam, T.dz);
    std::vector<float2> pbase(px);
    double count = 0;
    for (int ky = 0; ky < ny; ++ky) {
        const double qy = (double)signed_index(ky, ny) / g.cell_y;
        for (int kx = 0; kx < nx; ++kx) {
            const double qx = (double)signed_index(kx, nx) / g.cell_x;
            const double dqx = qx - tl.qtx;
            const double dqy = qy - tl.qty;
            if (inside_aperture(dqx, dqy, T.lam, probe->alpha_mrad * 1e-3)) {
                pbase[(size_t)ky * nx + kx] = phase_cycles(chi_cycles(dqx * dqx + dqy * dqy, T.lam, probe->c1, probe->c3));
                count += 1.0;
            } else {
                pbase[(size_t)ky * nx + kx] = make_float2(0.f, 0.f);
            }
        }
    }
    const int kx_half = probe_kx_half(T.kx_half, pbase, nx, ny);
    std::vector<int> off, idx;
    detector_csr(nx, ny, g.cell_x, g.cell_y, 1, 1, T.lam, det, off, idx);
    if (scratch_bytes == 0) scratch_bytes = (size_t)1 << 30;
    const int Pb = (int)std::max<long long>(1, std::min<long long>(Pn, (long long)(scratch_bytes / (px * 8))));
    const Tw64 tw = make_tw64();

    DevArena A;
    A.stream = st;
    float2 *t, *wave, *prop_x, *prop_y, *twr_f, *twr_i, *twc_f, *twc_i, *pb, *shx, *shy;
    float *inten;
    int *aa, *d_off, *d_idx;
    double *pos;
    auto done = [&](int code) {
        A.release();
        if (code) cudaStreamSynchronize(st);
        return code;
    };
    if ((rc = A.alloc((void **)&t, (size_t)g.n_slices * px * 8))) return done(rc);
    if ((rc = A.alloc((void **)&wave, (size_t)Pb * px * 8))) return done(rc);
    if ((rc = A.alloc((void **)&inten, (size_t)Pb * px * 4))) return done(rc);
    if ((rc = A.alloc((void **)&shx, (size_t)Pb * nx * 8))) return done(rc);
    if ((rc = A.alloc((void **)&shy, (size_t)Pb * ny * 8))) return done(rc);
    if ((rc = A.upload(&prop_x, T.prop_x))) return done(rc);
    if ((rc = A.upload(&prop_y, T.prop_y))) return done(rc);
    if ((rc = A.upload(&aa, T.aa_kmax))) return done(rc);
    if ((rc = A.upload(&twr_f, T.twr_f))) return done(rc);
    if ((rc = A.upload(&twr_i, T.twr_i))) return done(rc);
    if ((rc = A.upload(&twc_f, T.twc_f))) return done(rc);
    if ((rc = A.upload(&twc_i, T.twc_i))) return done(rc);
    if ((rc = A.upload(&pb, pbase))) return done(rc);
    if ((rc = A.upload(&d_off, off))) return done(rc);
    if ((rc = A.upload(&d_idx, idx))) return done(rc);
    if ((rc = A.alloc((void **)&pos, (size_t)Pn * 2 * sizeof(double)))) return done(rc);
    // the column passes between slices as in a plan's build: at 1024^2 the TMA-staged shape (tiles
    // loaded and stored by TMA through tensor maps of this call's wave buffer); their bounded waits
    // report to an error word that turns the affected bins into NaN
    int *err = nullptr;
    if ((rc = A.alloc((void **)&err, 16))) return done(rc);
    {
        const cudaError_t e = cudaMemsetAsync(err, 0, 16, st);
        if (e != cudaSuccess) {
            fail(PRISM_ERR_CUDA, std::string("error word: ") + cudaGetErrorString(e));
            return done(PRISM_ERR_CUDA);
        }
    }
    CUtensorMap map8, map4, out8, out4;
    const int col_tma = ny == 1024 ? tune_col_tma_shape(4) : -1;
    const bool maps_ok =
        col_tma >= 0 && tune_shape_valid(PRISM_TUNE_COL, ny, col_tma) && encode_wave_maps(map8, map4, out8, out4, wave, nx, ny, Pb);
    {
        // the probe phase uses r0 - h tan(theta) (zero without tilt)
        std::vector<double> xy((size_t)Pn * 2);
        for (long long i = 0; i < Pn; ++i) {
            xy[i] = sc->x0[i] - tl.sx;
            xy[Pn + i] = sc->y0[i] - tl.sy;
        }
        cudaError_t e = cudaMemcpyAsync(pos, xy.data(), xy.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            fail(PRISM_ERR_CUDA, std::string("position upload: ") + cudaGetErrorString(e));
            return done(PRISM_ERR_CUDA);
        }
    }
    auto check = [&](cudaError_t err, const char *what) {
        if (err != cudaSuccess) return fail(PRISM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
        return PRISM_OK;
    };
    if ((rc = check(launch_transmission(V_dev, t, (size_t)g.n_slices * px, T.sigma / (2.0 * PI), st), "transmission"))) return done(rc);
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
        sa.cell_x = g.cell_x;
        sa.cell_y = g.cell_y;
        if ((rc = check(launch_shift(sa, st), "shift phases"))) return done(rc);
        ColArgs ci = col_args(T, wave, prop_x, prop_y, aa, twc_f, twc_i, tw);
        ci.batch = nb;
        ci.probe_base = pb;
        ci.shift_x = shx;
        ci.shift_y = shy;
        ci.probe_scale = (float)(1.0 / ((double)nx * ny));
        if ((rc = check(launch_col(ny, COL_PROBE, ci, st), "probe init"))) return done(rc);
        for (int p = 0; p < g.n_slices; ++p) {
            RowArgs ra;
            std::memset(&ra, 0, sizeof(ra));
            ra.wave = wave;
            ra.trans = t + (size_t)p * px;
            ra.tw_fwd = twr_f;
            ra.tw_inv = twr_i;
            ra.ny = ny;
            ra.n_rows = nb * ny;
            ra.kx_half = kx_half;  // every row pass reads a wave band-limited in x (aperture and probe)
            ra.tw = tw;
            if ((rc = check(launch_row_std(nx, ra, st), "row pass"))) return done(rc);
            const int pi = T.slice_prop[p];
            ColArgs ca = col_args(T, wave, prop_x + (size_t)pi * nx, prop_y + (size_t)pi * ny, aa, twc_f, twc_i, tw);
            ca.batch = nb;
            ca.inten = inten;
            // the detecting pass reads every column (the initial probe left exact zeros in the
            // columns the row passes skip) and writes every intensity
            ca.kx_half = p + 1 == g.n_slices ? 0 : kx_half;
            ca.band4 = T.band4;
            if (p + 1 < g.n_slices && maps_ok) {
                ca.wave_map = map8;
                ca.wave_map4 = map4;
                ca.out_map = out8;
                ca.out_map4 = out4;
                ca.wave_map_ok = 1;
                ca.err = err;
                if ((rc = check(launch_col_shape(ny, col_tma, ca, st), "column pass"))) return done(rc);
            } else if ((rc = check(launch_col(ny, p + 1 == g.n_slices ? COL_DETECT : COL_STD, ca, st), "column pass"))) {
                return done(rc);
            }
        }
        BinArgs ba;
        ba.inten = inten;
        ba.bin_off = d_off;
        ba.bin_idx = d_idx;
        ba.out = out_dev + (size_t)p0 * det->nbins;
        const double nn = (double)nx * ny;
        ba.scale = count > 0 ? nn * nn / count : 0.0;
        ba.npix = (int)px;
        ba.nbins = det->nbins;
        ba.batch = nb;
        ba.err = err;
        if ((rc = check(launch_bins(ba, st), "bins"))) return done(rc);
    }
    // pageable uploads were staged before their calls returned; the frees below are stream-ordered
    return done(PRISM_OK);
}

// ------------------------------------------------------------------ introspection
extern "C" int prism_plan_info(const prism_plan *P, prism_info *out) {
    if (!P || !out) return fail(PRISM_ERR_INVALID, "NULL argument");
    out->n_beams = P->nbeams;
    out->nx_s = P->nxs;
    out->ny_s = P->nys;
    out->nw_x = P->nw;
    out->nw_y = P->nwy;
    out->beam_batch = P->batch;
    out->wavelength = P->T.lam;
    out->sigma = P->T.sigma;
    out->device_bytes = P->arena.bytes;
    return PRISM_OK;
}

extern "C" int prism_plan_smatrix_bytes(const prism_plan *P, size_t *out) {
    if (!P || !out) return fail(PRISM_ERR_INVALID, "NULL argument");
    *out = P->prec == PRISM_PRECISION_FP32 ? (size_t)P->nbeams * P->nxs * P->nys * 8
                                            : (size_t)P->nxs * P->nys * P->kp * 2 * tc_parts(P->prec) + (size_t)P->kp / 2 * sizeof(float);
    return PRISM_OK;
}

extern "C" int prism_plan_beams(const prism_plan *P, int *m, int *n, int capacity) {
    if (!P || !m || !n) return fail(PRISM_ERR_INVALID, "NULL argument");
    if (capacity < P->nbeams) return fail(PRISM_ERR_INVALID, "capacity < n_beams");
    for (int b = 0; b < P->nbeams; ++b) {
        m[b] = P->bm[b];
        n[b] = P->bn[b];
    }
    return PRISM_OK;
}

extern "C" int prism_plan_smatrix(const prism_plan *P, const void **dev_ptr) {
    if (!P || !dev_ptr) return fail(PRISM_ERR_INVALID, "NULL argument");
    if (P->prec != PRISM_PRECISION_FP32) return fail(PRISM_ERR_INVALID, "S is stored in 16-bit parts: use prism_plan_smatrix_copy");
    *dev_ptr = P->S;
    return PRISM_OK;
}

extern "C" int prism_plan_smatrix_copy(prism_plan *P, float *out_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    int rc;
    if ((rc = check_dev_ptr(out_dev, 8, "out_dev"))) return rc;
    if (!P->built) return fail(PRISM_ERR_INVALID, "S-matrix not built");
    const size_t npix = (size_t)P->nxs * P->nys;
    if (P->prec == PRISM_PRECISION_FP32) {
        CUDA_TRY(cudaMemcpyAsync(out_dev, P->S, (size_t)P->nbeams * npix * 8, cudaMemcpyDeviceToDevice, P->stream));
        return PRISM_OK;
    }
    cudaError_t e = launch_dequantize(P->S16, P->scale, (float2 *)out_dev, P->nbeams, (int)npix, P->kp,
                                      tc_mode(P->prec), P->stream);
    if (e != cudaSuccess) return fail(PRISM_ERR_CUDA, std::string("dequantize: ") + cudaGetErrorString(e));
    return PRISM_OK;
}

extern "C" int prism_plan_load_smatrix(prism_plan *P, const float *S_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    int rc;
    if ((rc = check_dev_ptr(S_dev, 8, "S_dev"))) return rc;
    const size_t sbeam = (size_t)P->nxs * P->nys * sizeof(float2);
    if (P->prec == PRISM_PRECISION_FP32) {
        CUDA_TRY(cudaMemcpyAsync(P->S, S_dev, (size_t)P->nbeams * sbeam, cudaMemcpyDeviceToDevice, P->stream));
    } else {
        // the FP32 beam-batch buffer takes each batch in turn; the quantiser writes its 16-bit rows
        for (int b0 = 0; b0 < P->nbeams; b0 += P->batch) {
            const int nb = std::min(P->batch, P->nbeams - b0);
            CUDA_TRY(cudaMemcpyAsync(P->S, reinterpret_cast<const char *>(S_dev) + (size_t)b0 * sbeam, (size_t)nb * sbeam,
                                     cudaMemcpyDeviceToDevice, P->stream));
            QuantArgs q;
            q.S = P->S;
            q.S16 = P->S16;
            q.scale = P->scale;
            q.beam0 = b0;
            q.nb = nb;
            q.npix = P->nxs * P->nys;
            q.kp = P->kp;
            q.mode = tc_mode(P->prec);
            if ((rc = plan_launch(P, PRISM_K_QUANT, [&] { return launch_quantize(q, P->stream); }))) return rc;
        }
    }
    P->built = true;
    return PRISM_OK;
}

extern "C" int prism_plan_transmission(const prism_plan *P, const void **dev_ptr) {
    if (!P || !dev_ptr) return fail(PRISM_ERR_INVALID, "NULL argument");
    *dev_ptr = P->t;
    return PRISM_OK;
}

extern "C" int prism_selftest_bounded_wait(int *status_dev, long long limit_cycles, int arrive, void *cuda_stream) {
    int rc;
    if ((rc = check_dev_ptr(status_dev, 4, "status_dev"))) return rc;
    if (limit_cycles < 0 || limit_cycles > 4000000000LL) return fail(PRISM_ERR_INVALID, "limit_cycles must be in [0, 4e9]");
    cudaError_t e = launch_wait_selftest(status_dev, limit_cycles, arrive, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(PRISM_ERR_CUDA, std::string("bounded-wait self-test launch: ") + cudaGetErrorString(e));
    return PRISM_OK;
}

extern "C" int prism_selftest_tcgen05(float *out_dev, int *status_dev, void *cuda_stream) {
    int rc;
    if ((rc = check_dev_ptr(out_dev, 16, "out_dev"))) return rc;
    if ((rc = check_dev_ptr(status_dev, 4, "status_dev"))) return rc;
    cudaError_t e = launch_tc_selftest(out_dev, status_dev, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(PRISM_ERR_CUDA, std::string("tcgen05 self-test launch: ") + cudaGetErrorString(e));
    return PRISM_OK;
}

// ------------------------------------------------------------------ timing
static const char *k_names[PRISM_K_COUNT] = {"transmission", "row_plane", "row", "col", "row_out", "scan", "quantize", "plane"};

extern "C" const char *prism_kernel_name(int kind) {
    if (kind < 0 || kind >= PRISM_K_COUNT) return "?";
    return k_names[kind];
}

extern "C" int prism_plan_set_profiling(prism_plan *P, int enable) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    P->profiling = enable != 0;
    return PRISM_OK;
}

static int drain_events(prism_plan *P) {
    if (P->pending.empty()) return PRISM_OK;
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    for (auto &pe : P->pending) {
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, pe.a, pe.b));
        P->kms[pe.kind] += ms;
        P->ev_pool.push_back(pe.a);
        P->ev_pool.push_back(pe.b);
    }
    P->pending.clear();
    return PRISM_OK;
}

extern "C" int prism_plan_kernel_stats(prism_plan *P, int kind, long *launches, double *total_ms) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    if (kind < 0 || kind >= PRISM_K_COUNT) return fail(PRISM_ERR_INVALID, "bad kernel kind");
    int rc = drain_events(P);
    if (rc) return rc;
    if (launches) *launches = P->kl[kind];
    if (total_ms) *total_ms = P->kms[kind];
    return PRISM_OK;
}

extern "C" long prism_plan_launches(const prism_plan *P) { return P ? P->launches : 0; }

extern "C" int prism_plan_reset_stats(prism_plan *P) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    int rc = drain_events(P);
    if (rc) return rc;
    for (int k = 0; k < PRISM_K_COUNT; ++k) {
        P->kms[k] = 0;
        P->kl[k] = 0;
    }
    P->launches = 0;
    return PRISM_OK;
}

// ------------------------------------------------------------------ helpers for the fixed-scratch entry point
namespace prism {

int internal_fail(int code, const char *msg) { return fail(code, msg); }

int internal_check_dev_ptr(const void *p, size_t align, const char *what) { return check_dev_ptr(p, align, what); }

int internal_multislice_tables(const prism_grid *grid, const prism_probe *probe, const prism_scan *sc,
                               const prism_detector *det, MsHostTables *out) {
    int rc;
    if ((rc = check_grid_common(grid))) return rc;
    if ((rc = check_probe(probe))) return rc;
    if ((rc = check_det(det))) return rc;
    const prism_grid &g = *grid;
    if ((rc = check_scan(sc, g.cell_x / g.nx * (double)(1 << 28), g.cell_y / g.ny * (double)(1 << 28)))) return rc;
    GridTables T;
    if ((rc = build_grid_tables(&g, T))) return rc;
    MsHostTables &M = *out;
    M.nx = g.nx;
    M.ny = g.ny;
    M.H = g.n_slices;
    M.lam = T.lam;
    M.sigma = T.sigma;
    M.slice_prop = T.slice_prop;
    M.prop_x = T.prop_x;
    M.prop_y = T.prop_y;
    M.aa_kmax = T.aa_kmax;
    M.twr_f = T.twr_f;
    M.twr_i = T.twr_i;
    M.twc_f = T.twc_f;
    M.twc_i = T.twc_i;
    const size_t px = (size_t)g.nx * g.ny;
    const Tilt tl = tilt_terms(probe, T.lam, T.dz);
    M.pbase.assign(px, make_float2(0.f, 0.f));
    M.count = 0;
    for (int ky = 0; ky < g.ny; ++ky) {
        const double qy = (double)signed_index(ky, g.ny) / g.cell_y;
        for (int kx = 0; kx < g.nx; ++kx) {
            const double qx = (double)signed_index(kx, g.nx) / g.cell_x;
            const double dqx = qx - tl.qtx;
            const double dqy = qy - tl.qty;
            if (inside_aperture(dqx, dqy, T.lam, probe->alpha_mrad * 1e-3)) {
                M.pbase[(size_t)ky * g.nx + kx] = phase_cycles(chi_cycles(dqx * dqx + dqy * dqy, T.lam, probe->c1, probe->c3));
                M.count += 1.0;
            }
        }
    }
    M.kx_half = probe_kx_half(T.kx_half, M.pbase, g.nx, g.ny);
    M.band4 = T.band4;
    detector_csr(g.nx, g.ny, g.cell_x, g.cell_y, 1, 1, T.lam, det, M.bin_off, M.bin_idx);
    const long long Pn = (long long)sc->px * sc->py;
    M.pos.resize((size_t)Pn * 2);
    for (long long i = 0; i < Pn; ++i) {
        M.pos[i] = sc->x0[i] - tl.sx;
        M.pos[Pn + i] = sc->y0[i] - tl.sy;
    }
    M.tw = make_tw64();
    return PRISM_OK;
}

}  // namespace prism

// ------------------------------------------------------------------ autotuner
struct TuneKey {
    int kind, n, batch;
    bool shared;  // tuned for a batch whose branches share the SMs
    bool radix;   // the FFT radix variants were candidates
    bool operator<(const TuneKey &o) const {
        return kind != o.kind     ? kind < o.kind
               : n != o.n         ? n < o.n
               : batch != o.batch ? batch < o.batch
               : shared != o.shared ? shared < o.shared
                                    : radix < o.radix;
    }
};
struct TuneVal {
    int chosen;
    double ms[PRISM_TUNE_MAX_SHAPES];
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune_cache;

extern "C" int prism_plan_set_tune_shape(prism_plan *P, int kind, int shape) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    if (kind == PRISM_TUNE_SCAN) {
        if (shape >= 0 && (P->prec != PRISM_PRECISION_FP32 || shape >= scan_gemm_shapes() || !scan_gemm_shape_valid(P->nw, P->nwy, shape)))
            return fail(PRISM_ERR_UNSUPPORTED, std::string("contraction shape ") + std::to_string(shape) + " is not compiled for this plan's "
                                                   "scan (FP32 GEMM scan, square windows of 16, 32 or 64 pixels)");
        P->scan_shape = shape < 0 ? 0 : shape;
        return PRISM_OK;
    }
    if (kind == PRISM_TUNE_SCAN_TC) {
        if (shape >= 0 && (P->prec == PRISM_PRECISION_FP32 || shape >= scan_tc_shapes(tc_mode(P->prec))))
            return fail(PRISM_ERR_UNSUPPORTED, std::string("ring shape ") + std::to_string(shape) +
                                                   " is not compiled for this plan's scan (tensor-core scan of a 16-bit plan; split mode has one)");
        P->tc_shape = shape < 0 ? 0 : shape;
        return PRISM_OK;
    }
    if (kind != PRISM_TUNE_ROW && kind != PRISM_TUNE_COL)
        return fail(PRISM_ERR_INVALID, "kind must be PRISM_TUNE_ROW, PRISM_TUNE_COL, PRISM_TUNE_SCAN or PRISM_TUNE_SCAN_TC");
    if (shape >= 0) {
        const int n = kind == PRISM_TUNE_ROW ? P->g.nx : P->g.ny;
        if (shape >= tune_shapes(kind) || !tune_shape_valid(kind, n, shape))
            return fail(PRISM_ERR_UNSUPPORTED, std::string("launch shape ") + std::to_string(shape) + " is not compiled for N = " + std::to_string(n));
        if (tune_shape_needs_map(kind, shape) && !P->wave_map_ok)
            return fail(PRISM_ERR_UNSUPPORTED, "the plan holds no tensor map of its wave scratch (TMA-staged shape)");
    }
    P->tune_shape[kind] = shape < 0 ? -1 : shape;
    return PRISM_OK;
}

extern "C" int prism_plan_autotune(prism_plan *P) { return prism_plan_autotune_flags(P, 0); }

extern "C" int prism_plan_autotune_flags(prism_plan *P, int flags) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    if (flags & ~PRISM_AUTOTUNE_FFT_RADIX) return fail(PRISM_ERR_INVALID, "unknown autotune flags");
    const bool radix = (flags & PRISM_AUTOTUNE_FFT_RADIX) != 0;
    const prism_grid &g = P->g;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    int rc = PRISM_OK;
    for (int kind = 0; kind < 2 && !rc; ++kind) {
        const int n = kind == 0 ? g.nx : g.ny;
        const TuneKey key{kind, n, P->batch, P->shared_sms, radix};
        for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) P->tune_ms[kind][v] = -1.0;
        P->tuned[kind] = true;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                P->tune_shape[kind] = it->second.chosen;
                for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) P->tune_ms[kind][v] = it->second.ms[v];
                continue;
            }
        }
        int best = -1;
        double best_ms = 0;
        for (int v = 0; v < tune_shapes(kind) && v < PRISM_TUNE_MAX_SHAPES && !rc; ++v) {
            if (!tune_shape_valid(kind, n, v) || (tune_shape_needs_map(kind, v) && !P->wave_map_ok) ||
                (P->shared_sms && tune_shape_fills_sm(kind, v)) ||
                (!radix && tune_shape_fft_variant(kind, v) != tune_default_fft_variant(n)))
                continue;
            RowArgs ra = row_args(P);
            ra.trans = P->t;
            ra.n_rows = P->batch * g.ny;
            ColArgs ca = col_args(P->T, P->wave, P->prop_x, P->prop_y, P->aa_kmax, P->twc_f, P->twc_i, P->tw64);
            ca.batch = P->batch;
            ca.kx_half = P->T.kx_half;
            ca.band4 = P->T.band4;
            col_wave_map(P, ca);
            auto once = [&]() {
                return kind == 0 ? launch_row_shape(g.nx, v, ra, P->stream) : launch_col_shape(g.ny, v, ca, P->stream);
            };
            cudaError_t e = cudaSuccess;
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = once();
            if (e == cudaSuccess) e = cudaEventRecord(e0, P->stream);
            for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = once();
            if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                rc = fail(PRISM_ERR_CUDA, std::string("autotune ") + tune_shape_name(kind, v) + ": " + cudaGetErrorString(e));
                break;
            }
            P->tune_ms[kind][v] = ms / 5.0;
            if (best < 0 || ms / 5.0 < best_ms) {
                best = v;
                best_ms = ms / 5.0;
            }
        }
        if (rc) break;
        P->tune_shape[kind] = best;
        TuneVal tv;
        tv.chosen = best;
        for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) tv.ms[v] = P->tune_ms[kind][v];
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = tv;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" int prism_plan_tune_result(const prism_plan *P, int kind, prism_tune_entry *out) {
    if (!P || !out) return fail(PRISM_ERR_INVALID, "NULL argument");
    if (kind == PRISM_TUNE_SCAN) {
        const bool gemm = P->prec == PRISM_PRECISION_FP32;
        out->n_shapes = gemm ? std::min(scan_gemm_shapes(), PRISM_TUNE_MAX_SHAPES) : 0;
        out->chosen = gemm ? gemm_shape(P) : -1;
        out->default_shape = gemm ? 0 : -1;
        for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) out->ms[v] = P->scan_tuned ? P->scan_ms[v] : -1.0;
        return PRISM_OK;
    }
    if (kind == PRISM_TUNE_SCAN_TC) {
        const bool tc = P->prec != PRISM_PRECISION_FP32;
        out->n_shapes = tc ? std::min(scan_tc_shapes(tc_mode(P->prec)), PRISM_TUNE_MAX_SHAPES) : 0;
        out->chosen = tc ? tc_shape(P) : -1;
        out->default_shape = tc ? 0 : -1;
        for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) out->ms[v] = P->tc_tuned ? P->tc_ms[v] : -1.0;
        return PRISM_OK;
    }
    if (kind != PRISM_TUNE_ROW && kind != PRISM_TUNE_COL) return fail(PRISM_ERR_INVALID, "bad tune kind");
    const int n = kind == 0 ? P->g.nx : P->g.ny;
    out->n_shapes = std::min(tune_shapes(kind), PRISM_TUNE_MAX_SHAPES);
    out->chosen = P->tune_shape[kind];
    const int dc = kind == PRISM_TUNE_COL ? col_default_shape(P) : row_default_shape(P);
    out->default_shape = dc >= 0 ? dc : tune_shape_valid(kind, n, tune_default_shape(kind, n)) ? tune_default_shape(kind, n) : -1;
    for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) out->ms[v] = P->tuned[kind] ? P->tune_ms[kind][v] : -1.0;
    return PRISM_OK;
}

extern "C" const char *prism_tune_shape_name(int kind, int shape) {
    return kind == PRISM_TUNE_SCAN      ? scan_gemm_shape_name(shape)
           : kind == PRISM_TUNE_SCAN_TC ? scan_tc_shape_name(shape)
                                        : tune_shape_name(kind, shape);
}

extern "C" int prism_tune_shape_fft_variant(int kind, int shape) {
    return kind == PRISM_TUNE_ROW || kind == PRISM_TUNE_COL ? tune_shape_fft_variant(kind, shape) : -1;
}

// 16-bit plans: time the caller's scan with each ring shape of the tensor-core scan (a warm-up and
// two timed launches each) and keep the fastest; every shape gives bitwise the same stack, which
// is left in a.out
static int autotune_scan_tc(prism_plan *P, ScanArgs &a) {
    for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) P->tc_ms[v] = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    int rc = PRISM_OK, best = 0;
    double best_ms = -1.0;
    for (int v = 0; v < scan_tc_shapes(tc_mode(P->prec)) && v < PRISM_TUNE_MAX_SHAPES && !rc; ++v) {
        P->tc_shape = v;
        int grid = 0;
        if (scan_tc_grid(P->nw, P->kp, tc_mode(P->prec), v, a.scan_px, a.scan_py) <= 0) continue;  // does not fit
        if ((rc = scan_setup(P, a, &grid))) break;
        if ((rc = scan_go(P, a, grid))) break;
        cudaError_t e = cudaEventRecord(e0, P->stream);
        for (int r = 0; r < 2 && e == cudaSuccess && !rc; ++r) rc = scan_go(P, a, grid);
        if (rc) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(PRISM_ERR_CUDA, std::string("scan autotune ") + scan_tc_shape_name(v) + ": " + cudaGetErrorString(e));
            break;
        }
        P->tc_ms[v] = ms / 2.0;
        if (best_ms < 0 || ms / 2.0 < best_ms) {
            best = v;
            best_ms = ms / 2.0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->tc_shape = best;
    P->tc_tuned = !rc;
    if (rc) return rc;
    return scan_launch(P, a);
}

// The scan's contraction tile shape (Calculation Time section: the scan term P B N^2 / (4 f^4) is
// the rate-limiting one for large f): run the caller's scan once per compiled shape (one warm-up and
// two timed launches each, CUDA events on the plan's stream), keep the fastest for the plan's later
// scans.  Every shape writes bitwise the same detector stack, which is left in out_dev.
extern "C" int prism_plan_autotune_scan(prism_plan *P, const prism_probe *probe, const prism_scan *sc,
                                        const prism_detector *det, float *out_dev) {
    if (!P) return fail(PRISM_ERR_INVALID, "plan is NULL");
    ScanArgs a;
    int rc = scan_prepare(P, probe, sc, det, a);
    if (rc) return rc;
    if (a.n_probes == 0) return PRISM_OK;
    if ((rc = check_dev_ptr(out_dev, 4, "out_dev"))) return rc;
    a.out = out_dev;
    if (P->prec != PRISM_PRECISION_FP32) return autotune_scan_tc(P, a);
    for (int v = 0; v < PRISM_TUNE_MAX_SHAPES; ++v) P->scan_ms[v] = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    int best = 0;
    double best_ms = -1.0;
    for (int v = 0; v < scan_gemm_shapes() && v < PRISM_TUNE_MAX_SHAPES && !rc; ++v) {
        if (!scan_gemm_shape_valid(P->nw, P->nwy, v)) continue;
        P->scan_shape = v;
        int grid = 0;
        if ((rc = scan_setup(P, a, &grid))) break;
        if (grid <= 0) continue;  // this shape's coefficient block does not fit shared memory
        if ((rc = scan_go(P, a, grid))) break;
        cudaError_t e = cudaEventRecord(e0, P->stream);
        for (int r = 0; r < 2 && e == cudaSuccess && !rc; ++r) rc = scan_go(P, a, grid);
        if (rc) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(PRISM_ERR_CUDA, std::string("scan autotune ") + scan_gemm_shape_name(v) + ": " + cudaGetErrorString(e));
            break;
        }
        P->scan_ms[v] = ms / 2.0;
        if (best_ms < 0 || ms / 2.0 < best_ms) {
            best = v;
            best_ms = ms / 2.0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->scan_shape = best;
    P->scan_tuned = !rc;
    if (rc) return rc;
    return scan_launch(P, a);  // the detector stack of the chosen shape (bitwise that of every shape)
}

// ------------------------------------------------------------------ batches of cells (one CUDA graph)
struct prism_batch {
    std::vector<prism_plan *> plans;
    std::vector<ScanArgs> scans;
    std::vector<int> scan_grid;
    std::vector<const float *> V;
    std::vector<int> branch_of;
    std::vector<cudaStream_t> branches;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t origin = nullptr;  // capture origin (the caller's stream may be the legacy stream)
    cudaStream_t stream = nullptr;  // the caller's stream: every run is launched into it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    long launches = 0;
};

static void batch_release(prism_batch *B) {
    if (!B) return;
    cudaStreamSynchronize(B->stream);  // graph runs are ordered on the caller's stream (NULL: legacy)
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (prism_plan *P : B->plans) prism_plan_destroy(P);
    for (cudaEvent_t e : B->joins) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    for (cudaStream_t st : B->branches) cudaStreamDestroy(st);
    if (B->origin) cudaStreamDestroy(B->origin);
    delete B;
}

extern "C" int prism_batch_create(const prism_cell *cells, int n_cells, size_t hbm_budget_bytes, int n_branches, int flags,
                                  void *cuda_stream, prism_batch **out) {
    if (!out) return fail(PRISM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!cells || n_cells < 1) return fail(PRISM_ERR_INVALID, "need at least one cell");
    if (n_branches < 0 || n_branches > 16) return fail(PRISM_ERR_INVALID, "n_branches must be in [0, 16]");
    if (flags & ~(PRISM_BATCH_AUTOTUNE | PRISM_BATCH_AUTOTUNE_FFT_RADIX)) return fail(PRISM_ERR_INVALID, "unknown batch flags");
    const int nb = n_branches ? std::min(n_branches, n_cells) : std::min(n_cells, 4);
    int rc;
    for (int i = 0; i < n_cells; ++i) {
        const prism_cell &c = cells[i];
        if ((rc = check_dev_ptr(c.V_dev, 16, "cell V_dev")) || (rc = check_probe(&c.probe)) || (rc = check_det(&c.det)))
            return fail(rc, "cell " + std::to_string(i) + ": " + g_err);
        if ((long long)c.scan.px * c.scan.py > 0 && (rc = check_dev_ptr(c.out_dev, 4, "cell out_dev")))
            return fail(rc, "cell " + std::to_string(i) + ": " + g_err);
    }
    prism_batch *B = new prism_batch();
    B->stream = (cudaStream_t)cuda_stream;
    auto bail = [&](int code) {
        const std::string msg = g_err;
        batch_release(B);
        g_err = msg;
        return code;
    };
    auto cuda_bail = [&](cudaError_t e, const char *what) {
        fail(PRISM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return bail(PRISM_ERR_CUDA);
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking)) != cudaSuccess) return cuda_bail(e, "stream");
    // plans on the origin stream first (their allocations and uploads), branches assigned after
    std::vector<double> cost(n_cells);
    size_t bytes = 0;
    for (int i = 0; i < n_cells; ++i) {
        const prism_cell &c = cells[i];
        prism_plan *P = nullptr;
        if ((rc = prism_plan_create(&c.grid, 0, B->origin, &P))) return fail(rc, "cell " + std::to_string(i) + ": " + g_err), bail(rc);
        B->plans.push_back(P);
        P->shared_sms = nb > 1;
        if ((flags & (PRISM_BATCH_AUTOTUNE | PRISM_BATCH_AUTOTUNE_FFT_RADIX)) &&
            (rc = prism_plan_autotune_flags(P, (flags & PRISM_BATCH_AUTOTUNE_FFT_RADIX) ? PRISM_AUTOTUNE_FFT_RADIX : 0)))
            return bail(rc);
        ScanArgs a;
        if ((rc = scan_prepare(P, &c.probe, &c.scan, &c.det, a, false))) return fail(rc, "cell " + std::to_string(i) + ": " + g_err), bail(rc);
        a.out = c.out_dev;
        int grid = 0;
        if (a.n_probes > 0 && (rc = scan_setup(P, a, &grid))) return bail(rc);
        B->scans.push_back(a);
        B->scan_grid.push_back(grid);
        B->V.push_back(c.V_dev);
        bytes += P->arena.bytes;
        const double px = (double)c.grid.nx * c.grid.ny;
        cost[i] = (double)P->nbeams * c.grid.n_slices * px * 32.0 +
                  (double)a.n_probes * P->nbeams * P->nw * P->nwy * (P->prec == PRISM_PRECISION_FP32 ? 8.0 : 1.0);
    }
    if (hbm_budget_bytes && bytes > hbm_budget_bytes)
        return fail(PRISM_ERR_BUDGET, "batch needs " + std::to_string(bytes) + " bytes, budget " + std::to_string(hbm_budget_bytes)), bail(PRISM_ERR_BUDGET);
    if ((e = cudaStreamSynchronize(B->origin)) != cudaSuccess) return cuda_bail(e, "batch setup");
    // longest estimated work first onto the least-loaded branch
    std::vector<int> order(n_cells);
    for (int i = 0; i < n_cells; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<double> load(nb, 0.0);
    B->branch_of.assign(n_cells, 0);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        B->branch_of[i] = k;
        load[k] += cost[i];
    }
    for (int k = 0; k < nb; ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return cuda_bail(e, "stream");
        B->branches.push_back(st);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_bail(e, "event");
        B->joins.push_back(ev);
    }
    if ((e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming)) != cudaSuccess) return cuda_bail(e, "event");
    for (int i = 0; i < n_cells; ++i) {
        B->plans[i]->stream = B->branches[B->branch_of[i]];
        B->plans[i]->arena.stream = B->plans[i]->stream;
    }
    // capture: fork every branch from the origin, each branch runs its cells in order, join
    long before = 0;
    for (prism_plan *P : B->plans) before += P->launches;
    if ((e = cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_bail(e, "begin capture");
    int crc = PRISM_OK;
    cudaError_t ce = cudaEventRecord(B->fork, B->origin);
    for (int k = 0; k < nb && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(B->branches[k], B->fork, 0);
    for (int i = 0; i < n_cells && ce == cudaSuccess && !crc; ++i) {
        prism_plan *P = B->plans[i];
        crc = build_launches(P, B->V[i]);
        if (!crc && B->scans[i].n_probes > 0) crc = scan_go(P, B->scans[i], B->scan_grid[i]);
    }
    for (int k = 0; k < nb && ce == cudaSuccess && !crc; ++k) {
        ce = cudaEventRecord(B->joins[k], B->branches[k]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(B->origin, B->joins[k], 0);
    }
    cudaError_t ee = cudaStreamEndCapture(B->origin, &B->graph);
    if (crc) return bail(crc);
    if (ce != cudaSuccess) return cuda_bail(ce, "capture");
    if (ee != cudaSuccess) return cuda_bail(ee, "end capture");
    if ((e = cudaGraphInstantiate(&B->exec, B->graph, 0)) != cudaSuccess) return cuda_bail(e, "graph instantiate");
    if ((e = cudaGraphGetNodes(B->graph, nullptr, &B->nodes)) != cudaSuccess) return cuda_bail(e, "graph nodes");
    long after = 0;
    for (prism_plan *P : B->plans) after += P->launches;
    B->launches = after - before;
    *out = B;
    return PRISM_OK;
}

extern "C" int prism_batch_run(prism_batch *B) {
    if (!B) return fail(PRISM_ERR_INVALID, "batch is NULL");
    CUDA_TRY(cudaGraphLaunch(B->exec, B->stream));
    return PRISM_OK;
}

extern "C" int prism_batch_sync(prism_batch *B) {
    if (!B) return fail(PRISM_ERR_INVALID, "batch is NULL");
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    for (size_t i = 0; i < B->plans.size(); ++i) {
        int err = 0;
        CUDA_TRY(cudaMemcpy(&err, B->plans[i]->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) {
            CUDA_TRY(cudaMemset(B->plans[i]->dev_err, 0, sizeof(int)));
            // a scan or column pass whose wait ran out may have left its counters mid-count
            if (B->plans[i]->win_cnt) CUDA_TRY(cudaMemset(B->plans[i]->win_cnt, 0, B->plans[i]->cnt_cap));
            CUDA_TRY(cudaMemset(B->plans[i]->col_ctr, 0, 2 * sizeof(int)));
            return fail(PRISM_ERR_DEVICE, "cell " + std::to_string(i) + ": a kernel's bounded wait ran out");
        }
    }
    return PRISM_OK;
}

extern "C" int prism_batch_info_get(const prism_batch *B, prism_batch_info *out) {
    if (!B || !out) return fail(PRISM_ERR_INVALID, "NULL argument");
    out->n_cells = (int)B->plans.size();
    out->n_branches = (int)B->branches.size();
    out->graph_nodes = B->nodes;
    out->kernel_launches = B->launches;
    size_t bytes = 0;
    for (prism_plan *P : B->plans) bytes += P->arena.bytes;
    out->device_bytes = bytes;
    return PRISM_OK;
}

extern "C" void prism_batch_destroy(prism_batch *B) { batch_release(B); }
