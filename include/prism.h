/*
 * prism.h -- C ABI of the GB300 PRISM / multislice STEM simulation library (libprism.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the two halves of the PRISM
 * algorithm of Ophus, "A Fast Image Simulation Algorithm for Scanning Transmission
 * Electron Microscopy" (2017), and conventional per-probe multislice beside it:
 *
 *   (a) the compact S-matrix: multislice (Eq. Multislice) of every plane wave of the
 *       f-subsampled probe aperture (PRISM Algorithm section, plane-wave set), stored in
 *       real space at half resolution per axis when the anti-aliasing aperture allows it;
 *   (b) the probe scan: coefficients alpha_mn(r0), the d/f window of Eq. RegionBounds,
 *       the beam sum of Eq. PRISMfinal, window FFT, |psi|^2 and annular detector bins
 *       (Fig. 1d-f);
 *   (c) plain multislice of each probe (Multislice section) as the baseline form.
 *
 * Conventions (all calls):
 *   - Units: lengths in Angstrom, angles in mrad, voltage in kV, potentials in V*Angstrom.
 *   - Arrays are C row-major.  "device" pointers are CUDA device addresses in the current
 *     device's context (e.g. from PyTorch); "host" pointers are ordinary CPU memory
 *     (pinned memory makes the host variants asynchronous).
 *   - FFT convention: forward exp(-2 pi i k.x / N) unnormalised, frequencies q = k / cell
 *     for the signed index k (0..N/2-1, -N/2..-1).
 *   - Asynchrony: calls that take a plan enqueue work on the plan's CUDA stream and return;
 *     results are valid after prism_sync() (or any later synchronisation of that stream).
 *   - Status: every int-returning call returns PRISM_OK (0) or a negative PRISM_ERR_* code;
 *     prism_last_error() then describes the failure (thread-local string).
 *   - Determinism: the same inputs give bitwise-identical outputs (fixed reduction trees; the
 *     only atomics hand out work units -- column tiles, probe blocks -- and which CTA
 *     computes a unit changes no result), autotuned or not; only a plan tuned with the FFT radix
 *     variants (PRISM_AUTOTUNE_FFT_RADIX) may pick another rounding by timing.
 *   - A plan's calls run on its stream, one after another: its scratch and its work-unit
 *     counters are the plan's, so calls on one plan must not overlap (different plans may).
 *   - Memory: the caller owns every pointer it passes in; the plan owns the transmission
 *     functions, the S-matrix, its wave scratch and small tables, allocated with
 *     stream-ordered cudaMallocAsync and released by prism_plan_destroy().
 */
#ifndef PRISM_H
#define PRISM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PRISM_OK               0
#define PRISM_ERR_INVALID     -1  /* bad argument: NULL pointer, N % (2f) != 0, nbins <= 0, ... */
#define PRISM_ERR_BUDGET      -2  /* the plan does not fit the HBM budget given at creation     */
#define PRISM_ERR_CUDA        -3  /* a CUDA runtime call failed (message has the CUDA error)     */
#define PRISM_ERR_DEVICE      -4  /* a kernel raised the device error flag: one of its bounded
                                     waits ran out (tensor-core scan, TMA-staged tiles or rows)    */
#define PRISM_ERR_UNSUPPORTED -5  /* valid but not implemented here (e.g. non power-of-two N)   */
#define PRISM_ERR_CANCELLED   -6  /* a serving request was cancelled (prism_server_cancel)        */

/* Simulation grid and PRISM build parameters.
 *   nx, ny       wave / potential grid, powers of two in [16, 2048].
 *   n_slices     H >= 1 (Eq. Multislice is applied H times, propagation after each slice).
 *   cell_x/_y    orthorhombic cell side (Angstrom); pixel = cell / n.
 *   dz           uniform slice thickness t (Angstrom) when slice_dz == NULL; may be 0.
 *   slice_dz     optional host array [n_slices] of per-slice thickness (copied at plan creation;
 *                the paper allows unequal slices, Fig. 1a text).
 *   kv           accelerating voltage; lambda and sigma are relativistic (CODATA 2018).
 *   f            interpolation factor (PRISM Algorithm section), >= 1.
 *   downsample   1 (S stored at full resolution) or 2 (S stored on the inner half of Fourier
 *                space, the x4 storage saving enabled by the anti-aliasing aperture).
 *   aa_frac      anti-aliasing aperture |q| < aa_frac * q_nyquist, q_nyquist = min(nx/2cx, ny/2cy);
 *                must be <= 0.5 when downsample == 2; 0 < aa_frac.
 *   alpha_max_mrad  radius of the plane-wave set: sqrt(m^2+n^2) f lambda dq <= alpha_max
 *                (PRISM Algorithm section).  Must lie inside the anti-aliasing aperture.
 *   precision    storage of the S-matrix and arithmetic of the beam sum (Eq. PRISMfinal):
 *                PRISM_PRECISION_FP32 (complex64 S, FP32 CUDA-core sum), or
 *                PRISM_PRECISION_FP16 / PRISM_PRECISION_BF16: S stored pixel-major in 16-bit
 *                floats with one power-of-two scale per beam, the beam sum run on the tensor
 *                cores with FP32 accumulation (scan windows of 16, 32 or 64 pixels), or
 *                PRISM_PRECISION_FP16X2: the same with every S value and coefficient stored as an
 *                FP16 value plus the FP16 rounding of its remainder and three tensor-core products
 *                per step (value x value + value x remainder + remainder x value), FP32-class
 *                accuracy with the storage of FP32.  The build
 *                (transmission, FFTs, propagator) is FP32 in every mode.  Ignored by
 *                multislice_scan_run.  Zero-initialised structs select FP32.
 *   f_y          interpolation factor along y when it differs from f (f is then the factor along
 *                x; the paper allows one per axis): beams q_mn = (m f / cell_x, n f_y / cell_y),
 *                scan windows of nx_s / f x ny_s / f_y pixels.  0 means f_y = f.  Unequal windows
 *                need FP32 precision and window sides of 16, 32 or 64 pixels.
 */
typedef struct prism_grid {
    int nx, ny, n_slices;
    double cell_x, cell_y;
    double dz;
    const double *slice_dz;
    double kv;
    int f;
    int downsample;
    double aa_frac;
    double alpha_max_mrad;
    int precision;
    int f_y;
} prism_grid;

#define PRISM_PRECISION_FP32 0
#define PRISM_PRECISION_FP16 1
#define PRISM_PRECISION_BF16 2
#define PRISM_PRECISION_FP16X2 3

/* Probe: aperture semi-angle (A(q) = 1 where lambda|q| <= alpha), defocus C1 and spherical
 * aberration C3 (Angstrom) in chi(q) = pi lambda q^2 C1 + (pi/2) lambda^3 q^4 C3, and tilt
 * (rad, |tilt| <= 0.5).  A tilted probe has its aperture and chi centred on q_t = tilt / lambda
 * and its coefficients evaluated at r0 - h tan(tilt), h = cell thickness, which brings it back to
 * the centre of the cut-out region (PRISM Algorithm section); the beam set must reach |tilt| +
 * alpha (alpha_max_mrad of the grid), else the probe is truncated to the beams present. */
typedef struct prism_probe {
    double alpha_mrad, c1, c3, tilt_x, tilt_y;
} prism_probe;

/* Scan: px * py probe positions (Angstrom), host arrays x0[py*px], y0[py*px], row-major [py][px].
 * Positions may lie anywhere; windows wrap periodically (Eq. RegionBounds). px*py may be 0.
 * The arrays are read before the call returns. */
typedef struct prism_scan {
    int px, py;
    const double *x0;
    const double *y0;
} prism_scan;

/* Annular detector: bin b = floor((1000 lambda |q| - start_mrad) / step_mrad), kept when
 * 0 <= b < nbins; a pixel on an edge goes to the upper bin; q is the pixel-centre frequency.
 * step_mrad > 0, nbins in [1, 4096]. */
typedef struct prism_detector {
    double start_mrad, step_mrad;
    int nbins;
} prism_detector;

/* Read-only facts about a plan (filled by prism_plan_info). */
typedef struct prism_info {
    int n_beams;              /* B: plane waves in the S-matrix                        */
    int nx_s, ny_s;           /* stored grid (nx/downsample, ny/downsample)             */
    int nw_x, nw_y;           /* scan window in stored pixels (nx_s/f, ny_s/f)          */
    int beam_batch;           /* beams propagated together (limited by the HBM budget)  */
    double wavelength;        /* lambda, Angstrom                                      */
    double sigma;             /* interaction constant, rad/(V*Angstrom)                */
    size_t device_bytes;      /* device memory held by the plan                        */
} prism_info;

typedef struct prism_plan prism_plan;

/* ---- plan lifetime ------------------------------------------------------------------ */

/* Validate the grid, build the beam set, the FFT/propagator tables and allocate the plan's
 * device memory on `cuda_stream` (a cudaStream_t; NULL = legacy default stream) of the
 * current device.  hbm_budget_bytes = 0 means "no budget"; otherwise the plan's device
 * memory (transmission H*nx*ny*8, S-matrix B*nx_s*ny_s*8, wave scratch beam_batch*nx*ny*8)
 * must fit, with at least one beam in flight, else PRISM_ERR_BUDGET.
 * Errors: INVALID (NULL, non-positive sizes, nx % (2f) with downsample 2, aa_frac > 0.5 with
 * downsample 2, beams outside the AA aperture), UNSUPPORTED (n not a power of two in
 * [16, 2048]; window wider than 128 pixels), BUDGET, CUDA.  *out is NULL on failure. */
int prism_plan_create(const prism_grid *grid, size_t hbm_budget_bytes, void *cuda_stream,
                      prism_plan **out);

/* Release all device memory of the plan (stream-ordered) and the plan itself.  NULL is a no-op. */
void prism_plan_destroy(prism_plan *plan);

/* Wait for the plan's stream; returns DEVICE if a kernel raised the error flag, CUDA on a
 * CUDA error, else OK. */
int prism_sync(prism_plan *plan);

/* Thread-local description of the last failure of a call on this thread ("" if none). */
const char *prism_last_error(void);

/* ---- hot path --------------------------------------------------------------------- */

/* S-matrix build (PRISM Algorithm section, Fig. 1c; Eq. Multislice per beam and slice).
 * V_dev: device float32 [n_slices][ny][nx] projected potentials V_p (V*Angstrom), read only,
 * must stay valid until the call's work has run on the stream.  Computes t_p = exp(i sigma V_p)
 * and propagates every beam exp(2 pi i q_mn . r) through all slices.  Result stays in the plan. */
int prism_build_smatrix(prism_plan *plan, const float *V_dev);

/* Same as prism_build_smatrix with V in host memory (copied to a plan-owned device buffer
 * on the plan's stream; the host buffer may be reused once the call has run). */
int prism_build_smatrix_host(prism_plan *plan, const float *V_host);

/* Probe scan (Eq. RegionBounds, Eq. PRISMfinal, Fig. 1d-f) over the plan's S-matrix.
 * out_dev: device float32 [py][px][nbins], intensities in units of the incident probe
 * intensity.  Requires a completed prism_build_smatrix on this plan (else INVALID).
 * The probe's alpha may differ from alpha_max: beams outside it get A(q) = 0. */
int prism_scan_run(prism_plan *plan, const prism_probe *probe, const prism_scan *scan,
                   const prism_detector *det, float *out_dev);

/* Same as prism_scan_run with the result copied to host memory out_host [py][px][nbins]
 * (asynchronous for pinned memory: read it after prism_sync). */
int prism_scan_run_host(prism_plan *plan, const prism_probe *probe, const prism_scan *scan,
                        const prism_detector *det, float *out_host);

/* Full diffraction patterns instead of annular bins (Fig. 1f, "full probe diffraction pattern";
 * 4D-STEM): out_dev float32 [py][px][nw_y][nw_x], |FFT(window)|^2 in units of the incident
 * intensity, window frequencies in FFT order (index k <-> q = k f / cell for k < nw/2, k - nw
 * above).  Same requirements and asynchrony as prism_scan_run. */
int prism_scan_run_cbed(prism_plan *plan, const prism_probe *probe, const prism_scan *scan, float *out_dev);

/* Accumulating scan: out_dev[p][k] += weight * I[p][k] (in place; out_dev must hold the running
 * sum).  Frozen-phonon averaging (Simulation and Analysis Implementation section) is one
 * prism_build_smatrix per displaced-atom configuration followed by this call with weight 1/n. */
int prism_scan_run_accumulate(prism_plan *plan, const prism_probe *probe, const prism_scan *scan,
                              const prism_detector *det, float weight, float *out_dev);

/* Conventional multislice STEM (Multislice section, Eq. Multislice) of every probe: the probe
 * A(q) exp(-i chi) exp(-2 pi i q.r0) on the full grid, H slices, far-field |Psi|^2 divided by
 * sum |Psi0|^2, annular bins.  Same grid rules as a plan (f, downsample and alpha_max are
 * ignored).  V_dev as above, out_dev float32 [py][px][nbins].  Uses its own stream-ordered
 * scratch on `cuda_stream`, sized to at most max(1, scratch_bytes / (8 nx ny)) probes in flight
 * (scratch_bytes = 0: 1 GiB).  Asynchronous; synchronise the stream before reading out_dev.  At
 * 1024^2 the column passes stage their tiles through TMA with bounded waits; a wait that runs out
 * (which would leave a wave incomplete) makes that batch's bins NaN. */
int multislice_scan_run(const prism_grid *grid, const float *V_dev, const prism_probe *probe,
                        const prism_scan *scan, const prism_detector *det, float *out_dev,
                        void *cuda_stream, size_t scratch_bytes);

/* ---- fixed-scratch multislice ------------------------------------------------------ */

/* Size of the library's fixed device scratch array used by multislice_scan_run_noalloc. */
#define PRISM_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Multislice STEM scan that allocates no device memory.  The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory themselves, e.g. a host application that
 * owns the whole device-memory budget through its own pool and forbids other allocations, or a
 * latency-critical loop in which cudaMalloc / cudaFree (which may synchronise the device) are not
 * allowed.  It computes the same result as multislice_scan_run (same kernels, same arguments,
 * same output layout, bitwise-identical output) and calls no cudaMalloc, cudaFree or allocating
 * library routine; its transmission functions, wave and intensity buffers and tables live in one
 * file-scope device array of PRISM_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the
 * library holds until the process exits.  The caller still provides V_dev and out_dev.
 * Limits: the grid must fit the array with at least one probe in flight, about
 * nx*ny*(8*n_slices + 24) bytes plus 16 bytes per probe position (e.g. 256^2 with up to ~28
 * slices); larger requests return PRISM_ERR_BUDGET with the required size in prism_last_error().
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and keeps it for the life of the process; make that first call before any stream
 * capture, and do not call this entry point again after a cudaDeviceReset of that device (the kept
 * address would be stale).  All calls share the array and
 * every call overwrites what it uses, so calls that overlap on the GPU (different streams, or
 * different host threads on one device) race: serialise them on one stream.  Asynchronous like
 * multislice_scan_run: synchronise `cuda_stream` before reading out_dev. */
int multislice_scan_run_noalloc(const prism_grid *grid, const float *V_dev, const prism_probe *probe,
                                const prism_scan *scan, const prism_detector *det, float *out_dev,
                                void *cuda_stream);

/* ---- serving: continuous batching of simulation requests --------------------------------- */

/* A request: one cell (grid + potential), one probe configuration, one scan and detector.
 * Requests with the same non-zero smatrix_key (and the same grid) share one S-matrix, which stays
 * resident between requests: V_host is read only when that S-matrix is not resident (the S-matrix
 * serves every probe configuration, Varying Probe Size section).  smatrix_key = 0: private
 * S-matrix, released after the request.  V_host [n_slices][ny][nx] should be pinned (pageable
 * memory is copied synchronously by the worker) and must stay valid until the request completes;
 * the scan arrays and grid.slice_dz are copied at submission; out_host [py][px][nbins] is written
 * before prism_server_wait reports completion. */
typedef struct prism_request {
    prism_grid grid;
    const float *V_host;
    unsigned long long smatrix_key;
    prism_probe probe;
    prism_scan scan;
    prism_detector det;
    float *out_host;
} prism_request;

typedef struct prism_request_stats {
    double queued_ms;   /* submission -> admission                       */
    double total_ms;    /* submission -> result in out_host              */
    int smatrix_reused; /* 1 if a resident S-matrix served the request  */
    int status;         /* PRISM_OK or the request's error code          */
    double device_start_ms; /* when the request's stream reached its first operation (S-matrix
                               build or scan) and when it finished its last (the copy of the
                               result), in ms of device time since the server was created (CUDA
                               events); -1 when the request never ran on the device */
    double device_end_ms;
} prism_request_stats;

typedef struct prism_server_info {
    int pending, running, resident;   /* queued / in flight / resident S-matrices */
    long admitted, completed;
    size_t used_bytes, peak_bytes;    /* device memory accounted to requests and S-matrices */
} prism_server_info;

typedef struct prism_server prism_server;

/* Start a request engine on the current device.  A worker thread admits queued requests in
 * arrival order whenever fewer than max_inflight are running and the request's device footprint
 * (its S-matrix plan unless resident, output and positions) fits hbm_budget_bytes (0 = no
 * budget), evicting idle resident S-matrices least-recently-used when needed; a request that does
 * not fit yet does not hold back later ones.  Requests on different S-matrices run on different
 * streams and overlap on the device.  Results equal those of the request run alone (the kernels
 * are deterministic).  (No counterpart in the paper: this is the serving form of the method.) */
int prism_server_create(size_t hbm_budget_bytes, int max_inflight, prism_server **out);
/* Queue a request; returns a ticket.  Errors: INVALID for malformed requests. */
int prism_server_submit(prism_server *server, const prism_request *req, unsigned long long *ticket);
/* Wait at most timeout_s seconds for a ticket; OK when its result is in out_host, the request's
 * error code if it failed (BUDGET if it can never fit), DEVICE on timeout.  A ticket is forgotten
 * after a wait that does not time out.  stats may be NULL. */
int prism_server_wait(prism_server *server, unsigned long long ticket, double timeout_s, prism_request_stats *stats);
int prism_server_stats(prism_server *server, prism_server_info *out);
/* Cancel a request.  A queued request leaves the queue at once; a running one finishes its device
 * work (kernels are never interrupted) but its result is discarded and out_host is not written.
 * Either way its prism_server_wait returns PRISM_ERR_CANCELLED.  INVALID for an unknown ticket or a
 * request that has already completed.  (Failure handling of the serving loop; no counterpart in the
 * paper.) */
int prism_server_cancel(prism_server *server, unsigned long long ticket);
/* Finish the queued and running requests, release every S-matrix and stop the worker. */
void prism_server_destroy(prism_server *server);

/* ---- autotuner ------------------------------------------------------------------------
 *
 * The build is two streaming passes per slice (Calculation Time section: its cost grows with
 * beams x slices x N^2); their fastest launch shape (threads or interleaved columns per CTA,
 * staging of the next row or tile through shared memory by cp.async or by TMA, or none) and FFT radix
 * (the split of the 32- and 64-point register DFTs, prism_tune_shape_fft_variant) depend on N and
 * the beam batch.  At N = 1024 the untuned column pass already uses the TMA-staged shape.  prism_plan_autotune times every
 * compiled shape of the row pass (PRISM_TUNE_ROW) and the column pass (PRISM_TUNE_COL) on the
 * plan's own wave scratch (5 launches each after 2 warm-ups, CUDA events on the plan's stream)
 * and keeps the fastest for the plan's later builds.  Shapes exist for N = 256 ... 2048; smaller
 * grids keep their single shape.  Shapes of one radix variant compute bitwise the same result; the
 * radix variants compute the same transforms rounded differently (they agree to FP32 rounding,
 * well inside the FP32 path's tolerance against the FP64 oracle) and are candidates only when the
 * caller asks for them (prism_plan_autotune_flags), so that a plainly autotuned plan reproduces the
 * untuned plan bit for bit.  Results are
 * cached for the process per (pass, N, batch).  Synchronous; overwrites the wave scratch only (the
 * S-matrix is untouched).  The paper has no counterpart. */
#define PRISM_TUNE_ROW 0
#define PRISM_TUNE_COL 1
#define PRISM_TUNE_SCAN 2  /* contraction tile shape of the FP32 GEMM scan (prism_plan_autotune_scan) */
#define PRISM_TUNE_SCAN_TC 3  /* ring shape of the tensor-core scan of a 16-bit plan: stages x K values of
                                 its A operand (3 x 96 default, 2 x 128, 4 x 64; split mode 2 x 32 only) */
#define PRISM_TUNE_MAX_SHAPES 16
typedef struct prism_tune_entry {
    int n_shapes;                     /* shapes listed for the pass                              */
    int chosen;                       /* index of the shape in use (-1: the single default shape)  */
    int default_shape;                /* index of the untuned default (-1 if N has no shapes)      */
    double ms[PRISM_TUNE_MAX_SHAPES]; /* mean time per launch of each shape, -1 if not compiled   */
} prism_tune_entry;
int prism_plan_autotune(prism_plan *plan);
/* prism_plan_autotune with flags: PRISM_AUTOTUNE_FFT_RADIX also times the FFT radix variants
 * (prism_tune_shape_fft_variant) and may keep one, whose results agree with the default's to
 * rounding but not bit for bit; without it (prism_plan_autotune) the tuner keeps the radix of the
 * default launchers at the plan's N (both transforms radix-4 first at N = 2048, the default split
 * elsewhere) and every result stays bitwise that of the untuned plan.  INVALID for unknown flags. */
#define PRISM_AUTOTUNE_FFT_RADIX 1
int prism_plan_autotune_flags(prism_plan *plan, int flags);
/* The scan's contraction tile shape (the scan term of the Calculation Time section's cost model):
 * raster blocks of 4 x 8, 8 x 4 or 2 x 16 probes and beam rings of 2 x 33 (default), 2 x 32 or 3 x 16, compiled for
 * the FP32 GEMM scan with square windows of 16, 32 or 64 pixels.  Runs the given scan once per
 * shape (a warm-up and two timed launches, CUDA events on the plan's stream), keeps the fastest
 * for the plan's later scans (prism_plan_tune_result with PRISM_TUNE_SCAN) and leaves the detector
 * stack in out_dev: every shape sums each pixel over the beams in the same order, so all give
 * bitwise the same stack.  A 16-bit plan times the ring shapes of its tensor-core scan the same way
 * (PRISM_TUNE_SCAN_TC; the K = 16 MMAs of a pixel tile go in the same order in every shape, so the
 * stacks are bitwise equal too).  Other plans (other windows) just run the scan.  Arguments
 * and errors as prism_scan_run; synchronous.  No counterpart in the paper. */
int prism_plan_autotune_scan(prism_plan *plan, const prism_probe *probe, const prism_scan *scan,
                             const prism_detector *det, float *out_dev);
int prism_plan_tune_result(const prism_plan *plan, int kind, prism_tune_entry *out);
const char *prism_tune_shape_name(int kind, int shape);
/* FFT radix variant of a row or column shape: bit 0 for the forward, bit 1 for the inverse
 * transform of the pass, each 0 for the default split of its 32- and 64-point register DFTs
 * (32 = 8 x 4 and 64 = 8 x 8, second stage radix 4 with tangent-form twiddles where it applies) or 1
 * for a radix-4 first stage (32 = 4 x 8, 64 = 4 x 16); -1 for another kind or an unknown shape. */
int prism_tune_shape_fft_variant(int kind, int shape);
/* Pin the launch shape of one pass (or the scan's contraction shape, PRISM_TUNE_SCAN) for the
 * plan's later builds (scans) without timing: `shape` indexes the kind's list
 * (prism_tune_shape_name), -1 restores the default.  PRISM_ERR_INVALID for a NULL plan or a kind
 * outside {PRISM_TUNE_ROW, PRISM_TUNE_COL, PRISM_TUNE_SCAN, PRISM_TUNE_SCAN_TC}; PRISM_ERR_UNSUPPORTED for a shape not
 * compiled for the plan's N (window), or one that stages through TMA when the plan holds no tensor
 * map of its wave scratch.  Shapes of the default's FFT radix variant compute bitwise the same
 * result; the other variant agrees to rounding. */
int prism_plan_set_tune_shape(prism_plan *plan, int kind, int shape);

/* ---- batches of uneven cells: one captured CUDA graph ------------------------------
 *
 * Many independent simulations of different sizes, slice counts, f and precision (the paper's
 * cost model, Calculation Time section, makes small cells launch-bound and large ones
 * bandwidth-bound) run as one CUDA graph: each cell gets its own plan, all scan inputs are uploaded
 * at creation, and every cell's transmission, build, quantisation and scan launches are captured
 * once.  Cells are spread over n_branches parallel graph branches, longest estimated work first
 * (beams x slices x pixels for the build plus probes x beams x window pixels for the scan), so
 * small cells run beside large ones.  prism_batch_run is one cudaGraphLaunch.  The paper has no
 * counterpart; this is the batched form of its algorithm. */
typedef struct prism_cell {
    prism_grid grid;          /* the cell (any precision); grid.slice_dz is copied at creation    */
    const float *V_dev;       /* [n_slices][ny][nx] potential, caller-owned device memory, read at
                                 every run (its contents may change between runs, not its address) */
    prism_probe probe;
    prism_scan scan;          /* positions are copied at creation; px * py may be 0                */
    prism_detector det;
    float *out_dev;           /* [py*px][nbins] caller-owned device output, written at every run    */
} prism_cell;

typedef struct prism_batch_info {
    int n_cells;
    int n_branches;
    size_t graph_nodes;       /* kernel and event nodes of the captured graph                     */
    long kernel_launches;     /* kernels one run launches                                           */
    size_t device_bytes;      /* device memory held by the batch's plans                          */
} prism_batch_info;

typedef struct prism_batch prism_batch;

/* Validate every cell, create its plan (INVALID/UNSUPPORTED as prism_plan_create, with the cell
 * index in the message), upload its scan inputs, optionally autotune it (flags), and capture the
 * graph.  n_branches in [1, 16] (0 = min(n_cells, 4)).  hbm_budget_bytes bounds the sum of the plans' device memory (0 = no
 * limit; BUDGET if exceeded).  The graph is launched into cuda_stream (NULL = legacy default). */
#define PRISM_BATCH_AUTOTUNE 1  /* flags: autotune every cell's plan's launch shapes before the capture */
#define PRISM_BATCH_AUTOTUNE_FFT_RADIX 2  /* flags: the same with the FFT radix variants as candidates */
int prism_batch_create(const prism_cell *cells, int n_cells, size_t hbm_budget_bytes, int n_branches, int flags,
                       void *cuda_stream, prism_batch **out);
/* Enqueue one run of the whole batch (asynchronous on the batch's stream). */
int prism_batch_run(prism_batch *batch);
/* Wait for the batch's stream; DEVICE if a kernel of any cell raised its error word. */
int prism_batch_sync(prism_batch *batch);
int prism_batch_info_get(const prism_batch *batch, prism_batch_info *out);
void prism_batch_destroy(prism_batch *batch);

/* ---- introspection (tests, tools) ----------------------------------------------- */

int prism_plan_info(const prism_plan *plan, prism_info *out);

/* Bytes of the stored S-matrix: B * nx_s * ny_s * 8 in FP32 mode; nx_s * ny_s * K * 2 + 4 * K / 2
 * (16-bit values, K = 2 * roundup(B, 8), plus the per-beam scales) in FP16/BF16 mode; twice the
 * 16-bit part in FP16X2 mode. */
int prism_plan_smatrix_bytes(const prism_plan *plan, size_t *out);

/* Beam indices (m, n) of the plane-wave set, q_mn = (m f / cell_x, n f / cell_y), in the
 * plan's order (n ascending, then m ascending).  capacity >= n_beams else INVALID. */
int prism_plan_beams(const prism_plan *plan, int *m, int *n, int capacity);

/* Device pointers owned by the plan (valid until destroy): the S-matrix complex64
 * [B][ny_s][nx_s] (interleaved re, im) and the transmission functions complex64 [H][ny][nx].
 * prism_plan_smatrix fails with INVALID in FP16/BF16 mode (use prism_plan_smatrix_copy). */
int prism_plan_smatrix(const prism_plan *plan, const void **dev_ptr);
int prism_plan_transmission(const prism_plan *plan, const void **dev_ptr);

/* Write the S-matrix as complex64 [B][ny_s][nx_s] into out_dev (caller-owned device buffer of
 * B * nx_s * ny_s * 8 bytes), asynchronously on the plan's stream: a copy in FP32 mode, the
 * 16-bit values times their beam scale in FP16/BF16 mode (the values the beam sum uses).
 * INVALID before the S-matrix is built. */
int prism_plan_smatrix_copy(prism_plan *plan, float *out_dev);

/* Load an S-matrix instead of building it (checkpoint / resume: the build is the expensive part of
 * the method, Calculation Time section, and the same S serves every later probe configuration,
 * Varying Probe Size section).  S_dev is complex64 [B][ny_s][nx_s] as written by
 * prism_plan_smatrix_copy of a plan with the same grid, in caller-owned device memory that must stay
 * valid until the plan's stream has passed this call (prism_sync).  FP32 plans copy it; 16-bit plans
 * quantise it beam batch by beam batch as their build does.  The plan is then built.  INVALID for a
 * NULL plan or a misaligned S_dev. */
int prism_plan_load_smatrix(prism_plan *plan, const float *S_dev);

/* Diagnostic of the tensor-core path (no counterpart in the paper): one tcgen05 MMA
 * D[128][16] = A[128][16] B[16][16]^T on small-integer FP16 operands, A[m][k] = (m + 3k) % 7 - 3,
 * B[n][k] = (5n + k) % 5 - 2, written to out_dev float32 [128][16]; status_dev[0] is set to 1 if the
 * MMA did not complete within its poll limit (caller zeroes it).  Asynchronous on cuda_stream. */
int prism_selftest_tcgen05(float *out_dev, int *status_dev, void *cuda_stream);

/* Diagnostic of failure detection (no counterpart in the paper): the library's in-kernel waits
 * (tensor-core scan, TMA staging) are mbarrier waits that give up after a clock budget and report
 * through an error word instead of hanging.  This launches one CTA whose threads wait at most
 * limit_cycles SM cycles (0 ... 4e9) for a barrier's first phase; with arrive = 0 nothing completes
 * it and status_dev[0] is set to 1 (the wait ran out, the context stays usable), with arrive != 0
 * one arrival completes it and status_dev[0] is left alone (caller zeroes it).  Asynchronous on
 * cuda_stream.  INVALID for a NULL status_dev or a limit outside that range. */
int prism_selftest_bounded_wait(int *status_dev, long long limit_cycles, int arrive, void *cuda_stream);

/* Relativistic wavelength (Angstrom) and interaction constant (rad/(V*Angstrom)), CODATA 2018. */
double prism_wavelength(double kv);
double prism_interaction_constant(double kv);

/* Beam-set radius for a probe (PRISM Algorithm section: the maximum incident semi-angle should be
 * the largest desired probe semi-angle plus f times the Fourier pixel size).  Writes to
 * *alpha_max_mrad = probe->alpha_mrad + 1000 |tilt| + 1000 lambda max(f / cell_x, f_y / cell_y)
 * (mrad; |tilt| = hypot(tilt_x, tilt_y) in rad, the tilted aperture's centre offset; f_y = 0 means
 * f), the value to put in prism_grid.alpha_max_mrad so that the plan's plane-wave set holds every
 * beam of the (tilted) probe with one lattice step of margin.  Reads grid->kv, f, f_y, cell_x and
 * cell_y only.  Host-only, synchronous.  INVALID for NULL pointers, kv <= 0, f < 1, f_y < 0,
 * cells <= 0 or a negative probe semi-angle. */
int prism_recommended_alpha_max(const prism_grid *grid, const prism_probe *probe, double *alpha_max_mrad);

/* ---- per-kernel timing ------------------------------------------------------------ */

/* Kernel classes timed by the plan when profiling is on. */
#define PRISM_K_TRANSMIT   0  /* t_p = exp(i sigma V_p)                                    */
#define PRISM_K_ROW_PLANE  1  /* first slice: row FFT of t_0 (once per build)                */
#define PRISM_K_ROW        2  /* row IFFT, x t_p, row FFT                                   */
#define PRISM_K_COL        3  /* column FFT, x propagator (AA-masked), column IFFT          */
#define PRISM_K_ROW_OUT    4  /* last row IFFT, store S                                     */
#define PRISM_K_SCAN       5  /* coefficients + window gather + beam sum + window FFT + bins */
#define PRISM_K_QUANT      6  /* FP16/BF16 mode: per-beam scales, S to pixel-major 16-bit     */
#define PRISM_K_PLANE      7  /* first slice of every beam: the row FFT of t_0 shifted by the
                                 beam's m f columns, times its y phase (shift theorem)        */
#define PRISM_K_COUNT      8

/* profiling on: every launch of the plan is bracketed by CUDA events on the plan's stream. */
int prism_plan_set_profiling(prism_plan *plan, int enable);
/* Launch count and summed event time (ms) of one kernel class since profiling was enabled
 * (synchronises the plan's stream).  Also counts launches while profiling is off. */
int prism_plan_kernel_stats(prism_plan *plan, int kind, long *launches, double *total_ms);
/* Total kernel launches issued by the plan since creation (or the last reset). */
long prism_plan_launches(const prism_plan *plan);
int prism_plan_reset_stats(prism_plan *plan);
const char *prism_kernel_name(int kind);

#ifdef __cplusplus
}
#endif
#endif /* PRISM_H */
