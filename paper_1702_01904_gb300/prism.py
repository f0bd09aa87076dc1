"""ctypes binding of libprism.so (include/prism.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device buffers are passed as
integers (CUDA device addresses) or as objects with ``data_ptr()`` (torch tensors); streams as
integers (``torch.cuda.current_stream().cuda_stream``) or ``None`` for the legacy default stream.
A non-zero status raises :class:`PrismError` carrying the status and ``prism_last_error()``.
There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_long, c_size_t, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libprism.so")

PRISM_OK = 0
PRISM_ERR_INVALID = -1
PRISM_ERR_BUDGET = -2
PRISM_ERR_CUDA = -3
PRISM_ERR_DEVICE = -4
PRISM_ERR_UNSUPPORTED = -5
PRISM_ERR_CANCELLED = -6

PRISM_K_TRANSMIT, PRISM_K_ROW_PLANE, PRISM_K_ROW, PRISM_K_COL, PRISM_K_ROW_OUT, PRISM_K_SCAN, PRISM_K_QUANT, PRISM_K_PLANE = range(8)
PRISM_K_COUNT = 8

PRISM_PRECISION_FP32 = 0
PRISM_PRECISION_FP16 = 1
PRISM_PRECISION_BF16 = 2
PRISM_PRECISION_FP16X2 = 3

PRISM_TUNE_ROW = 0
PRISM_TUNE_COL = 1
PRISM_TUNE_SCAN = 2
PRISM_TUNE_SCAN_TC = 3
PRISM_TUNE_MAX_SHAPES = 16
PRISM_BATCH_AUTOTUNE = 1
PRISM_BATCH_AUTOTUNE_FFT_RADIX = 2
PRISM_AUTOTUNE_FFT_RADIX = 1

# every entry point declared in include/prism.h
EXPORTED = [
    "prism_plan_create", "prism_plan_destroy", "prism_sync", "prism_last_error",
    "prism_build_smatrix", "prism_build_smatrix_host", "prism_scan_run", "prism_scan_run_host",
    "prism_scan_run_cbed", "prism_scan_run_accumulate",
    "multislice_scan_run", "multislice_scan_run_noalloc", "prism_plan_info", "prism_plan_smatrix_bytes", "prism_plan_beams",
    "prism_plan_smatrix", "prism_plan_smatrix_copy", "prism_plan_transmission", "prism_wavelength", "prism_interaction_constant",
    "prism_recommended_alpha_max", "prism_plan_set_profiling", "prism_plan_kernel_stats", "prism_plan_launches", "prism_plan_reset_stats",
    "prism_kernel_name",
    "prism_server_create", "prism_server_submit", "prism_server_wait", "prism_server_stats", "prism_server_destroy",
    "prism_server_cancel",
    "prism_selftest_tcgen05", "prism_selftest_bounded_wait",
    "prism_batch_create", "prism_batch_run", "prism_batch_sync", "prism_batch_info_get", "prism_batch_destroy",
    "prism_plan_autotune", "prism_plan_autotune_scan", "prism_plan_tune_result", "prism_tune_shape_name", "prism_plan_set_tune_shape",
    "prism_tune_shape_fft_variant", "prism_plan_autotune_flags",
    "prism_plan_load_smatrix",
]


class PrismError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libprism status {status}: {msg}")
        self.status = status


class PrismGrid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("n_slices", c_int),
                ("cell_x", c_double), ("cell_y", c_double), ("dz", c_double),
                ("slice_dz", POINTER(c_double)), ("kv", c_double), ("f", c_int),
                ("downsample", c_int), ("aa_frac", c_double), ("alpha_max_mrad", c_double),
                ("precision", c_int), ("f_y", c_int)]


class PrismProbe(ctypes.Structure):
    _fields_ = [("alpha_mrad", c_double), ("c1", c_double), ("c3", c_double),
                ("tilt_x", c_double), ("tilt_y", c_double)]


class PrismScan(ctypes.Structure):
    _fields_ = [("px", c_int), ("py", c_int), ("x0", POINTER(c_double)), ("y0", POINTER(c_double))]


class PrismDetector(ctypes.Structure):
    _fields_ = [("start_mrad", c_double), ("step_mrad", c_double), ("nbins", c_int)]


class PrismInfo(ctypes.Structure):
    _fields_ = [("n_beams", c_int), ("nx_s", c_int), ("ny_s", c_int), ("nw_x", c_int), ("nw_y", c_int),
                ("beam_batch", c_int), ("wavelength", c_double), ("sigma", c_double),
                ("device_bytes", c_size_t)]


class PrismRequest(ctypes.Structure):
    _fields_ = [("grid", PrismGrid), ("V_host", c_void_p), ("smatrix_key", ctypes.c_ulonglong),
                ("probe", PrismProbe), ("scan", PrismScan), ("det", PrismDetector), ("out_host", c_void_p)]


class PrismRequestStats(ctypes.Structure):
    _fields_ = [("queued_ms", c_double), ("total_ms", c_double), ("smatrix_reused", c_int), ("status", c_int),
                ("device_start_ms", c_double), ("device_end_ms", c_double)]


class PrismServerInfo(ctypes.Structure):
    _fields_ = [("pending", c_int), ("running", c_int), ("resident", c_int), ("admitted", c_long),
                ("completed", c_long), ("used_bytes", c_size_t), ("peak_bytes", c_size_t)]


_lib = None


class PrismTuneEntry(ctypes.Structure):
    _fields_ = [("n_shapes", c_int), ("chosen", c_int), ("default_shape", c_int), ("ms", c_double * PRISM_TUNE_MAX_SHAPES)]


class PrismCell(ctypes.Structure):
    _fields_ = [("grid", PrismGrid), ("V_dev", c_void_p), ("probe", PrismProbe), ("scan", PrismScan),
                ("det", PrismDetector), ("out_dev", c_void_p)]


class PrismBatchInfo(ctypes.Structure):
    _fields_ = [("n_cells", c_int), ("n_branches", c_int), ("graph_nodes", c_size_t),
                ("kernel_launches", c_long), ("device_bytes", c_size_t)]


def load(path: str = LIB_PATH):
    """Load libprism.so (built by ``paper_1702_01904_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libprism.so not found at {path}: run `python -m paper_1702_01904_gb300.build`")
    L = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "prism_plan_create": (c_int, [POINTER(PrismGrid), c_size_t, P, POINTER(P)]),
        "prism_plan_destroy": (None, [P]),
        "prism_sync": (c_int, [P]),
        "prism_last_error": (c_char_p, []),
        "prism_build_smatrix": (c_int, [P, P]),
        "prism_build_smatrix_host": (c_int, [P, P]),
        "prism_scan_run": (c_int, [P, POINTER(PrismProbe), POINTER(PrismScan), POINTER(PrismDetector), P]),
        "prism_scan_run_host": (c_int, [P, POINTER(PrismProbe), POINTER(PrismScan), POINTER(PrismDetector), P]),
        "prism_scan_run_cbed": (c_int, [P, POINTER(PrismProbe), POINTER(PrismScan), P]),
        "prism_scan_run_accumulate": (c_int, [P, POINTER(PrismProbe), POINTER(PrismScan), POINTER(PrismDetector),
                                              ctypes.c_float, P]),
        "multislice_scan_run": (c_int, [POINTER(PrismGrid), P, POINTER(PrismProbe), POINTER(PrismScan),
                                        POINTER(PrismDetector), P, P, c_size_t]),
        "multislice_scan_run_noalloc": (c_int, [POINTER(PrismGrid), P, POINTER(PrismProbe), POINTER(PrismScan),
                                                POINTER(PrismDetector), P, P]),
        "prism_plan_info": (c_int, [P, POINTER(PrismInfo)]),
        "prism_plan_smatrix_bytes": (c_int, [P, POINTER(c_size_t)]),
        "prism_plan_beams": (c_int, [P, POINTER(c_int), POINTER(c_int), c_int]),
        "prism_plan_smatrix": (c_int, [P, POINTER(P)]),
        "prism_plan_smatrix_copy": (c_int, [P, P]),
        "prism_batch_create": (c_int, [POINTER(PrismCell), c_int, c_size_t, c_int, c_int, P, POINTER(P)]),
        "prism_plan_autotune": (c_int, [P]),
        "prism_plan_autotune_flags": (c_int, [P, c_int]),
        "prism_plan_autotune_scan": (c_int, [P, POINTER(PrismProbe), POINTER(PrismScan), POINTER(PrismDetector), P]),
        "prism_plan_tune_result": (c_int, [P, c_int, POINTER(PrismTuneEntry)]),
        "prism_tune_shape_name": (c_char_p, [c_int, c_int]),
        "prism_tune_shape_fft_variant": (c_int, [c_int, c_int]),
        "prism_plan_set_tune_shape": (c_int, [P, c_int, c_int]),
        "prism_plan_load_smatrix": (c_int, [P, P]),
        "prism_batch_run": (c_int, [P]),
        "prism_batch_sync": (c_int, [P]),
        "prism_batch_info_get": (c_int, [P, POINTER(PrismBatchInfo)]),
        "prism_batch_destroy": (None, [P]),
        "prism_plan_transmission": (c_int, [P, POINTER(P)]),
        "prism_wavelength": (c_double, [c_double]),
        "prism_interaction_constant": (c_double, [c_double]),
        "prism_recommended_alpha_max": (c_int, [POINTER(PrismGrid), POINTER(PrismProbe), POINTER(c_double)]),
        "prism_plan_set_profiling": (c_int, [P, c_int]),
        "prism_plan_kernel_stats": (c_int, [P, c_int, POINTER(c_long), POINTER(c_double)]),
        "prism_plan_launches": (c_long, [P]),
        "prism_plan_reset_stats": (c_int, [P]),
        "prism_kernel_name": (c_char_p, [c_int]),
        "prism_server_create": (c_int, [c_size_t, c_int, POINTER(P)]),
        "prism_server_submit": (c_int, [P, POINTER(PrismRequest), POINTER(ctypes.c_ulonglong)]),
        "prism_server_wait": (c_int, [P, ctypes.c_ulonglong, c_double, POINTER(PrismRequestStats)]),
        "prism_server_stats": (c_int, [P, POINTER(PrismServerInfo)]),
        "prism_server_destroy": (None, [P]),
        "prism_server_cancel": (c_int, [P, ctypes.c_ulonglong]),
        "prism_selftest_tcgen05": (c_int, [P, P, P]),
        "prism_selftest_bounded_wait": (c_int, [P, ctypes.c_longlong, c_int, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != PRISM_OK:
        raise PrismError(status, load().prism_last_error().decode())
    return status


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return c_void_p(x.ctypes.data)
    return c_void_p(int(x))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return c_void_p(s.cuda_stream)
    return c_void_p(int(s))


# ------------------------------------------------------------------ struct helpers
def make_grid(nx, ny, n_slices, cell_x, cell_y, dz, kv, f=1, downsample=2, aa_frac=0.5,
              alpha_max_mrad=20.0, slice_dz=None, precision=PRISM_PRECISION_FP32, f_y=0):
    g = PrismGrid(nx, ny, n_slices, cell_x, cell_y, dz, None, kv, f, downsample, aa_frac, alpha_max_mrad,
                  precision, f_y)
    if slice_dz is not None:
        arr = np.ascontiguousarray(slice_dz, dtype=np.float64)
        g._keep = arr
        g.slice_dz = arr.ctypes.data_as(POINTER(c_double))
    return g


def grid_from_workload(w, precision=PRISM_PRECISION_FP32):
    return make_grid(w.nx, w.ny, w.n_slices, w.cell_x, w.cell_y, w.dz, w.kv, w.f, w.downsample,
                     w.aa_frac, w.alpha_mrad, precision=precision)


def make_probe(alpha_mrad, c1=0.0, c3=0.0, tilt_x=0.0, tilt_y=0.0):
    return PrismProbe(alpha_mrad, c1, c3, tilt_x, tilt_y)


def make_scan(px, py, x0, y0):
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    s = PrismScan(px, py, x0.ctypes.data_as(POINTER(c_double)), y0.ctypes.data_as(POINTER(c_double)))
    s._keep = (x0, y0)
    return s


def make_detector(start_mrad, step_mrad, nbins):
    return PrismDetector(start_mrad, step_mrad, nbins)


# ------------------------------------------------------------------ entry points (same names as C)
def prism_plan_create(grid, hbm_budget_bytes=0, cuda_stream=None):
    L = load()
    plan = c_void_p()
    _check(L.prism_plan_create(byref(grid), hbm_budget_bytes, _stream(cuda_stream), byref(plan)))
    return plan


def prism_plan_destroy(plan):
    load().prism_plan_destroy(plan)


def prism_sync(plan):
    return _check(load().prism_sync(plan))


def prism_last_error():
    return load().prism_last_error().decode()


def prism_build_smatrix(plan, V_dev):
    return _check(load().prism_build_smatrix(plan, _ptr(V_dev)))


def prism_build_smatrix_host(plan, V_host):
    return _check(load().prism_build_smatrix_host(plan, _ptr(V_host)))


def prism_scan_run(plan, probe, scan, det, out_dev):
    return _check(load().prism_scan_run(plan, byref(probe), byref(scan), byref(det), _ptr(out_dev)))


def prism_scan_run_host(plan, probe, scan, det, out_host):
    return _check(load().prism_scan_run_host(plan, byref(probe), byref(scan), byref(det), _ptr(out_host)))


def prism_scan_run_cbed(plan, probe, scan, out_dev):
    return _check(load().prism_scan_run_cbed(plan, byref(probe), byref(scan), _ptr(out_dev)))


def prism_scan_run_accumulate(plan, probe, scan, det, weight, out_dev):
    return _check(load().prism_scan_run_accumulate(plan, byref(probe), byref(scan), byref(det), weight, _ptr(out_dev)))


def multislice_scan_run(grid, V_dev, probe, scan, det, out_dev, cuda_stream=None, scratch_bytes=0):
    return _check(load().multislice_scan_run(byref(grid), _ptr(V_dev), byref(probe), byref(scan), byref(det),
                                             _ptr(out_dev), _stream(cuda_stream), scratch_bytes))


def multislice_scan_run_noalloc(grid, V_dev, probe, scan, det, out_dev, cuda_stream=None):
    """Same as multislice_scan_run, using the library's fixed 16 MiB device scratch instead of
    allocating (for callers that may not allocate device memory; see include/prism.h)."""
    return _check(load().multislice_scan_run_noalloc(byref(grid), _ptr(V_dev), byref(probe), byref(scan),
                                                     byref(det), _ptr(out_dev), _stream(cuda_stream)))


PRISM_NOALLOC_SCRATCH_BYTES = 16 << 20


def prism_plan_info(plan):
    info = PrismInfo()
    _check(load().prism_plan_info(plan, byref(info)))
    return info


def prism_plan_smatrix_bytes(plan):
    n = c_size_t()
    _check(load().prism_plan_smatrix_bytes(plan, byref(n)))
    return n.value


def prism_plan_beams(plan):
    nb = prism_plan_info(plan).n_beams
    m = (c_int * nb)()
    n = (c_int * nb)()
    _check(load().prism_plan_beams(plan, m, n, nb))
    return np.array(m[:], dtype=np.int64), np.array(n[:], dtype=np.int64)


def prism_plan_smatrix(plan):
    p = c_void_p()
    _check(load().prism_plan_smatrix(plan, byref(p)))
    return p.value


def prism_plan_smatrix_copy(plan, out_dev):
    _check(load().prism_plan_smatrix_copy(plan, _ptr(out_dev)))


def prism_plan_transmission(plan):
    p = c_void_p()
    _check(load().prism_plan_transmission(plan, byref(p)))
    return p.value


def prism_wavelength(kv):
    return load().prism_wavelength(kv)


def prism_interaction_constant(kv):
    return load().prism_interaction_constant(kv)


def prism_recommended_alpha_max(grid, probe):
    """The plane-wave-set radius (mrad) that keeps every beam of `probe` with one lattice step of
    margin (prism_recommended_alpha_max in include/prism.h)."""
    out = c_double()
    _check(load().prism_recommended_alpha_max(byref(grid), byref(probe), byref(out)))
    return out.value


def prism_plan_set_profiling(plan, enable=True):
    return _check(load().prism_plan_set_profiling(plan, 1 if enable else 0))


def prism_plan_kernel_stats(plan, kind):
    n = c_long()
    ms = c_double()
    _check(load().prism_plan_kernel_stats(plan, kind, byref(n), byref(ms)))
    return n.value, ms.value


def prism_plan_launches(plan):
    return load().prism_plan_launches(plan)


def prism_plan_reset_stats(plan):
    return _check(load().prism_plan_reset_stats(plan))


def prism_kernel_name(kind):
    return load().prism_kernel_name(kind).decode()


# ------------------------------------------------------------------ serving
def prism_server_create(hbm_budget_bytes=0, max_inflight=4):
    srv = c_void_p()
    _check(load().prism_server_create(hbm_budget_bytes, max_inflight, byref(srv)))
    return srv


def prism_server_submit(server, request):
    t = ctypes.c_ulonglong()
    _check(load().prism_server_submit(server, byref(request), byref(t)))
    return t.value


def prism_server_wait(server, ticket, timeout_s=600.0):
    st = PrismRequestStats()
    _check(load().prism_server_wait(server, ticket, timeout_s, byref(st)))
    return st


def prism_server_stats(server):
    info = PrismServerInfo()
    _check(load().prism_server_stats(server, byref(info)))
    return info


def prism_server_cancel(server, ticket):
    _check(load().prism_server_cancel(server, ticket))


def prism_server_destroy(server):
    load().prism_server_destroy(server)


def prism_selftest_tcgen05(out_dev, status_dev, cuda_stream=None):
    return _check(load().prism_selftest_tcgen05(_ptr(out_dev), _ptr(status_dev), _stream(cuda_stream)))


def prism_selftest_bounded_wait(status_dev, limit_cycles, arrive, cuda_stream=None):
    return _check(load().prism_selftest_bounded_wait(_ptr(status_dev), int(limit_cycles), int(arrive), _stream(cuda_stream)))


# ------------------------------------------------------------------ batches of cells
def make_cell(grid, V_dev, probe, scan, det, out_dev):
    c = PrismCell(grid, _ptr(V_dev), probe, scan, det, _ptr(out_dev))
    c._keep = (grid, scan)
    return c


def prism_batch_create(cells, hbm_budget_bytes=0, n_branches=0, cuda_stream=None, flags=0):
    arr = (PrismCell * len(cells))(*cells)
    b = c_void_p()
    _check(load().prism_batch_create(arr, len(cells), hbm_budget_bytes, n_branches, flags, _stream(cuda_stream),
                                     byref(b)))
    return b


def prism_batch_run(batch):
    _check(load().prism_batch_run(batch))


def prism_batch_sync(batch):
    _check(load().prism_batch_sync(batch))


def prism_batch_info_get(batch):
    i = PrismBatchInfo()
    _check(load().prism_batch_info_get(batch, byref(i)))
    return i


def prism_batch_destroy(batch):
    load().prism_batch_destroy(batch)


# ------------------------------------------------------------------ autotuner
def prism_plan_autotune(plan):
    _check(load().prism_plan_autotune(plan))


def prism_plan_autotune_flags(plan, flags):
    _check(load().prism_plan_autotune_flags(plan, flags))


def prism_plan_autotune_scan(plan, probe, scan, det, out_dev):
    return _check(load().prism_plan_autotune_scan(plan, byref(probe), byref(scan), byref(det), _ptr(out_dev)))


def prism_plan_tune_result(plan, kind):
    e = PrismTuneEntry()
    _check(load().prism_plan_tune_result(plan, kind, byref(e)))
    return e


def prism_tune_shape_name(kind, shape):
    return load().prism_tune_shape_name(kind, shape).decode()


def prism_tune_shape_fft_variant(kind, shape):
    return load().prism_tune_shape_fft_variant(kind, shape)


def prism_plan_set_tune_shape(plan, kind, shape):
    _check(load().prism_plan_set_tune_shape(plan, kind, shape))


def prism_plan_load_smatrix(plan, S_dev):
    _check(load().prism_plan_load_smatrix(plan, _ptr(S_dev)))
