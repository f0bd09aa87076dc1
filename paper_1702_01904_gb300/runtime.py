"""Torch-facing convenience layer over the C ABI (marshalling only; all arithmetic runs in libprism).

PyTorch provides device memory and streams; every step of the simulation runs in the library's
CUDA kernels.  Nothing here falls back to a CPU path: a missing library or GPU raises.
"""
from __future__ import annotations

import numpy as np
import torch

from . import prism as P


class _CudaView:
    """Expose a device pointer owned by the library as a zero-copy torch tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3}


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libprism needs a CUDA device; none is available")


class PrismSimulation:
    """One PRISM plan: build the compact S-matrix once, scan probes against it many times."""

    def __init__(self, grid: P.PrismGrid, hbm_budget_bytes: int = 0, stream=None):
        _require_cuda()
        P.load()
        self.grid = grid
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.plan = P.prism_plan_create(grid, hbm_budget_bytes, self.stream)
        self.info = P.prism_plan_info(self.plan)

    # -- hot path
    def build(self, V: torch.Tensor):
        assert V.is_cuda and V.dtype == torch.float32 and V.is_contiguous()
        assert tuple(V.shape) == (self.grid.n_slices, self.grid.ny, self.grid.nx)
        self._V = V  # keep alive until the stream has consumed it
        P.prism_build_smatrix(self.plan, V)

    def build_host(self, V_host: torch.Tensor):
        assert not V_host.is_cuda and V_host.dtype == torch.float32 and V_host.is_contiguous()
        P.prism_build_smatrix_host(self.plan, V_host)

    def scan(self, probe, x0, y0, det, out: torch.Tensor | None = None, px=None, py=None):
        x0 = np.ascontiguousarray(x0, np.float64)
        y0 = np.ascontiguousarray(y0, np.float64)
        n = len(x0)
        px = n if px is None else px
        py = 1 if py is None else py
        assert px * py == n
        if out is None:
            out = torch.empty((n, det.nbins), dtype=torch.float32, device="cuda")
        P.prism_scan_run(self.plan, probe, P.make_scan(px, py, x0, y0), det, out)
        return out

    def scan_host(self, probe, x0, y0, det, out_host: torch.Tensor, px=None, py=None):
        x0 = np.ascontiguousarray(x0, np.float64)
        y0 = np.ascontiguousarray(y0, np.float64)
        n = len(x0)
        px = n if px is None else px
        py = 1 if py is None else py
        P.prism_scan_run_host(self.plan, probe, P.make_scan(px, py, x0, y0), det, out_host)
        return out_host

    def scan_cbed(self, probe, x0, y0, out: torch.Tensor | None = None, px=None, py=None):
        """Full window diffraction patterns [P][nw][nw] (FFT order), units of incident intensity."""
        x0 = np.ascontiguousarray(x0, np.float64)
        y0 = np.ascontiguousarray(y0, np.float64)
        n = len(x0)
        px = n if px is None else px
        py = 1 if py is None else py
        assert px * py == n
        nw = self.info.nw_x
        if out is None:
            out = torch.empty((n, self.info.nw_y, nw), dtype=torch.float32, device="cuda")
        P.prism_scan_run_cbed(self.plan, probe, P.make_scan(px, py, x0, y0), out)
        return out

    def scan_accumulate(self, probe, x0, y0, det, weight, out: torch.Tensor, px=None, py=None):
        """out += weight * (annular bins of this S-matrix), e.g. frozen-phonon averaging."""
        x0 = np.ascontiguousarray(x0, np.float64)
        y0 = np.ascontiguousarray(y0, np.float64)
        px = len(x0) if px is None else px
        py = 1 if py is None else py
        assert px * py == len(x0)
        P.prism_scan_run_accumulate(self.plan, probe, P.make_scan(px, py, x0, y0), det, weight, out)
        return out

    def sync(self):
        P.prism_sync(self.plan)

    def autotune(self, fft_radix: bool = False):
        """Time every launch shape of the row and column passes on this plan and keep the fastest
        (prism_plan_autotune); with fft_radix also the FFT radix variants, which round differently
        (prism_plan_autotune_flags).  Returns {pass: {"chosen": name, "default": name, "ms": {name:
        ms}, "fft_variant": v}}."""
        P.prism_plan_autotune_flags(self.plan, P.PRISM_AUTOTUNE_FFT_RADIX if fft_radix else 0)
        return self.tune_result()

    def autotune_scan(self, probe, x0, y0, det, out: torch.Tensor | None = None, px=None, py=None):
        """Run this scan once per contraction tile shape of the FP32 GEMM scan, keep the fastest for
        later scans (prism_plan_autotune_scan); returns the detector stack (the same for every shape)."""
        x0 = np.ascontiguousarray(x0, np.float64)
        y0 = np.ascontiguousarray(y0, np.float64)
        n = len(x0)
        px = n if px is None else px
        py = 1 if py is None else py
        assert px * py == n
        if out is None:
            out = torch.empty((n, det.nbins), dtype=torch.float32, device="cuda")
        P.prism_plan_autotune_scan(self.plan, probe, P.make_scan(px, py, x0, y0), det, out)
        return out

    def set_shape(self, kind, shape):
        """Pin one pass's launch shape by index (prism_plan_set_tune_shape); -1 restores the default."""
        P.prism_plan_set_tune_shape(self.plan, kind, shape)

    def tune_result(self):
        out = {}
        for kind, label in ((P.PRISM_TUNE_ROW, "row"), (P.PRISM_TUNE_COL, "col"), (P.PRISM_TUNE_SCAN, "scan"),
                            (P.PRISM_TUNE_SCAN_TC, "scan_tc")):
            e = P.prism_plan_tune_result(self.plan, kind)
            name = (lambda v: P.prism_tune_shape_name(kind, v) if v >= 0 else "default")
            out[label] = {"chosen": name(e.chosen), "default": name(e.default_shape),
                          "ms": {P.prism_tune_shape_name(kind, v): e.ms[v] for v in range(e.n_shapes) if e.ms[v] >= 0}}
            if kind in (P.PRISM_TUNE_ROW, P.PRISM_TUNE_COL):
                # FFT radix variant of the shape in use (the default launcher: the default shape's)
                v = e.chosen if e.chosen >= 0 else e.default_shape
                out[label]["fft_variant"] = max(P.prism_tune_shape_fft_variant(kind, v), 0)
        return out

    # -- introspection
    def beams(self):
        return P.prism_plan_beams(self.plan)

    def smatrix(self) -> torch.Tensor:
        """Copy of the S-matrix as complex64 [B][ny_s][nx_s] (in 16-bit mode the stored values times
        their beam scales); waits for the plan's stream."""
        i = self.info
        out = torch.empty((i.n_beams, i.ny_s, i.nx_s, 2), dtype=torch.float32, device="cuda")
        torch.cuda.current_stream().synchronize()
        P.prism_plan_smatrix_copy(self.plan, out)
        self.sync()
        return torch.view_as_complex(out)

    def load_smatrix(self, S: torch.Tensor):
        """Use an S-matrix (complex64 [B][ny_s][nx_s] on the GPU, e.g. from smatrix() of a plan with the
        same grid, or loaded from a file) instead of building one (prism_plan_load_smatrix)."""
        i = self.info
        S = torch.view_as_real(S.to(torch.complex64).contiguous()) if S.is_complex() else S.contiguous()
        assert S.is_cuda and S.numel() == i.n_beams * i.ny_s * i.nx_s * 2, "S-matrix shape of this plan"
        torch.cuda.current_stream().synchronize()
        P.prism_plan_load_smatrix(self.plan, S)
        self.sync()

    def transmission(self) -> torch.Tensor:
        """Copy of the transmission functions complex64 [H][ny][nx] (waits for the plan's stream)."""
        self.sync()
        g = self.grid
        v = torch.as_tensor(_CudaView(P.prism_plan_transmission(self.plan), (g.n_slices, g.ny, g.nx, 2), "<f4"),
                            device="cuda")
        return torch.view_as_complex(v.clone())

    def set_profiling(self, on=True):
        P.prism_plan_set_profiling(self.plan, on)

    def kernel_stats(self):
        return {P.prism_kernel_name(k): P.prism_plan_kernel_stats(self.plan, k) for k in range(P.PRISM_K_COUNT)}

    def launches(self):
        return P.prism_plan_launches(self.plan)

    def reset_stats(self):
        P.prism_plan_reset_stats(self.plan)

    def close(self):
        if getattr(self, "plan", None) is not None:
            P.prism_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def multislice(grid, V: torch.Tensor, probe, x0, y0, det, stream=None, scratch_bytes=0, out=None, px=None, py=None):
    """Conventional multislice STEM of every probe position (device result [P][nbins])."""
    _require_cuda()
    x0 = np.ascontiguousarray(x0, np.float64)
    y0 = np.ascontiguousarray(y0, np.float64)
    n = len(x0)
    px = n if px is None else px
    py = 1 if py is None else py
    if out is None:
        out = torch.empty((n, det.nbins), dtype=torch.float32, device="cuda")
    stream = stream if stream is not None else torch.cuda.current_stream()
    P.multislice_scan_run(grid, V, probe, P.make_scan(px, py, x0, y0), det, out, stream, scratch_bytes)
    return out


class Batch:
    """Many independent cells (any size, slices, f, precision) as one captured CUDA graph.

    ``cells`` is a list of dicts with keys grid (PrismGrid), V (CUDA float32 tensor
    [n_slices][ny][nx]), probe, x0, y0, det and optionally px, py.  The potentials are read and the
    outputs (``self.outs[i]``, [px*py][nbins]) written at every ``run``; V's contents may change
    between runs.  ``autotune`` times each cell's pass launch shapes before the capture,
    ``fft_radix`` adds the FFT radix variants as candidates (results then agree to rounding)."""

    def __init__(self, cells, hbm_budget_bytes: int = 0, n_branches: int = 0, stream=None, autotune: bool = False,
                 fft_radix: bool = False):
        _require_cuda()
        P.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = []
        self.outs = []
        cs = []
        for c in cells:
            V = c["V"]
            assert V.is_cuda and V.dtype == torch.float32 and V.is_contiguous()
            g = c["grid"]
            assert tuple(V.shape) == (g.n_slices, g.ny, g.nx)
            x0 = np.ascontiguousarray(c["x0"], np.float64)
            y0 = np.ascontiguousarray(c["y0"], np.float64)
            px = c.get("px") or len(x0)
            py = c.get("py") or 1
            assert px * py == len(x0)
            det = c["det"]
            out = torch.empty((px * py, det.nbins), dtype=torch.float32, device="cuda")
            sc = P.make_scan(px, py, x0, y0)
            cs.append(P.make_cell(g, V, c["probe"], sc, det, out))
            self._keep.append((V, sc, g))
            self.outs.append(out)
        torch.cuda.current_stream().synchronize()
        flags = (P.PRISM_BATCH_AUTOTUNE_FFT_RADIX if fft_radix else P.PRISM_BATCH_AUTOTUNE) if autotune else 0
        self.batch = P.prism_batch_create(cs, hbm_budget_bytes, n_branches, self.stream, flags)
        self.info = P.prism_batch_info_get(self.batch)

    def run(self):
        P.prism_batch_run(self.batch)

    def sync(self):
        P.prism_batch_sync(self.batch)

    def close(self):
        if getattr(self, "batch", None) is not None:
            P.prism_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request engine (libprism's prism_server_*): submit simulation requests
    from any thread; results arrive in host arrays.  S-matrices with a non-zero key stay resident
    for later requests on the same cell."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=4):
        _require_cuda()
        P.load()
        self.srv = P.prism_server_create(hbm_budget_bytes, max_inflight)
        self._keep = {}

    def submit(self, grid, V_host, probe, x0, y0, det, key=0, px=None, py=None):
        """V_host: float32 [H][ny][nx] host tensor/array (pinned is best), kept alive until done.
        Returns (ticket, out) where out is the numpy [P][nbins] array filled on completion."""
        x0 = np.ascontiguousarray(x0, np.float64)
        y0 = np.ascontiguousarray(y0, np.float64)
        n = len(x0)
        px = n if px is None else px
        py = 1 if py is None else py
        out = np.zeros((n, det.nbins), np.float32)
        vp = V_host.data_ptr() if hasattr(V_host, "data_ptr") else V_host.ctypes.data
        req = P.PrismRequest(grid, vp, key, probe, P.make_scan(px, py, x0, y0), det, out.ctypes.data)
        t = P.prism_server_submit(self.srv, req)
        self._keep[t] = (V_host, out, grid)
        return t, out

    def wait(self, ticket, timeout_s=600.0):
        try:
            return P.prism_server_wait(self.srv, ticket, timeout_s)
        finally:
            self._keep.pop(ticket, None)

    def stats(self):
        return P.prism_server_stats(self.srv)

    def cancel(self, ticket):
        """Cancel a queued or running request: its wait() then raises PrismError(PRISM_ERR_CANCELLED)
        and its output array is left as it was."""
        P.prism_server_cancel(self.srv, ticket)

    def close(self):
        if getattr(self, "srv", None) is not None:
            P.prism_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
