"""C-ABI checks that need no GPU: the library builds and loads, exports every entry point the
header declares, and the ctypes binding matches the header's constants and struct layouts."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1702_01904_gb300 import build as B
from paper_1702_01904_gb300 import prism as P

HEADER = os.path.join(B.INCLUDE, "prism.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:prism|multislice)_\w+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = header_functions()
    assert "prism_plan_create" in names and "multislice_scan_run" in names
    assert sorted(P.EXPORTED) == names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_sets_signatures(lib):
    L = P.load()
    for name in P.EXPORTED:
        assert getattr(L, name).argtypes is not None or name == "prism_last_error"


def test_status_and_kernel_constants_match_header():
    src = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(PRISM_\w+)\s+(-?\d+)", src))
    for k, v in defs.items():
        assert getattr(P, k) == int(v), k


def test_struct_layout_matches_c(tmp_path):
    probe = tmp_path / "layout.c"
    probe.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "prism.h"
#define F(s, m) printf(#s "." #m " %zu\\n", offsetof(s, m));
int main(void) {
  printf("prism_grid %zu\\n", sizeof(prism_grid));
  printf("prism_probe %zu\\n", sizeof(prism_probe));
  printf("prism_scan %zu\\n", sizeof(prism_scan));
  printf("prism_detector %zu\\n", sizeof(prism_detector));
  printf("prism_info %zu\\n", sizeof(prism_info));
  F(prism_grid, cell_x) F(prism_grid, slice_dz) F(prism_grid, kv) F(prism_grid, f) F(prism_grid, aa_frac)
  F(prism_grid, alpha_max_mrad) F(prism_grid, precision) F(prism_grid, f_y) F(prism_scan, x0) F(prism_scan, y0) F(prism_detector, nbins)
  F(prism_info, wavelength) F(prism_info, device_bytes)
  printf("prism_cell %zu\\n", sizeof(prism_cell));
  printf("prism_batch_info %zu\\n", sizeof(prism_batch_info));
  F(prism_cell, V_dev) F(prism_cell, probe) F(prism_cell, scan) F(prism_cell, det) F(prism_cell, out_dev)
  F(prism_batch_info, graph_nodes) F(prism_batch_info, kernel_launches) F(prism_batch_info, device_bytes)
  printf("prism_tune_entry %zu\\n", sizeof(prism_tune_entry));
  F(prism_tune_entry, default_shape) F(prism_tune_entry, ms)
  printf("prism_request %zu\\n", sizeof(prism_request));
  printf("prism_request_stats %zu\\n", sizeof(prism_request_stats));
  printf("prism_server_info %zu\\n", sizeof(prism_server_info));
  F(prism_request, V_host) F(prism_request, smatrix_key) F(prism_request, probe) F(prism_request, scan)
  F(prism_request, det) F(prism_request, out_host)
  F(prism_request_stats, status) F(prism_request_stats, device_start_ms) F(prism_request_stats, device_end_ms)
  F(prism_server_info, admitted) F(prism_server_info, peak_bytes)
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", B.INCLUDE, str(probe), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                check=True).stdout.split("\n") if line)
    cls = {"prism_grid": P.PrismGrid, "prism_probe": P.PrismProbe, "prism_scan": P.PrismScan,
           "prism_detector": P.PrismDetector, "prism_info": P.PrismInfo, "prism_cell": P.PrismCell,
           "prism_batch_info": P.PrismBatchInfo, "prism_tune_entry": P.PrismTuneEntry,
           "prism_request": P.PrismRequest, "prism_request_stats": P.PrismRequestStats,
           "prism_server_info": P.PrismServerInfo}
    for k, v in out.items():
        if "." in k:
            s, m = k.split(".")
            assert getattr(cls[s], m).offset == int(v), k
        else:
            assert ctypes.sizeof(cls[k]) == int(v), k


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(RuntimeError):
        P.load(str(tmp_path / "nope.so"))


def test_plan_arguments_rejected_before_any_device_call():
    """Argument checks of prism_plan_create run on the host before the first CUDA call."""
    def status(**over):
        g = P.make_grid(64, 64, 1, 8.0, 8.0, 2.0, 300.0, 2, 2, 0.5, 20.0)
        for k, v in over.items():
            setattr(g, k, v)
        with pytest.raises(P.PrismError) as e:
            P.prism_plan_create(g)
        return e.value.status
    assert status(precision=4) == P.PRISM_ERR_INVALID
    assert status(precision=-1) == P.PRISM_ERR_INVALID
    # 16-bit S needs a 16, 32 or 64 pixel window: 64 px / 2 / f=4 is 8
    assert status(precision=P.PRISM_PRECISION_FP16, f=4) == P.PRISM_ERR_UNSUPPORTED
    assert status(precision=P.PRISM_PRECISION_BF16, f=4) == P.PRISM_ERR_UNSUPPORTED
    assert status(precision=P.PRISM_PRECISION_FP16X2, f=4) == P.PRISM_ERR_UNSUPPORTED
    assert status(nx=100) == P.PRISM_ERR_UNSUPPORTED
    assert status(f=0) == P.PRISM_ERR_INVALID
    assert status(f_y=-1) == P.PRISM_ERR_INVALID
    assert status(f_y=3) == P.PRISM_ERR_INVALID            # 64 not divisible by 2 * 3
    assert status(f_y=1, precision=P.PRISM_PRECISION_FP16) == P.PRISM_ERR_UNSUPPORTED  # 16 x 32 window
    assert status(f=1, f_y=8) == P.PRISM_ERR_UNSUPPORTED  # 32 x 4 window


def test_bounded_wait_selftest_rejects_a_null_status():
    with pytest.raises(P.PrismError) as e:
        P.prism_selftest_bounded_wait(None, 1000, 0)
    assert e.value.status == P.PRISM_ERR_INVALID


def test_tune_shape_arguments_rejected_without_a_device():
    """prism_plan_set_tune_shape checks its plan and pass on the host."""
    with pytest.raises(P.PrismError) as e:
        P.prism_plan_set_tune_shape(None, P.PRISM_TUNE_COL, 0)
    assert e.value.status == P.PRISM_ERR_INVALID
    names = [P.prism_tune_shape_name(P.PRISM_TUNE_COL, v) for v in range(P.PRISM_TUNE_MAX_SHAPES)]
    assert "W8, TMA" in names and "W8, staged" in names


def test_tune_shapes_list_both_fft_radix_variants():
    """Each pass lists launch shapes of both FFT radix variants (the split of the 32- and 64-point
    register DFTs); the defaults are variant 0, other kinds and unknown shapes report -1."""
    for kind in (P.PRISM_TUNE_ROW, P.PRISM_TUNE_COL):
        rv = {}
        for v in range(P.PRISM_TUNE_MAX_SHAPES):
            name = P.prism_tune_shape_name(kind, v)
            if name == "?":
                assert P.prism_tune_shape_fft_variant(kind, v) == -1
                continue
            rv[name] = P.prism_tune_shape_fft_variant(kind, v)
        assert set(rv.values()) == {0, 1, 2, 3}  # forward (bit 0) and inverse (bit 1) split
        assert all(("radix-4 first" in n) == (r != 0) for n, r in rv.items())
        assert all(n.endswith({1: "forward", 2: "inverse", 3: "both"}[r]) for n, r in rv.items() if r)
    assert rv["W4, TMA, 3/SM"] == 0 and rv["W8, staged"] == 0
    assert P.prism_tune_shape_fft_variant(P.PRISM_TUNE_SCAN, 0) == -1
    assert [P.prism_tune_shape_name(P.PRISM_TUNE_SCAN_TC, v) for v in range(4)] == [
        "3 x 96 K ring", "2 x 128 K ring", "4 x 64 K ring", "?"]
    with pytest.raises(P.PrismError) as e:
        P.prism_plan_autotune_flags(None, P.PRISM_AUTOTUNE_FFT_RADIX)
    assert e.value.status == P.PRISM_ERR_INVALID
    assert P.prism_tune_shape_fft_variant(P.PRISM_TUNE_ROW, P.PRISM_TUNE_MAX_SHAPES) == -1


def test_no_cpu_fallback_without_a_gpu():
    """The torch-facing layer refuses to run without a CUDA device instead of falling back to a
    host path (there is none)."""
    import torch
    from paper_1702_01904_gb300 import runtime
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = P.make_grid(64, 64, 1, 8.0, 8.0, 2.0, 300.0, 2, 2, 0.5, 20.0)
    with pytest.raises(RuntimeError):
        runtime.PrismSimulation(g)
    with pytest.raises(RuntimeError):
        runtime.multislice(g, torch.zeros(1, 64, 64), P.make_probe(20.0), np.zeros(1), np.zeros(1),
                           P.make_detector(0.0, 1.0, 10))


@pytest.mark.parametrize("f,f_y,cell_x,cell_y,alpha,tx,ty", [
    (8, 0, 50.0, 50.0, 20.0, 0.0, 0.0),
    (4, 0, 16.0, 16.0, 20.0, 0.004, -0.003),
    (3, 2, 12.0, 8.0, 15.0, -0.006, 0.002),
])
def test_recommended_alpha_max_keeps_the_tilted_aperture_with_a_lattice_step_margin(f, f_y, cell_x, cell_y, alpha, tx, ty):
    # the beam set of radius alpha_max (PRISM Algorithm section) must hold every lattice beam whose
    # frequency lies within one lattice step of the tilted probe aperture lambda |q - q_t| <= alpha
    from oracle import prism_oracle as O
    kv = 300.0
    g = P.make_grid(256, 256, 1, cell_x, cell_y, 2.0, kv, f, 2, 0.5, 0.0, f_y=f_y)
    amax = P.prism_recommended_alpha_max(g, P.make_probe(alpha, tilt_x=tx, tilt_y=ty))
    lam = O.wavelength(kv)
    fy = f_y or f
    m, n = O.beam_set(256, 256, cell_x, cell_y, kv, f, amax, fy)
    have = set(zip(m.tolist(), n.tolist()))
    step = max(f / cell_x, fy / cell_y)  # the coarser lattice step (1/A)
    qtx, qty = tx / lam, ty / lam
    r = int(amax / (1000 * lam * min(f / cell_x, fy / cell_y))) + 2
    needed = 0
    for mm in range(-r, r + 1):
        for nn in range(-r, r + 1):
            qx, qy = mm * f / cell_x, nn * fy / cell_y
            if math.hypot(qx - qtx, qy - qty) <= alpha * 1e-3 / lam + step * (1 - 1e-9):
                needed += 1
                assert (mm, nn) in have, (mm, nn)
    assert needed > 0


def test_recommended_alpha_max_rejects_bad_arguments():
    g = P.make_grid(64, 64, 1, 8.0, 8.0, 2.0, 300.0, 0)
    with pytest.raises(P.PrismError) as e:
        P.prism_recommended_alpha_max(g, P.make_probe(20.0))
    assert e.value.status == P.PRISM_ERR_INVALID
    g = P.make_grid(64, 64, 1, 8.0, 8.0, 2.0, 300.0, 2)
    with pytest.raises(P.PrismError):
        P.prism_recommended_alpha_max(g, P.make_probe(-1.0))
