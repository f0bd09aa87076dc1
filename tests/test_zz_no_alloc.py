"""GPU test of multislice_scan_run_noalloc, the multislice scan for callers that may not allocate
device memory themselves (for example a host application that owns the device-memory budget through
its own pool, or a latency-critical loop in which cudaMalloc / cudaFree are not allowed).

It must give the detector stack of the allocating entry point multislice_scan_run, on consecutive
calls with different inputs (the fixed scratch keeps the previous call's contents), and a call must
not change the device's free memory.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_1702_01904_gb300 import build as B
from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300 import specimens

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def ready():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    yield
    torch.cuda.synchronize()


def images_close(got, ref, rel=1e-4, floor=1e-7, abs_dim=1e-9):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    bright = ref.mean(0) >= floor
    num = np.sqrt(np.sum((got[:, bright] - ref[:, bright]) ** 2, axis=0))
    den = np.sqrt(np.sum(ref[:, bright] ** 2, axis=0))
    assert np.all(num <= rel * den)
    assert np.all(np.abs(got[:, ~bright] - ref[:, ~bright]) <= abs_dim)


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    w = specimens.workload_small()
    V = torch.from_numpy(w.potential()).cuda()
    x0, y0 = w.scan_positions()
    grid = P.grid_from_workload(w)
    det = P.make_detector(0.0, 1.0, 100)
    stream = torch.cuda.current_stream()
    calls = [(P.make_probe(20.0), np.arange(0, 256, 7)), (P.make_probe(18.0, c1=30.0), np.arange(3, 256, 11))]
    for k, (probe, sel) in enumerate(calls):
        scan = P.make_scan(len(sel), 1, x0[sel], y0[sel])
        ref = torch.empty((len(sel), 100), device="cuda")
        P.multislice_scan_run(grid, V, probe, scan, det, ref, stream, 0)
        out = torch.full((len(sel), 100), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        P.multislice_scan_run_noalloc(grid, V, probe, scan, det, out, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if k > 0:  # the first call may load the library's module (which holds the fixed array)
            assert free_after == free_before
        assert not torch.isnan(out).any()
        # same kernels with the same arguments: bitwise equal, and within the FP32 parity bar
        assert torch.equal(out, ref)
        images_close(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    grid = P.make_grid(512, 512, 8, 32.0, 32.0, 2.0, 300.0)
    V = torch.zeros((8, 512, 512), device="cuda")
    out = torch.empty((1, 10), device="cuda")
    with pytest.raises(P.PrismError) as e:
        P.multislice_scan_run_noalloc(grid, V, P.make_probe(20.0), P.make_scan(1, 1, [1.0], [1.0]),
                                      P.make_detector(0.0, 1.0, 10), out, torch.cuda.current_stream())
    assert e.value.status == P.PRISM_ERR_BUDGET
    assert "scratch" in str(e.value)
