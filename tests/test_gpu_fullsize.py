"""GPU parity at full size: the amorphous-carbon workload (1024^2, 50 slices, f = 8, 129 beams,
200 x 200 probes) in the launch configurations the benchmark times, and a 2048^2 cell of the large
serving workload (102.4 A, f = 8, 529 beams, 128-pixel windows).

The oracle cannot redo a whole 1024^2 or 2048^2 job, so each test compares sampled outputs that the
oracle computes one by one: single probes of multislice (``multislice_probe``), single PRISM probes
by linearity of Eq. PRISMfinal (``prism_probe_direct``: one multislice of the probe's d/f-periodic
incident wave, stored, windowed and binned as the S-matrix scan does) and single S-matrix beams.
The oracle runs in spawned worker processes (``oracle_pool``).  Bars: relative L2 <= 1e-4 per
detector image over the sampled probes for images of oracle mean >= 1e-7, absolute error <= 1e-9
below; S-matrix beams relative L2 <= 5e-5 (50 slices of FP32 FFT pairs).
"""
import numpy as np
import pytest
import torch

import oracle_pool
from oracle import prism_oracle as O
from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300 import specimens
from paper_1702_01904_gb300.runtime import PrismSimulation, multislice

pytestmark = pytest.mark.gpu

DET = dict(start_mrad=0.0, step_mrad=1.0, nbins=100)


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    yield
    torch.cuda.synchronize()


def grid_of(w):
    return dict(nx=w.nx, ny=w.ny, cell_x=w.cell_x, cell_y=w.cell_y, n_slices=w.n_slices, dz=w.dz, kv=w.kv,
                f=w.f, downsample=w.downsample, aa_frac=w.aa_frac, alpha_mrad=w.alpha_mrad)


def det_c():
    return P.make_detector(DET["start_mrad"], DET["step_mrad"], DET["nbins"])


def assert_images_close(gpu, ref, rel=1e-4, floor=1e-7, abs_dim=1e-9):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape
    bright = ref.mean(0) >= floor
    assert bright.sum() >= 10
    err = O.rel_l2_per_image(gpu[:, bright], ref[:, bright])
    assert err.max() <= rel, f"max rel L2 {err.max():.3e} at bin {np.flatnonzero(bright)[err.argmax()]}"
    if (~bright).any():
        assert np.max(np.abs(gpu[:, ~bright] - ref[:, ~bright])) <= abs_dim


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def carbon():
    w = specimens.workload_amorphous_carbon()
    return w, w.potential()


# probes of the 200 x 200 raster (row-major [iy][ix]) sampled for the PRISM scans: the four corners
# (windows wrapping across both cell edges), both sides of raster-block boundaries, the last block row
# (rows 192-199, whose blocks the persistent grid's last round splits over idle CTAs) and scattered
# interior probes
def carbon_probe_sample():
    pts = [(0, 0), (0, 199), (199, 0), (199, 199),            # corners
           (7, 3), (8, 4), (7, 4), (8, 3),                    # across 8 x 4 / 4 x 8 block edges
           (192, 64), (193, 100), (195, 130), (196, 150),     # the split last round
           (197, 171), (198, 188), (199, 64), (192, 199),
           (100, 100), (57, 13), (31, 177), (150, 42), (120, 121), (3, 96), (88, 0), (176, 55)]
    return [iy * 200 + ix for iy, ix in pts]


def test_carbon_prism_scan_sampled_fp32_and_fp16x2(carbon):
    """The headline step: S-matrix build and 40 000-probe FP32 scan, plus the same scan by the
    tensor-core path in its FP32-class mode, against the oracle on 24 probes and 2 beams."""
    w, V = carbon
    g = grid_of(w)
    x0, y0 = w.scan_positions()
    probe = P.make_probe(w.alpha_mrad)
    Vd = torch.from_numpy(V).cuda()
    sel = carbon_probe_sample()
    items = [(dict(alpha_mrad=w.alpha_mrad), DET, float(x0[i]), float(y0[i])) for i in sel]

    sim = PrismSimulation(P.grid_from_workload(w))
    assert sim.info.n_beams == 129 and sim.info.nw_x == 64
    sim.build(Vd)
    out = sim.scan(probe, x0, y0, det_c(), px=w.scan_px, py=w.scan_py).cpu().numpy()
    S = sim.smatrix()
    m, nn = sim.beams()
    beams = (0, 64, 128)
    S_b = [S[b].cpu().numpy() for b in beams]
    sim.close()
    del S

    tsim = PrismSimulation(P.grid_from_workload(w, precision=P.PRISM_PRECISION_FP16X2))
    tsim.build(Vd)
    tout = tsim.scan(probe, x0, y0, det_c(), px=w.scan_px, py=w.scan_py).cpu().numpy()
    tsim.close()

    ref = np.array(oracle_pool.evaluate("prism", V, g, items))
    ref_beams = oracle_pool.evaluate("beam", V, g, [(int(m[b]), int(nn[b])) for b in beams])
    for got, want in zip(S_b, ref_beams):
        assert rel_l2(got, want) < 5e-5
    assert_images_close(out[sel], ref)
    assert_images_close(tout[sel], ref)
    # every probe's binned intensity is the incident one up to PRISM's crop approximation
    tot = out.sum(1)
    assert np.all(tot > 0.98) and np.all(tot < 1.01)


def test_carbon_multislice_bench_config_sampled(carbon):
    """The multislice baseline exactly as the benchmark runs it (1024 probes spread over the raster,
    2 GiB of scratch: four batches of 256 probes), 8 probes against the oracle: the first and last
    probe of each batch edge, the raster origin (a probe wrapping across both cell edges) and the
    last raster probe."""
    w, V = carbon
    g = grid_of(w)
    x0, y0 = w.scan_positions()
    probe = P.make_probe(w.alpha_mrad)
    Vd = torch.from_numpy(V).cuda()
    nms = 1024
    sel = np.linspace(0, len(x0) - 1, nms).astype(np.int64)
    out = multislice(P.grid_from_workload(w), Vd, probe, x0[sel], y0[sel], det_c(),
                     scratch_bytes=2 << 30).cpu().numpy()
    pick = [0, 255, 256, 511, 512, 700, 1022, 1023]
    items = [(dict(alpha_mrad=w.alpha_mrad), DET, float(x0[sel[k]]), float(y0[sel[k]])) for k in pick]
    ref = np.array(oracle_pool.evaluate("multislice", V, g, items))
    assert_images_close(out[pick], ref)
    # multislice conserves the incident intensity up to what leaves the anti-aliasing aperture
    tot = out.sum(1)
    assert np.all(tot > 0.95) and np.all(tot <= 1.0 + 1e-4)


@pytest.fixture(scope="module")
def cell_2048():
    # 6 slices of the large serving cell: an 8 A Au cluster over 4 A of amorphous carbon
    w = specimens.workload_nanoparticle_on_carbon(n_slices=6, particle_diameter=8.0)
    V = specimens.project_potential_vectorised(w.specimen, w.nx, w.ny, w.n_slices, w.dz)
    return w, V


def test_2048_cell_prism_and_multislice_sampled(cell_2048):
    """N = 2048 passes, 529 beams and 128-pixel windows: 2 S-matrix beams, 8 PRISM probes of a
    24 x 24 raster that wraps across the cell edge, and 2 multislice probes, against the oracle."""
    w, V = cell_2048
    g = grid_of(w)
    probe = P.make_probe(w.alpha_mrad)
    Vd = torch.from_numpy(V).cuda()
    sim = PrismSimulation(P.grid_from_workload(w))
    assert sim.info.n_beams == 529 and sim.info.nw_x == 128 and sim.info.nx_s == 1024
    sim.build(Vd)
    m, nn = sim.beams()
    xs = (95.0 + 0.35 * np.arange(24)) % w.cell_x      # crosses x = 102.4 -> 0
    ys = 40.0 + 0.3 * np.arange(24)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    x0, y0 = xx.ravel(), yy.ravel()
    out = sim.scan(probe, x0, y0, det_c(), px=24, py=24).cpu().numpy()
    beams = (0, 264)
    S_b = [sim.smatrix()[b].cpu().numpy() for b in beams]
    sim.close()
    pick = [0, 23, 24, 300, 551, 575, 21 + 24 * 5, 22 + 24 * 17]
    items = [(dict(alpha_mrad=w.alpha_mrad), DET, float(x0[k]), float(y0[k])) for k in pick]
    ref = np.array(oracle_pool.evaluate("prism", V, g, items))
    assert_images_close(out[pick], ref)
    ref_beams = oracle_pool.evaluate("beam", V, g, [(int(m[b]), int(nn[b])) for b in beams])
    for got, want in zip(S_b, ref_beams):
        assert rel_l2(got, want) < 2e-5
    mx, my = np.array([101.9, 51.2]), np.array([0.1, 77.7])
    ms = multislice(P.grid_from_workload(w), Vd, probe, mx, my, det_c()).cpu().numpy()
    mref = np.array(oracle_pool.evaluate("multislice", V, g, [(dict(alpha_mrad=w.alpha_mrad), DET, float(a), float(b))
                                                             for a, b in zip(mx, my)]))
    assert_images_close(ms, mref)
