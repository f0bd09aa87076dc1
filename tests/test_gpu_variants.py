"""GPU parity of the method variants: tilted probes, full diffraction patterns (4D-STEM), several
probes from one S-matrix, and frozen-phonon averaging with the accumulating scan."""
import numpy as np
import pytest
import torch

from oracle import prism_oracle as O
from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300 import specimens
from paper_1702_01904_gb300.runtime import PrismSimulation, multislice

from test_gpu_parity import DET, assert_images_close, c_grid, det_c, grid_dict, rand_v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()
    yield
    torch.cuda.synchronize()


TILTED = dict(alpha_mrad=16.0, c1=25.0, c3=5.0e3, tilt_x=0.008, tilt_y=-0.005)


def cprobe(d):
    return P.make_probe(d["alpha_mrad"], d.get("c1", 0.0), d.get("c3", 0.0), d.get("tilt_x", 0.0), d.get("tilt_y", 0.0))


def test_tilted_probe_prism_and_multislice():
    g = grid_dict(64, 64, 8.0, 8.0, 3, 2.0, 2, alpha=26.0)
    V = rand_v(3, 64, 64, 21)
    rng = np.random.Generator(np.random.PCG64(22))
    x0, y0 = rng.uniform(-2, 10, 9), rng.uniform(-2, 10, 9)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    out = sim.scan(cprobe(TILTED), x0, y0, det_c(DET)).cpu().numpy()
    S, m, n = O.smatrix_build(V, g)
    assert_images_close(out, O.prism_scan(S, m, n, g, TILTED, DET, x0, y0))
    ms = multislice(c_grid(g), torch.from_numpy(V).cuda(), cprobe(TILTED), x0, y0, det_c(DET)).cpu().numpy()
    assert_images_close(ms, O.multislice_scan(V, g, TILTED, DET, x0, y0))
    sim.close()


def test_many_probes_from_one_smatrix():
    # once S is built only the coefficients change: defocus, C3, aperture and tilt (Varying Probe Size section)
    g = grid_dict(64, 64, 8.0, 8.0, 3, 2.0, 2, alpha=30.0)
    V = rand_v(3, 64, 64, 23)
    x0, y0 = np.linspace(0, 8, 7), np.linspace(1, 6, 7)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    S, m, n = O.smatrix_build(V, g)
    for pr in (dict(alpha_mrad=10.0), dict(alpha_mrad=20.0, c1=-30.0), dict(alpha_mrad=28.0, c3=2.0e4),
               dict(alpha_mrad=15.0, tilt_x=0.01)):
        out = sim.scan(cprobe(pr), x0, y0, det_c(DET)).cpu().numpy()
        assert_images_close(out, O.prism_scan(S, m, n, g, pr, DET, x0, y0))
    sim.close()


@pytest.mark.parametrize("n,cell,f", [(64, 8.0, 2), (128, 12.8, 2), (64, 8.0, 4)])
def test_cbed_matches_oracle(n, cell, f):
    g = grid_dict(n, n, cell, cell, 2, 2.0, f)
    V = rand_v(2, n, n, 24)
    rng = np.random.Generator(np.random.PCG64(25))
    x0, y0 = rng.uniform(0, cell, 11), rng.uniform(0, cell, 11)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    cb = sim.scan_cbed(cprobe(TILTED if f == 2 else dict(alpha_mrad=20.0)), x0, y0).cpu().numpy()
    S, m, nn = O.smatrix_build(V, g)
    ref = O.prism_cbed(S, m, nn, g, TILTED if f == 2 else dict(alpha_mrad=20.0), x0, y0)
    nw = n // 2 // f
    assert cb.shape == (11, nw, nw)
    # every window pixel is an image over the probes: same gate as the detector images
    assert_images_close(cb.reshape(11, -1), ref.reshape(11, -1))
    sim.close()


def test_frozen_phonon_average_with_accumulating_scan():
    base = specimens.simple_cubic(8.0, 2.0, 29)
    g = grid_dict(64, 64, 8.0, 8.0, 4, 2.0, 2)
    configs = [specimens.project_potential(specimens.displaced(base, 0.08, s), 64, 64, 4, 2.0) for s in (31, 32, 33)]
    x0, y0 = np.linspace(0.2, 7.7, 6), np.linspace(0.5, 7.1, 6)
    sim = PrismSimulation(c_grid(g))
    acc = torch.zeros((6, DET["nbins"]), device="cuda")
    for V in configs:
        sim.build(torch.from_numpy(V).cuda())
        sim.scan_accumulate(cprobe(dict(alpha_mrad=20.0)), x0, y0, det_c(DET), 1.0 / len(configs), acc)
    sim.sync()
    ref = O.frozen_phonon_scan(configs, g, dict(alpha_mrad=20.0), DET, x0, y0)
    assert_images_close(acc.cpu().numpy(), ref)
    sim.close()


def test_tilt_out_of_range_rejected():
    g = grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2)
    sim = PrismSimulation(c_grid(g))
    V = torch.zeros((1, 64, 64), device="cuda")
    sim.build(V)
    with pytest.raises(P.PrismError) as e:
        sim.scan(P.make_probe(20.0, tilt_x=0.7), [0.0], [0.0], det_c(DET))
    assert e.value.status == P.PRISM_ERR_INVALID
    sim.close()


# ------------------------------------------------------------------ separate interpolation factors f_x, f_y
def rect_grid(n, cell, H, f, fy):
    g = grid_dict(n, n, cell, cell, H, 2.0, f)
    g["f_y"] = fy
    return g, P.make_grid(n, n, H, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0, f_y=fy)


@pytest.mark.parametrize("n,cell,H,f,fy,nwx,nwy", [
    (64, 8.0, 3, 2, 1, 16, 32),
    (128, 12.8, 2, 4, 2, 16, 32),
    (128, 12.8, 2, 1, 2, 64, 32),
    (128, 12.8, 2, 2, 4, 32, 16),
])
def test_rectangular_window_scan_matches_oracle(n, cell, H, f, fy, nwx, nwy):
    g, cg = rect_grid(n, cell, H, f, fy)
    V = rand_v(H, n, n, 31)
    sim = PrismSimulation(cg)
    assert (sim.info.nw_x, sim.info.nw_y) == (nwx, nwy)
    m, nn = sim.beams()
    om, on = O.beam_set(n, n, cell, cell, 300.0, f, 20.0, fy)
    assert np.array_equal(m, om) and np.array_equal(nn, on)
    sim.build(torch.from_numpy(V).cuda())
    S, m, nn = O.smatrix_build(V, g)
    probe = dict(alpha_mrad=20.0, c1=12.0)
    # scattered, wrapped positions (probe by probe) and a ragged raster (shared union tiles)
    rng = np.random.Generator(np.random.PCG64(32))
    x0 = rng.uniform(-cell, 2 * cell, 13)
    y0 = rng.uniform(-cell, 2 * cell, 13)
    out = sim.scan(cprobe(probe), x0, y0, det_c(DET)).cpu().numpy()
    assert_images_close(out, O.prism_scan(S, m, nn, g, probe, DET, x0, y0))
    X, Y = np.meshgrid(np.arange(7) * 0.35, np.arange(3) * 0.35 + 1.0)
    out = sim.scan(cprobe(probe), X.ravel(), Y.ravel(), det_c(DET), px=7, py=3).cpu().numpy()
    assert_images_close(out, O.prism_scan(S, m, nn, g, probe, DET, X.ravel(), Y.ravel()))
    cb = sim.scan_cbed(cprobe(probe), x0[:4], y0[:4]).cpu().numpy()
    assert cb.shape == (4, nwy, nwx)
    ref = O.prism_cbed(S, m, nn, g, probe, x0[:4], y0[:4])
    assert np.linalg.norm(cb - ref) / np.linalg.norm(ref) < 1e-5
    sim.close()


def test_rectangular_window_limits():
    # 16-bit storage needs square windows; rectangular windows need sides of 16, 32 or 64
    with pytest.raises(P.PrismError) as e:
        PrismSimulation(P.make_grid(64, 64, 1, 8.0, 8.0, 2.0, 300.0, 2, 2, 0.5, 20.0,
                                    precision=P.PRISM_PRECISION_FP16X2, f_y=1))
    assert e.value.status == P.PRISM_ERR_UNSUPPORTED
    with pytest.raises(P.PrismError) as e:
        PrismSimulation(P.make_grid(256, 256, 1, 16.0, 16.0, 2.0, 300.0, 1, 2, 0.5, 20.0, f_y=2))  # 128 x 64
    assert e.value.status == P.PRISM_ERR_UNSUPPORTED
