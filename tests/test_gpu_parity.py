"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Bars (per detector image = one bin over all probes): relative L2 <= 1e-4 for images whose oracle
mean is >= 1e-7 of the incident intensity, absolute error <= 1e-9 for dimmer images; integer
decisions (beam set) bit-exact.  Intermediate S-matrices: relative L2 per beam <= 2e-5 (8 slices)
or 5e-5 (50 slices), from the FP32 error of two FFT pairs per slice.
"""
import math

import numpy as np
import pytest
import torch

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
    torch.cuda.init()
    yield
    torch.cuda.synchronize()


def grid_dict(nx, ny, cx, cy, H, dz, f, ds=2, aa=0.5, alpha=20.0, kv=300.0, slice_dz=None):
    d = dict(nx=nx, ny=ny, cell_x=cx, cell_y=cy, n_slices=H, dz=dz, kv=kv, f=f, downsample=ds,
             aa_frac=aa, alpha_mrad=alpha)
    if slice_dz is not None:
        d["slice_dz"] = list(slice_dz)
    return d


def c_grid(g):
    return P.make_grid(g["nx"], g["ny"], g["n_slices"], g["cell_x"], g["cell_y"], g["dz"], g["kv"], g["f"],
                       g["downsample"], g["aa_frac"], g["alpha_mrad"], slice_dz=g.get("slice_dz"))


def rand_v(H, ny, nx, seed, amp=120.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (amp * rng.random((H, ny, nx))).astype(np.float32)


def det_c(d):
    return P.make_detector(d["start_mrad"], d["step_mrad"], d["nbins"])


def assert_images_close(gpu, ref, rel=1e-4, floor=1e-7, abs_dim=1e-9):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape
    bright = ref.mean(0) >= floor
    if bright.any():
        err = O.rel_l2_per_image(gpu[:, bright], ref[:, bright])
        assert err.max() <= rel, f"max rel L2 {err.max():.3e} at bin {np.flatnonzero(bright)[err.argmax()]}"
    if (~bright).any():
        assert np.max(np.abs(gpu[:, ~bright] - ref[:, ~bright])) <= abs_dim
    return gpu


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def run_prism(g, V, probe, x0, y0, det, budget=0):
    sim = PrismSimulation(c_grid(g), budget)
    sim.build(torch.from_numpy(V).cuda())
    out = sim.scan(probe, x0, y0, det_c(det))
    sim.sync()
    return sim, out.cpu().numpy()


# ------------------------------------------------------------------ constants and integer decisions
def test_constants_bit_exact():
    for kv in (80.0, 200.0, 300.0):
        assert P.prism_wavelength(kv) == O.wavelength(kv)
        assert P.prism_interaction_constant(kv) == O.interaction_constant(kv)


@pytest.mark.parametrize("n,cell,f", [(256, 16.0, 4), (1024, 50.0, 8), (64, 8.0, 2), (128, 12.8, 1)])
def test_beam_set_bit_exact(n, cell, f):
    sim = PrismSimulation(c_grid(grid_dict(n, n, cell, cell, 1, 2.0, f, ds=2 if n // 2 // f <= 128 else 1)))
    m, nn = sim.beams()
    om, on = O.beam_set(n, n, cell, cell, 300.0, f, 20.0)
    assert np.array_equal(m, om) and np.array_equal(nn, on)
    sim.close()


def test_transmission_matches_oracle():
    g = grid_dict(64, 64, 8.0, 8.0, 3, 2.0, 2)
    V = rand_v(3, 64, 64, 1, amp=4000.0)   # phases up to ~2.6 rad
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    t = sim.transmission().cpu().numpy()
    assert np.max(np.abs(t - O.transmission(V, 300.0))) < 1e-6


# ------------------------------------------------------------------ S-matrix parity
@pytest.mark.parametrize("case", [
    dict(n=64, cell=8.0, H=3, f=2, ds=2),
    dict(n=64, cell=6.4, H=2, f=1, ds=1),
    dict(n=32, cell=4.0, H=1, f=1, ds=2),
    dict(n=128, cell=12.8, H=2, f=4, ds=2, slice_dz=[1.0, 3.5]),
    dict(n=16, cell=2.0, H=2, f=1, ds=2, alpha=20.0),
])
def test_smatrix_matches_oracle(case):
    n = case["n"]
    g = grid_dict(n, n, case["cell"], case["cell"], case["H"], 2.0, case["f"], ds=case["ds"],
                  alpha=case.get("alpha", 20.0), slice_dz=case.get("slice_dz"))
    V = rand_v(case["H"], n, n, 2)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    S = sim.smatrix().cpu().numpy()
    So, _, _ = O.smatrix_build(V, g)
    assert S.shape == So.shape
    for b in range(len(So)):
        assert rel_l2(S[b], So[b]) < 2e-5, b
    sim.close()


def test_smatrix_rectangular_cell():
    g = grid_dict(64, 64, 8.0, 6.4, 2, 2.0, 2)
    V = rand_v(2, 64, 64, 3)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    S = sim.smatrix().cpu().numpy()
    So, om, on = O.smatrix_build(V, g)
    m, nn = sim.beams()
    assert np.array_equal(m, om) and np.array_equal(nn, on)
    assert max(rel_l2(S[b], So[b]) for b in range(len(So))) < 2e-5


# ------------------------------------------------------------------ end-to-end PRISM and multislice, small configs
@pytest.mark.parametrize("case", [
    dict(n=64, cell=8.0, H=3, f=2, ds=2, nw=16),
    dict(n=64, cell=8.0, H=2, f=4, ds=2, nw=8),
    dict(n=64, cell=6.4, H=2, f=1, ds=2, nw=32),
    dict(n=128, cell=12.8, H=2, f=1, ds=2, nw=64),
    dict(n=128, cell=12.8, H=1, f=1, ds=1, nw=128),
])
def test_prism_scan_matches_oracle(case):
    n = case["n"]
    g = grid_dict(n, n, case["cell"], case["cell"], case["H"], 2.0, case["f"], ds=case["ds"])
    V = rand_v(case["H"], n, n, 4)
    rng = np.random.Generator(np.random.PCG64(5))
    x0 = rng.uniform(-case["cell"], 2 * case["cell"], 21)   # ragged count, wrapped positions
    y0 = rng.uniform(-case["cell"], 2 * case["cell"], 21)
    probe = P.make_probe(20.0, c1=15.0, c3=2.0e4)
    sim, out = run_prism(g, V, probe, x0, y0, DET)
    assert sim.info.nw_x == case["nw"]
    S, m, nn = O.smatrix_build(V, g)
    ref = O.prism_scan(S, m, nn, g, dict(alpha_mrad=20.0, c1=15.0, c3=2.0e4), DET, x0, y0)
    assert_images_close(out, ref)
    sim.close()


def test_prism_f1_equals_multislice_on_gpu():
    g = grid_dict(64, 64, 6.4, 6.4, 3, 2.0, 1, ds=2)
    V = rand_v(3, 64, 64, 6)
    x0 = np.array([0.0, 1.3, 4.4, 6.1])
    y0 = np.array([0.2, 5.0, 2.2, 3.3])
    probe = P.make_probe(20.0)
    sim, pr = run_prism(g, V, probe, x0, y0, DET)
    ms = multislice(c_grid(g), torch.from_numpy(V).cuda(), probe, x0, y0, det_c(DET)).cpu().numpy()
    assert_images_close(pr, ms)
    sim.close()


@pytest.mark.parametrize("case", [
    dict(nx=64, ny=64, cx=8.0, cy=8.0, H=3),
    dict(nx=128, ny=64, cx=12.8, cy=8.0, H=2),
    dict(nx=32, ny=64, cx=4.0, cy=8.0, H=2, slice_dz=[2.0, 0.5]),
])
def test_multislice_matches_oracle(case):
    g = grid_dict(case["nx"], case["ny"], case["cx"], case["cy"], case["H"], 2.0, 1, slice_dz=case.get("slice_dz"))
    V = rand_v(case["H"], case["ny"], case["nx"], 7)
    rng = np.random.Generator(np.random.PCG64(8))
    x0 = rng.uniform(0, case["cx"], 5)
    y0 = rng.uniform(0, case["cy"], 5)
    out = multislice(c_grid(g), torch.from_numpy(V).cuda(), P.make_probe(20.0, c1=-20.0), x0, y0,
                     det_c(DET), scratch_bytes=2 * case["nx"] * case["ny"] * 8).cpu().numpy()
    ref = O.multislice_scan(V, g, dict(alpha_mrad=20.0, c1=-20.0, c3=0.0), DET, x0, y0)
    assert_images_close(out, ref)


# ------------------------------------------------------------------ the small published-shape workload, in full
@pytest.fixture(scope="module")
def small_workload():
    w = specimens.workload_small()
    V = w.potential()
    g = grid_dict(w.nx, w.ny, w.cell_x, w.cell_y, w.n_slices, w.dz, w.f, ds=w.downsample, alpha=w.alpha_mrad)
    x0, y0 = w.scan_positions()
    return w, V, g, x0, y0


def test_small_workload_smatrix_and_scan(small_workload):
    w, V, g, x0, y0 = small_workload
    probe = P.make_probe(w.alpha_mrad)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    out = sim.scan(probe, x0, y0, det_c(DET), px=w.scan_px, py=w.scan_py).cpu().numpy()
    S = sim.smatrix().cpu().numpy()
    So, m, nn = O.smatrix_build(V, g)
    assert len(So) == 49
    assert max(rel_l2(S[b], So[b]) for b in range(len(So))) < 2e-5
    ref = O.prism_scan(So, m, nn, g, dict(alpha_mrad=w.alpha_mrad), DET, x0, y0)
    assert_images_close(out, ref)
    sim.close()


def test_small_workload_multislice(small_workload):
    w, V, g, x0, y0 = small_workload
    sel = np.arange(0, len(x0), 17)
    out = multislice(c_grid(g), torch.from_numpy(V).cuda(), P.make_probe(w.alpha_mrad), x0[sel], y0[sel],
                     det_c(DET)).cpu().numpy()
    ref = O.multislice_scan(V, g, dict(alpha_mrad=w.alpha_mrad), DET, x0[sel], y0[sel])
    assert_images_close(out, ref)


# The amorphous-carbon workload at full size (sampled against the oracle) is in test_gpu_fullsize.py.


# ------------------------------------------------------------------ properties, edge cases, errors
def test_batched_build_is_bitwise_identical():
    g = grid_dict(64, 64, 8.0, 8.0, 3, 2.0, 2)
    V = rand_v(3, 64, 64, 9)
    x0 = np.linspace(0, 8, 9)
    y0 = np.linspace(1, 7, 9)
    probe = P.make_probe(20.0)
    full, a = run_prism(g, V, probe, x0, y0, DET)
    # plan memory: t_p of the 3 slices, the row transform of t_0, the FP32 S, 1 MiB; then one wave per beam
    need = 3 * 64 * 64 * 8 + 64 * 64 * 8 + full.info.n_beams * 32 * 32 * 8 + (1 << 20)
    small, b = run_prism(g, V, probe, x0, y0, DET, budget=need + 5 * 64 * 64 * 8)
    assert small.info.beam_batch == 5 < full.info.n_beams
    assert np.array_equal(a, b)
    assert np.array_equal(full.smatrix().cpu().numpy(), small.smatrix().cpu().numpy())


def test_deterministic_and_host_variants_identical():
    g = grid_dict(64, 64, 8.0, 8.0, 2, 2.0, 2)
    V = rand_v(2, 64, 64, 10)
    x0 = np.linspace(-3, 11, 15)
    y0 = np.linspace(2, 5, 15)
    probe = P.make_probe(20.0, c1=10.0)
    sim, a = run_prism(g, V, probe, x0, y0, DET)
    b = sim.scan(probe, x0, y0, det_c(DET)).cpu().numpy()
    sim2 = PrismSimulation(c_grid(g))
    sim2.build_host(torch.from_numpy(V).pin_memory())
    host = torch.empty((15, DET["nbins"]), dtype=torch.float32).pin_memory()
    sim2.scan_host(probe, x0, y0, det_c(DET), host)
    sim2.sync()
    assert np.array_equal(a, b) and np.array_equal(a, host.numpy())


def test_host_build_chunks_and_rebuild_identical():
    # host-buffer builds copy the potential in chunks of slices (here 9 slices: chunks of 2, the
    # last ragged) on their own stream; two builds back to back reuse the staging buffer, and a
    # small HBM budget splits the beams into batches: every result equals the device-buffer build
    g = grid_dict(64, 64, 8.0, 8.0, 9, 2.0, 2)
    V1 = rand_v(9, 64, 64, 21)
    V2 = rand_v(9, 64, 64, 22)
    x0 = np.linspace(0.5, 7.5, 12)
    y0 = np.linspace(1.0, 6.0, 12)
    probe = P.make_probe(20.0)
    full, ref = run_prism(g, V2, probe, x0, y0, DET)
    # plan memory: t_p of every slice, the row transform of t_0, the FP32 S, 1 MiB; then one wave per
    # beam of a batch
    small = 9 * 64 * 64 * 8 + 64 * 64 * 8 + full.info.n_beams * 32 * 32 * 8 + (1 << 20) + 5 * 64 * 64 * 8
    for budget, batch in ((0, full.info.n_beams), (small, 5)):
        sim = PrismSimulation(c_grid(g), budget)
        assert sim.info.beam_batch == batch
        sim.build_host(torch.from_numpy(V1).pin_memory())
        sim.build_host(torch.from_numpy(V2).pin_memory())
        host = torch.empty((12, DET["nbins"]), dtype=torch.float32).pin_memory()
        sim.scan_host(probe, x0, y0, det_c(DET), host)
        sim.sync()
        assert np.array_equal(ref, host.numpy())
        sim.close()


def test_scan_partition_invariant():
    # a probe's result does not depend on which raster block or part of a split block computed it:
    # a 160 x 64 raster (320 blocks of 4 x 8: 304 whole on the persistent grid, the last 16 split)
    # equals the same raster scanned as 8 bands of 8 rows (40 blocks each, all split) and as 64
    # single rows, bitwise; sampled probes match the oracle
    g = grid_dict(64, 64, 8.0, 8.0, 3, 2.0, 2)
    V = rand_v(3, 64, 64, 31)
    xs, ys = np.meshgrid(np.arange(160) * 0.05, 0.5 + np.arange(64) * 0.11)
    x0, y0 = xs.ravel(), ys.ravel()
    probe = P.make_probe(20.0)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    whole = sim.scan(probe, x0, y0, det_c(DET), px=160, py=64).cpu().numpy()
    bands = np.concatenate([sim.scan(probe, x0[r * 1280:(r + 1) * 1280], y0[r * 1280:(r + 1) * 1280], det_c(DET),
                                     px=160, py=8).cpu().numpy() for r in range(8)])
    rows = np.concatenate([sim.scan(probe, x0[r * 160:(r + 1) * 160], y0[r * 160:(r + 1) * 160], det_c(DET),
                                    px=160, py=1).cpu().numpy() for r in range(64)])
    assert np.array_equal(whole, bands) and np.array_equal(whole, rows)
    S, m, nn = O.smatrix_build(V, g)
    sel = np.array([0, 159, 5000, 10079, 10239])
    ref = O.prism_scan(S, m, nn, g, dict(alpha_mrad=20.0), DET, x0[sel], y0[sel])
    assert_images_close(whole[sel], ref)
    sim.close()


@pytest.mark.parametrize("prec", [P.PRISM_PRECISION_FP32, P.PRISM_PRECISION_FP16])
def test_scans_of_other_grid_sizes_leave_the_unit_counters_zero(prec):
    # the scans take their work units from a counter placed after one split counter per CTA, so its
    # place moves with the grid; a full-grid scan (160 x 64 raster) and a one-block scan (4 x 8
    # probes: a grid of 16 CTAs, one split block) alternate on one plan, and every repeat equals the
    # first run bitwise (a counter left non-zero would skip units)
    g = grid_dict(64, 64, 8.0, 8.0, 2, 2.0, 2)
    V = rand_v(2, 64, 64, 37)
    xs, ys = np.meshgrid(np.arange(160) * 0.05, 0.5 + np.arange(64) * 0.11)
    xb, yb = xs.ravel(), ys.ravel()
    xs1, ys1 = np.meshgrid(1.0 + np.arange(4) * 0.25, 2.0 + np.arange(8) * 0.25)
    xt, yt = xs1.ravel(), ys1.ravel()
    probe = P.make_probe(20.0)
    sim = PrismSimulation(P.make_grid(64, 64, 2, 8.0, 8.0, 2.0, 300.0, 2, 2, 0.5, 20.0, precision=prec))
    sim.build(torch.from_numpy(V).cuda())
    big = sim.scan(probe, xb, yb, det_c(DET), px=160, py=64).cpu().numpy()
    small = sim.scan(probe, xt, yt, det_c(DET), px=4, py=8).cpu().numpy()
    for _ in range(2):
        assert np.array_equal(sim.scan(probe, xb, yb, det_c(DET), px=160, py=64).cpu().numpy(), big)
        assert np.array_equal(sim.scan(probe, xt, yt, det_c(DET), px=4, py=8).cpu().numpy(), small)
    assert np.all(np.isfinite(small)) and small.sum() > 0
    sim.close()


@pytest.mark.parametrize("prec", [P.PRISM_PRECISION_FP32, P.PRISM_PRECISION_FP16, P.PRISM_PRECISION_FP16X2])
def test_smatrix_checkpoint_resume(prec, tmp_path):
    # an S-matrix saved to a file and loaded into a fresh plan scans like the plan that built it:
    # bitwise in FP32 and FP16 (a power-of-two scale and its 16-bit values survive the round trip);
    # in FP16X2 the stored value + remainder pairs may split differently where a remainder sits on a
    # rounding tie (same sum, other pair), which moves the products by about 2^-22 of a term; that
    # mode is held to the FP32 parity bar (relative L2 1e-4 per image), and so is its reload
    g = grid_dict(64, 64, 8.0, 8.0, 2, 2.0, 2)
    V = rand_v(2, 64, 64, 41)
    x0 = np.linspace(0.5, 7.5, 8)
    y0 = np.linspace(1.0, 2.0, 8)
    probe = P.make_probe(20.0, c1=5.0)
    grid = P.make_grid(64, 64, 2, 8.0, 8.0, 2.0, 300.0, 2, 2, 0.5, 20.0, precision=prec)
    a = PrismSimulation(grid)
    a.build(torch.from_numpy(V).cuda())
    ref = a.scan(probe, x0, y0, det_c(DET), px=8, py=1).cpu().numpy()
    np.save(tmp_path / "s.npy", a.smatrix().cpu().numpy())
    a.close()
    b = PrismSimulation(grid)
    b.load_smatrix(torch.from_numpy(np.load(tmp_path / "s.npy")).cuda())
    got = b.scan(probe, x0, y0, det_c(DET), px=8, py=1).cpu().numpy()
    b.close()
    if prec == P.PRISM_PRECISION_FP16X2:
        assert_images_close(got, ref, rel=1e-4)
    else:
        assert np.array_equal(ref, got)


def test_empty_scan_and_single_bin():
    g = grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2)
    V = rand_v(1, 64, 64, 11)
    sim = PrismSimulation(c_grid(g))
    sim.build(torch.from_numpy(V).cuda())
    out = sim.scan(P.make_probe(20.0), np.zeros(0), np.zeros(0), det_c(DET))
    assert out.shape == (0, 100)
    one = dict(start_mrad=5.0, step_mrad=200.0, nbins=1)
    x0, y0 = np.array([1.0, 2.0]), np.array([3.0, 4.0])
    got = sim.scan(P.make_probe(20.0), x0, y0, det_c(one)).cpu().numpy()
    S, m, nn = O.smatrix_build(V, g)
    ref = O.prism_scan(S, m, nn, g, dict(alpha_mrad=20.0), one, x0, y0)
    assert np.max(np.abs(got - ref) / ref) < 1e-5


def test_empty_sample_is_one_pixel_per_beam():
    g = grid_dict(64, 64, 8.0, 8.0, 2, 2.0, 2)
    V = np.zeros((2, 64, 64), np.float32)
    x0, y0 = np.array([1.7, 5.0]), np.array([3.2, -1.0])
    sim, out = run_prism(g, V, P.make_probe(20.0), x0, y0, DET)
    lam = O.wavelength(300.0)
    ref = np.zeros(DET["nbins"])
    m, nn = sim.beams()
    for b in range(len(m)):
        ref[int(1000 * lam * 2 * math.sqrt(m[b] ** 2 + nn[b] ** 2) / 8.0)] += 1.0 / len(m)
    assert np.max(np.abs(out - ref[None])) < 1e-6


def test_error_codes():
    def code(fn):
        with pytest.raises(P.PrismError) as e:
            fn()
        return e.value.status
    assert code(lambda: P.prism_plan_create(c_grid(grid_dict(100, 100, 8.0, 8.0, 1, 2.0, 1)))) == P.PRISM_ERR_UNSUPPORTED
    assert code(lambda: P.prism_plan_create(c_grid(grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 3)))) == P.PRISM_ERR_INVALID
    assert code(lambda: P.prism_plan_create(c_grid(grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2, aa=0.6)))) == P.PRISM_ERR_INVALID
    assert code(lambda: P.prism_plan_create(c_grid(grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2, alpha=90.0)))) == P.PRISM_ERR_INVALID
    assert code(lambda: P.prism_plan_create(c_grid(grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2)), 1000)) == P.PRISM_ERR_BUDGET
    plan = P.prism_plan_create(c_grid(grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2)))
    out = torch.empty((1, 10), device="cuda")
    sc = P.make_scan(1, 1, [0.0], [0.0])
    assert code(lambda: P.prism_scan_run(plan, P.make_probe(20.0), sc, P.make_detector(0, 1, 10), out)) == P.PRISM_ERR_INVALID
    V0 = torch.zeros((1, 64, 64), device="cuda")
    P.prism_build_smatrix(plan, V0)
    assert code(lambda: P.prism_scan_run(plan, P.make_probe(20.0, tilt_x=0.9), sc, P.make_detector(0, 1, 10), out)) == P.PRISM_ERR_INVALID
    assert code(lambda: P.prism_scan_run(plan, P.make_probe(20.0), sc, P.make_detector(0, 1, 0), out)) == P.PRISM_ERR_INVALID
    bad = P.make_scan(1, 1, [float("nan")], [0.0])
    assert code(lambda: P.prism_scan_run(plan, P.make_probe(20.0), bad, P.make_detector(0, 1, 10), out)) == P.PRISM_ERR_INVALID
    P.prism_sync(plan)
    P.prism_plan_destroy(plan)
