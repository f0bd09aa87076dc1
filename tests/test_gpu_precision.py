"""Reduced-precision PRISM on the GPU: S-matrix stored in FP16 or BF16 with one power-of-two scale per
beam, beam sum of Eq. PRISMfinal on the tcgen05 tensor cores with FP32 accumulation; and the split
mode FP16X2 (value + remainder, three products per step), which is held to the FP32 bars.

Bars.  Stored values: each dequantised S element is within half a unit in the last place of its
16-bit value of the FP32 S (unit roundoff u = 2^-11 FP16, 2^-8 BF16, relative to the element, plus
the subnormal spacing of the scaled value).

Detector stacks, relative L2 per detector image against the FP64 oracle.  Rounding the stored S
adds independent errors of relative size ~u to every window pixel, i.e. a white noise floor over
the window's diffraction pattern whose power is ~u^2/3 of the total.  A bin of intensity I then
carries an error ~2 sqrt(I * noise in the bin): its relative error grows like 1/sqrt(I).  Measured
on the particle sweep and random potentials: FP16 stays below 5e-3 for images of mean >= 1e-5 of
the incident intensity and below 5e-4 above 1e-3; BF16 (three mantissa bits fewer, 8x the noise
amplitude) below 4e-3 above 1e-3 and 1.3e-2 between 1e-4 and 1e-3.  The gates, with about 2x
margin: FP16 <= 2e-3 for images of mean >= 1e-3 and <= 1e-2 for mean >= 1e-5; BF16 <= 1e-2 for
mean >= 1e-3; dimmer images absolute <= 5e-7 (FP16) and 2e-5 (BF16).  Every per-image error is
written to $PRISM_REPORT_DIR when it is set.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import prism_oracle as O
from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300 import specimens
from paper_1702_01904_gb300.runtime import PrismSimulation

pytestmark = pytest.mark.gpu

DET = dict(start_mrad=0.0, step_mrad=1.0, nbins=100)
HALF = {"fp16": P.PRISM_PRECISION_FP16, "bf16": P.PRISM_PRECISION_BF16, "fp16x2": P.PRISM_PRECISION_FP16X2}
# relative representation bound of a stored value (fp16x2: value + remainder, about 22 bits)
U = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16x2": 2.0 ** -21}
# (image mean floor, relative L2 bar) tiers and the absolute bar for images below every floor
TIERS = {"fp16": ([(1e-3, 2e-3), (1e-5, 1e-2)], 5e-7), "bf16": ([(1e-3, 1e-2)], 2e-5),
         "fp32": ([(1e-7, 1e-4)], 1e-9), "fp16x2": ([(1e-7, 1e-4)], 1e-9)}


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    yield
    torch.cuda.synchronize()


def grid_dict(nx, ny, cx, cy, H, dz, f, ds=2, alpha=20.0):
    return dict(nx=nx, ny=ny, cell_x=cx, cell_y=cy, n_slices=H, dz=dz, kv=300.0, f=f, downsample=ds,
                aa_frac=0.5, alpha_mrad=alpha)


def c_grid(g, precision):
    return P.make_grid(g["nx"], g["ny"], g["n_slices"], g["cell_x"], g["cell_y"], g["dz"], g["kv"], g["f"],
                       g["downsample"], g["aa_frac"], g["alpha_mrad"], precision=precision)


def det_c(d):
    return P.make_detector(d["start_mrad"], d["step_mrad"], d["nbins"])


def rand_v(H, ny, nx, seed, amp=120.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (amp * rng.random((H, ny, nx))).astype(np.float32)


def check(gpu, ref, prec):
    """Apply the tiers of `prec`; returns the relative L2 of every image above the lowest floor."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape
    tiers, abs_dim = TIERS[prec]
    mean = ref.mean(0)
    for floor, bar in tiers:
        sel = mean >= floor
        if sel.any():
            rel = O.rel_l2_per_image(gpu[:, sel], ref[:, sel])
            assert rel.max() <= bar, f"{prec}: rel L2 {rel.max():.3e} at bin {np.flatnonzero(sel)[rel.argmax()]} (floor {floor:g})"
    low = tiers[-1][0]
    dim = mean < low
    if dim.any():
        err = np.max(np.abs(gpu[:, dim] - ref[:, dim]))
        assert err <= abs_dim, f"{prec}: dim-image abs error {err:.3e}"
    sel = mean >= low
    return O.rel_l2_per_image(gpu[:, sel], ref[:, sel]) if sel.any() else np.zeros(0)


def run(g, V, precision, probe, x0, y0, px=None, py=None, det=DET):
    sim = PrismSimulation(c_grid(g, precision))
    sim.build(torch.from_numpy(V).cuda())
    out = sim.scan(probe, x0, y0, det_c(det), px=px, py=py)
    sim.sync()
    return sim, out.cpu().numpy()


def report(name, data):
    d = os.environ.get("PRISM_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, f"precision_{name}.json"), "w") as fh:
            json.dump(data, fh, indent=1)


# ------------------------------------------------------------------ stored values
@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp16x2"])
def test_dequantised_smatrix_within_half_ulp(prec):
    g = grid_dict(128, 128, 12.8, 12.8, 3, 2.0, 2)
    V = rand_v(3, 128, 128, 21)
    ref = PrismSimulation(c_grid(g, P.PRISM_PRECISION_FP32))
    ref.build(torch.from_numpy(V).cuda())
    S32 = ref.smatrix().cpu().numpy()
    sim = PrismSimulation(c_grid(g, HALF[prec]))
    sim.build(torch.from_numpy(V).cuda())
    Sq = sim.smatrix().cpu().numpy()
    assert Sq.shape == S32.shape
    for b in range(len(S32)):
        a32 = np.stack([S32[b].real, S32[b].imag]).astype(np.float64)
        aq = np.stack([Sq[b].real, Sq[b].imag]).astype(np.float64)
        scale = 2.0 ** (np.floor(np.log2(np.abs(a32).max())) + 1)
        tiny = scale * (2.0 ** -133 if prec == "bf16" else 2.0 ** -24)
        assert np.all(np.abs(aq - a32) <= U[prec] * np.abs(a32) + tiny), b
    info = sim.info
    kp = 2 * ((info.n_beams + 7) // 8 * 8)
    parts = 2 if prec == "fp16x2" else 1
    assert P.prism_plan_smatrix_bytes(sim.plan) == info.nx_s * info.ny_s * kp * 2 * parts + kp // 2 * 4
    with pytest.raises(P.PrismError):
        P.prism_plan_smatrix(sim.plan)


# ------------------------------------------------------------------ small grids vs the oracle
CASES = [
    dict(n=64, cell=8.0, H=3, f=2, nw=16),
    dict(n=128, cell=12.8, H=2, f=2, nw=32),
    dict(n=256, cell=12.8, H=2, f=2, nw=64),
    dict(n=128, cell=12.8, H=2, f=1, nw=64),   # 529 beams: K = 1072
]


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp16x2"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nw{c['nw']}-f{c['f']}")
def test_tc_scan_matches_oracle(case, prec):
    n = case["n"]
    g = grid_dict(n, n, case["cell"], case["cell"], case["H"], 2.0, case["f"])
    V = rand_v(case["H"], n, n, 22)
    probe = dict(alpha_mrad=20.0, c1=15.0, c3=2.0e4)
    if prec == "fp16x2" and case["f"] == 1:
        # the value and remainder coefficient matrices of 529 beams (2 x 137 KB) exceed shared memory
        with pytest.raises(P.PrismError) as e:
            PrismSimulation(c_grid(g, HALF[prec]))
        assert e.value.status == P.PRISM_ERR_UNSUPPORTED
        return
    S, m, nn = O.smatrix_build(V, g)
    # (1) scattered, wrapped positions: every group is run probe by probe
    rng = np.random.Generator(np.random.PCG64(23))
    x0 = rng.uniform(-case["cell"], 2 * case["cell"], 21)
    y0 = rng.uniform(-case["cell"], 2 * case["cell"], 21)
    sim, out = run(g, V, HALF[prec], P.make_probe(**probe), x0, y0)
    assert sim.info.nw_x == case["nw"]
    check(out, O.prism_scan(S, m, nn, g, probe, DET, x0, y0), prec)
    # (2) a ragged raster (11 x 5, step 0.3 A, across the periodic edge): groups share union tiles
    xs = (np.arange(11) * 0.3 - 1.0) % case["cell"]
    ys = np.arange(5) * 0.3 + 0.5
    X, Y = np.meshgrid(xs, ys)
    x0, y0 = X.ravel(), Y.ravel()
    out = sim.scan(P.make_probe(**probe), x0, y0, det_c(DET), px=11, py=5).cpu().numpy()
    check(out, O.prism_scan(S, m, nn, g, probe, DET, x0, y0), prec)
    sim.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp16x2"])
def test_tc_small_workload(prec):
    w = specimens.workload_small()
    V = w.potential()
    g = grid_dict(w.nx, w.ny, w.cell_x, w.cell_y, w.n_slices, w.dz, w.f, alpha=w.alpha_mrad)
    x0, y0 = w.scan_positions()
    sim, out = run(g, V, HALF[prec], P.make_probe(w.alpha_mrad), x0, y0, w.scan_px, w.scan_py)
    S, m, nn = O.smatrix_build(V, g)
    check(out, O.prism_scan(S, m, nn, g, dict(alpha_mrad=w.alpha_mrad), DET, x0, y0), prec)
    sim.close()


# ------------------------------------------------------------------ precision sweep: Au particle on Cu, f = 4, 8, 16
@pytest.fixture(scope="module")
def nanoparticle():
    cache = {}

    def get(f):
        if f not in cache:
            w = specimens.workload_nanoparticle(f=f)
            V = w.potential()
            g = grid_dict(w.nx, w.ny, w.cell_x, w.cell_y, w.n_slices, w.dz, w.f, alpha=w.alpha_mrad)
            x0, y0 = w.scan_positions()
            S, m, nn = O.smatrix_build(V, g)
            ref = O.prism_scan(S, m, nn, g, dict(alpha_mrad=w.alpha_mrad), DET, x0, y0)
            cache[f] = (w, V, g, x0, y0, ref)
        return cache[f]
    return get


@pytest.mark.parametrize("f,beams,nw", [(16, 13, 16), (8, 49, 32), (4, 213, 64)])
def test_precision_sweep_nanoparticle(nanoparticle, f, beams, nw):
    w, V, g, x0, y0, ref = nanoparticle(f)
    probe = P.make_probe(w.alpha_mrad)
    rows = {}
    for prec, code in [("fp32", P.PRISM_PRECISION_FP32), ("fp16", HALF["fp16"]), ("bf16", HALF["bf16"]),
                       ("fp16x2", HALF["fp16x2"])]:
        sim, out = run(g, V, code, probe, x0, y0, w.scan_px, w.scan_py)
        assert sim.info.n_beams == beams and sim.info.nw_x == nw
        check(out, ref, prec)
        lit = np.linalg.norm(ref, axis=0) > 0
        rel = np.full(ref.shape[1], np.nan)
        rel[lit] = O.rel_l2_per_image(np.asarray(out, np.float64)[:, lit], ref[:, lit])
        rows[prec] = [None if np.isnan(e) else float(e) for e in rel]
        sim.close()
    rows["oracle_image_mean"] = [float(v) for v in ref.mean(0)]
    report(f"nanoparticle_f{f}", dict(workload=w.name, beams=beams, nw=nw, probes=len(x0), errors=rows))


# ------------------------------------------------------------------ full-size amorphous carbon: 16-bit vs FP32 path and oracle samples
def test_tc_carbon_workload_full_size():
    w = specimens.workload_amorphous_carbon()
    V = w.potential()
    g = grid_dict(w.nx, w.ny, w.cell_x, w.cell_y, w.n_slices, w.dz, w.f, alpha=w.alpha_mrad)
    x0, y0 = w.scan_positions()
    probe = P.make_probe(w.alpha_mrad)
    s32, o32 = run(g, V, P.PRISM_PRECISION_FP32, probe, x0, y0, w.scan_px, w.scan_py)
    s32.close()
    sx, ox2 = run(g, V, HALF["fp16x2"], probe, x0, y0, w.scan_px, w.scan_py)
    relx = check(ox2, o32, "fp16x2")
    sx.close()
    sim, o16 = run(g, V, HALF["fp16"], probe, x0, y0, w.scan_px, w.scan_py)
    rel = check(o16, o32, "fp16")
    # sampled probes against the oracle (one direct multislice of each periodic probe)
    sel = [0, 199, 20101, 39999]
    ref = np.array([O.prism_probe_direct(V, g, dict(alpha_mrad=w.alpha_mrad), DET, x0[i], y0[i]) for i in sel])
    b = ref.mean(0) >= 1e-5
    e = np.linalg.norm(o16[sel][:, b] - ref[:, b]) / np.linalg.norm(ref[:, b])
    assert e <= 2e-3
    # bitwise repeatable
    again = sim.scan(probe, x0, y0, det_c(DET), px=w.scan_px, py=w.scan_py).cpu().numpy()
    assert np.array_equal(again, o16)
    report("carbon_fp16_vs_fp32", dict(workload=w.name, max=float(rel.max()), median=float(np.median(rel)),
                                       sampled_vs_oracle=float(e), fp16x2_max=float(relx.max())))
    sim.close()


# ------------------------------------------------------------------ scan variants in 16-bit mode
def test_tc_cbed_and_accumulate_match_fp32():
    g = grid_dict(128, 128, 12.8, 12.8, 2, 2.0, 2)
    V = rand_v(2, 128, 128, 24)
    xs, ys = np.meshgrid(np.linspace(0, 12.8, 9, endpoint=False), np.linspace(0, 3, 3))
    x0, y0 = xs.ravel(), ys.ravel()
    probe = P.make_probe(20.0, c1=5.0)
    a = PrismSimulation(c_grid(g, P.PRISM_PRECISION_FP32))
    b = PrismSimulation(c_grid(g, HALF["fp16"]))
    for s in (a, b):
        s.build(torch.from_numpy(V).cuda())
    ca = a.scan_cbed(probe, x0, y0, px=9, py=3).cpu().numpy()
    cb = b.scan_cbed(probe, x0, y0, px=9, py=3).cpu().numpy()
    assert np.linalg.norm(cb - ca) / np.linalg.norm(ca) < 3e-3
    acc_a = torch.zeros((27, DET["nbins"]), device="cuda")
    acc_b = torch.zeros((27, DET["nbins"]), device="cuda")
    for wgt in (0.25, 0.75):
        a.scan_accumulate(probe, x0, y0, det_c(DET), wgt, acc_a, px=9, py=3)
        b.scan_accumulate(probe, x0, y0, det_c(DET), wgt, acc_b, px=9, py=3)
    a.sync()
    b.sync()
    check(acc_b.cpu().numpy(), acc_a.cpu().numpy(), "fp16")
    one = b.scan(probe, x0, y0, det_c(DET), px=9, py=3).cpu().numpy()
    assert np.allclose(acc_b.cpu().numpy(), one, rtol=1e-6, atol=1e-12)
    a.close()
    b.close()


def test_tc_edge_cases():
    g = grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 2)
    V = rand_v(1, 64, 64, 25)
    sim = PrismSimulation(c_grid(g, HALF["fp16"]))
    sim.build(torch.from_numpy(V).cuda())
    out = sim.scan(P.make_probe(20.0), np.zeros(0), np.zeros(0), det_c(DET))
    assert out.shape == (0, 100)
    S, m, nn = O.smatrix_build(V, g)
    x0, y0 = np.array([3.3]), np.array([-2.0])
    got = sim.scan(P.make_probe(20.0), x0, y0, det_c(DET)).cpu().numpy()
    check(got, O.prism_scan(S, m, nn, g, dict(alpha_mrad=20.0), DET, x0, y0), "fp16")
    sim.close()
    # 16-bit mode needs a 16, 32 or 64 pixel window
    with pytest.raises(P.PrismError) as e:
        PrismSimulation(c_grid(grid_dict(64, 64, 8.0, 8.0, 1, 2.0, 4), HALF["fp16"]))
    assert e.value.status == P.PRISM_ERR_UNSUPPORTED
