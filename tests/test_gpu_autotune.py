"""Autotuner: the launch shapes of the row and column passes of one FFT radix variant compute bitwise
the same transform, so an autotuned plan (or batch) that keeps the default radix reproduces the
default plan's S-matrix and detector stack exactly, whatever launch shapes it picks; the other radix
variant (the 32- and 64-point register DFTs split radix-4 first) computes the same transforms
rounded differently and agrees to FP32 rounding."""
import numpy as np
import pytest
import torch

from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300.runtime import Batch, PrismSimulation

pytestmark = pytest.mark.gpu

DET = P.make_detector(0.0, 1.0, 100)


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    yield
    torch.cuda.synchronize()


def rand_v(H, n, seed, amp=120.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return torch.from_numpy((amp * rng.random((H, n, n))).astype(np.float32)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# radix variants against the default: a few FP32 roundings per transform (the FP32 path's bar
# against the FP64 oracle is 1e-4; a 16-bit S-matrix can round a differing FP32 value to the
# neighbouring 16-bit one, 5e-4 relative, in a few elements)
RADIX_TOL = {P.PRISM_PRECISION_FP32: 1e-5, P.PRISM_PRECISION_FP16: 1e-4}


def run(grid, V, tune, x0, y0, fft_radix=False):
    sim = PrismSimulation(grid)
    res = sim.autotune(fft_radix) if tune else None
    sim.build(V)
    out = sim.scan(P.make_probe(20.0, c1=8.0), x0, y0, DET, px=len(x0), py=1).cpu().numpy()
    S = sim.smatrix().cpu().numpy()
    sim.close()
    return out, S, res


@pytest.mark.parametrize("fft_radix", [False, True])
@pytest.mark.parametrize("n,cell,f,prec", [(256, 16.0, 4, P.PRISM_PRECISION_FP32), (512, 32.0, 8, P.PRISM_PRECISION_FP16)])
def test_autotuned_plan_matches_the_default_plan(n, cell, f, prec, fft_radix):
    # plain autotuning keeps the default FFT radix: bit for bit; with the radix variants as
    # candidates a plan that keeps one agrees to rounding
    grid = P.make_grid(n, n, 3, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0, precision=prec)
    V = rand_v(3, n, 11)
    x0 = np.linspace(0.0, cell, 13, endpoint=False)
    y0 = np.linspace(1.0, 3.0, 13)
    a, Sa, _ = run(grid, V, False, x0, y0)
    b, Sb, res = run(grid, V, True, x0, y0, fft_radix)
    if res["row"]["fft_variant"] == 0 and res["col"]["fft_variant"] == 0:
        assert np.array_equal(a, b) and np.array_equal(Sa, Sb)
    else:
        assert fft_radix and n >= 512  # variants only when asked for, where 32-/64-point DFTs are used
        assert rel_l2(Sb, Sa) <= RADIX_TOL[prec] and rel_l2(b, a) <= RADIX_TOL[prec]
    for label in ("row", "col"):
        names = [k for k in res[label]["ms"]]
        assert fft_radix or not any("radix-4 first" in k for k in names)
        assert not fft_radix or n < 512 or any("radix-4 first" in k for k in names)
        ms = res[label]["ms"]
        assert len(ms) >= 2 and all(v > 0 for v in ms.values())
        assert res[label]["chosen"] in ms and res[label]["default"] in ms
        assert ms[res[label]["chosen"]] == min(ms.values())
    # a second plan of the same shape reuses the cached choice
    sim = PrismSimulation(grid)
    assert sim.autotune(fft_radix) == res
    sim.close()


@pytest.mark.parametrize("n,cell,f", [(1024, 50.0, 8), (512, 32.0, 8)])
@pytest.mark.parametrize("kind", [P.PRISM_TUNE_ROW, P.PRISM_TUNE_COL])
def test_every_shape_of_a_radix_is_bitwise_identical(n, cell, f, kind):
    # each compiled shape of a pass pinned in turn -- threads or columns per CTA, unstaged,
    # cp.async-staged and TMA-staged rows or tiles, register caps -- builds the same S-matrix and
    # detector stack as every other shape of its FFT radix variant, bit for bit; the radix-4-first
    # variant agrees with the default to FP32 rounding
    grid = P.make_grid(n, n, 2, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0)
    V = rand_v(2, n, 12)
    x0 = np.linspace(0.0, cell, 9, endpoint=False)
    y0 = np.linspace(1.0, 3.0, 9)
    probe = P.make_probe(20.0)
    ref = PrismSimulation(grid)
    ref.build(V)
    S0 = ref.smatrix().cpu().numpy()
    o0 = ref.scan(probe, x0, y0, DET).cpu().numpy()
    ref.close()
    ran, first = [], {}
    for v in range(P.PRISM_TUNE_MAX_SHAPES):
        if P.prism_tune_shape_name(kind, v) == "?":
            continue
        sim = PrismSimulation(grid)
        try:
            sim.set_shape(kind, v)
        except P.PrismError as e:
            assert e.status == P.PRISM_ERR_UNSUPPORTED
            sim.close()
            continue
        sim.build(V)
        out = sim.scan(probe, x0, y0, DET).cpu().numpy()
        sim.sync()
        S = sim.smatrix().cpu().numpy()
        name, rv = P.prism_tune_shape_name(kind, v), P.prism_tune_shape_fft_variant(kind, v)
        if rv == 0:
            assert np.array_equal(S0, S) and np.array_equal(o0, out), name
        else:
            assert rel_l2(S, S0) <= RADIX_TOL[P.PRISM_PRECISION_FP32] and rel_l2(out, o0) <= RADIX_TOL[P.PRISM_PRECISION_FP32], name
            assert not np.array_equal(S0, S), name  # the variant does run: other roundings
            if rv in first:
                assert np.array_equal(first[rv][0], S) and np.array_equal(first[rv][1], out), name
            first.setdefault(rv, (S, out))
        ran.append(name)
        sim.close()
    assert 3 in first and (n < 1024 or {1, 2, 3} <= set(first))  # the radix variants ran
    if kind == P.PRISM_TUNE_COL:
        assert "W8, TMA" in ran and "W8, staged" in ran and "W8, staged, radix-4 first: both" in ran
    else:
        assert "128 thr" in ran and ("128 thr, TMA" in ran) == (n >= 1024) and "128 thr, radix-4 first: both" in ran


def test_small_grid_has_only_the_default_shape():
    grid = P.make_grid(64, 64, 2, 8.0, 8.0, 2.0, 300.0, 2, 2, 0.5, 20.0)
    sim = PrismSimulation(grid)
    res = sim.autotune()
    assert res["row"]["chosen"] == "default" and res["row"]["ms"] == {}
    sim.close()


@pytest.mark.parametrize("fft_radix", [False, True])
def test_autotuned_batch_equals_untuned(fft_radix):
    cells = []
    for i, (n, cell, f, H) in enumerate([(256, 16.0, 4, 3), (512, 32.0, 8, 2), (128, 12.8, 2, 2)]):
        x0 = np.linspace(0.0, 4.0, 8)
        cells.append(dict(grid=P.make_grid(n, n, H, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0), V=rand_v(H, n, 20 + i),
                          probe=P.make_probe(20.0), x0=x0, y0=np.full(8, 1.5), det=DET))
    outs = []
    for tune in (False, True):
        b = Batch(cells, n_branches=2, autotune=tune, fft_radix=fft_radix and tune)
        b.run()
        b.sync()
        outs.append([o.cpu().numpy() for o in b.outs])
        b.close()
    for c, u, t in zip(cells, *outs):
        # launch shapes alone, or below N = 512 (one radix variant): bit for bit; the 512^2 cell tuned
        # with the radix variants may take another
        if not fft_radix or c["grid"].nx < 512:
            assert np.array_equal(u, t)
        else:
            assert np.array_equal(u, t) or rel_l2(t, u) <= RADIX_TOL[P.PRISM_PRECISION_FP32]


@pytest.mark.parametrize("n,cell,f,px,py,step", [(256, 16.0, 4, 13, 9, 0.3), (256, 32.0, 8, 10, 21, 0.45),
                                                (512, 32.0, 4, 23, 17, 0.25)])
def test_every_scan_contraction_shape_is_bitwise_identical(n, cell, f, px, py, step):
    # FP32 GEMM scan with 32-, 16- and 64-pixel windows: raster blocks 4 x 8, 8 x 4, 2 x 16 and beam
    # rings 2 x 32, 3 x 16, 2 x 33 sum every window pixel over the beams in the same order; ragged rasters
    # (px, py not multiples of the block sides) cover partial blocks and the split last round
    grid = P.make_grid(n, n, 3, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0)
    V = rand_v(3, n, 21)
    X, Y = np.meshgrid(0.7 + step * np.arange(px), cell - 1.0 + step * np.arange(py))  # wraps in y
    x0, y0 = X.ravel(), Y.ravel()
    probe = P.make_probe(20.0, c1=12.0)
    sim = PrismSimulation(grid)
    sim.build(V)
    nw = sim.info.nw_x
    assert nw == n // 2 // f
    ref = sim.scan(probe, x0, y0, DET, px=px, py=py).cpu().numpy()
    n_shapes = P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN).n_shapes
    assert n_shapes == 6
    for v in range(n_shapes):
        sim.set_shape(P.PRISM_TUNE_SCAN, v)
        got = sim.scan(probe, x0, y0, DET, px=px, py=py).cpu().numpy()
        assert np.array_equal(got, ref), P.prism_tune_shape_name(P.PRISM_TUNE_SCAN, v)
    sim.set_shape(P.PRISM_TUNE_SCAN, -1)
    out = sim.autotune_scan(probe, x0, y0, DET, px=px, py=py).cpu().numpy()
    assert np.array_equal(out, ref)
    res = sim.tune_result()["scan"]
    assert len(res["ms"]) == n_shapes and all(t > 0 for t in res["ms"].values())
    assert res["ms"][res["chosen"]] == min(res["ms"].values())
    assert np.array_equal(sim.scan(probe, x0, y0, DET, px=px, py=py).cpu().numpy(), ref)
    sim.close()


def test_every_scan_contraction_shape_sizes_its_own_scratch():
    # a plan whose scans first ran small, pinned to each contraction shape in turn, then scanning a
    # larger raster: the window scratch grows for that shape's blocks (the result equals the
    # default shape's, bit for bit)
    n, cell, f = 256, 16.0, 4
    grid = P.make_grid(n, n, 2, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0)
    V = rand_v(2, n, 22)
    X, Y = np.meshgrid(0.3 + 0.35 * np.arange(21), 0.4 + 0.35 * np.arange(19))
    x0, y0 = X.ravel(), Y.ravel()
    probe = P.make_probe(20.0)
    ref = None
    n_shapes = None
    for v in range(16):
        sim = PrismSimulation(grid)
        if n_shapes is None:
            n_shapes = P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN).n_shapes
        if v >= n_shapes:
            sim.close()
            break
        sim.build(V)
        sim.scan(probe, x0[:2], y0[:2], DET, px=2, py=1)  # a small first scan: a small scratch
        sim.set_shape(P.PRISM_TUNE_SCAN, v)
        out = sim.scan(probe, x0, y0, DET, px=21, py=19).cpu().numpy()
        sim.close()
        if ref is None:
            ref = out
        assert np.array_equal(out, ref), P.prism_tune_shape_name(P.PRISM_TUNE_SCAN, v)
    assert n_shapes == 6


@pytest.mark.parametrize("prec", [P.PRISM_PRECISION_FP16, P.PRISM_PRECISION_BF16])
def test_every_tensor_core_ring_shape_is_bitwise_identical(prec):
    # 16-bit plans: the tensor-core scan's A-operand ring (3 x 96, 2 x 128, 4 x 64 K values) issues the
    # K = 16 MMAs of a pixel tile in the same order in every shape, so the detector stacks are equal
    # bit for bit; the autotuner keeps the fastest and leaves the same stack
    n, cell, f = 512, 32.0, 8
    grid = P.make_grid(n, n, 2, cell, cell, 2.0, 300.0, f, 2, 0.5, 20.0, precision=prec)
    V = rand_v(2, n, 23)
    X, Y = np.meshgrid(0.5 + 0.3 * np.arange(17), cell - 2.0 + 0.3 * np.arange(13))  # wraps in y
    x0, y0 = X.ravel(), Y.ravel()
    probe = P.make_probe(20.0, c1=10.0)
    sim = PrismSimulation(grid)
    sim.build(V)
    ref = sim.scan(probe, x0, y0, DET, px=17, py=13).cpu().numpy()
    res = P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN_TC)
    assert res.n_shapes == 3 and res.chosen == 0
    assert P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN).n_shapes == 0
    for v in range(res.n_shapes):
        sim.set_shape(P.PRISM_TUNE_SCAN_TC, v)
        got = sim.scan(probe, x0, y0, DET, px=17, py=13).cpu().numpy()
        assert np.array_equal(got, ref), P.prism_tune_shape_name(P.PRISM_TUNE_SCAN_TC, v)
    with pytest.raises(P.PrismError) as e:
        sim.set_shape(P.PRISM_TUNE_SCAN_TC, 3)
    assert e.value.status == P.PRISM_ERR_UNSUPPORTED
    sim.set_shape(P.PRISM_TUNE_SCAN_TC, -1)
    out = sim.autotune_scan(probe, x0, y0, DET, px=17, py=13).cpu().numpy()
    assert np.array_equal(out, ref)
    tr = sim.tune_result()["scan_tc"]
    assert len(tr["ms"]) == 3 and tr["ms"][tr["chosen"]] == min(tr["ms"].values())
    sim.close()
    # an FP32 plan has no ring shapes; split mode has one
    sim = PrismSimulation(P.make_grid(256, 256, 1, 16.0, 16.0, 2.0, 300.0, 4, 2, 0.5, 20.0))
    assert P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN_TC).n_shapes == 0
    with pytest.raises(P.PrismError):
        sim.set_shape(P.PRISM_TUNE_SCAN_TC, 0)
    sim.close()
    sim = PrismSimulation(P.make_grid(256, 256, 1, 16.0, 16.0, 2.0, 300.0, 4, 2, 0.5, 20.0, precision=P.PRISM_PRECISION_FP16X2))
    assert P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN_TC).n_shapes == 1
    sim.close()


def test_scan_shape_limits():
    # 16-bit plans have one (tensor-core) scan shape; shapes past the list are refused
    grid = P.make_grid(256, 256, 1, 16.0, 16.0, 2.0, 300.0, 4, 2, 0.5, 20.0, precision=P.PRISM_PRECISION_FP16)
    sim = PrismSimulation(grid)
    with pytest.raises(P.PrismError) as e:
        sim.set_shape(P.PRISM_TUNE_SCAN, 1)
    assert e.value.status == P.PRISM_ERR_UNSUPPORTED
    assert P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN).n_shapes == 0
    sim.close()
    sim = PrismSimulation(P.make_grid(256, 256, 1, 16.0, 16.0, 2.0, 300.0, 4, 2, 0.5, 20.0))
    n = P.prism_plan_tune_result(sim.plan, P.PRISM_TUNE_SCAN).n_shapes
    sim.set_shape(P.PRISM_TUNE_SCAN, n - 1)
    with pytest.raises(P.PrismError):
        sim.set_shape(P.PRISM_TUNE_SCAN, n)
    sim.close()


def test_concurrent_scans_of_different_beam_counts():
    # plans of different beam counts (so different shared memory for the same scan kernel) scanning
    # from four host threads at once: every launch keeps its resources and each result equals the
    # plan's own result scanned alone
    import threading
    cases = [(256, 16.0, 4, 20.0), (256, 16.0, 4, 12.0), (256, 16.0, 4, 28.0), (256, 16.0, 4, 16.0)]
    sims, inputs, refs = [], [], []
    for i, (n, cell, f, amax) in enumerate(cases):
        g = P.make_grid(n, n, 2, cell, cell, 2.0, 300.0, f, 2, 0.5, amax)
        sim = PrismSimulation(g)
        sim.build(rand_v(2, n, 30 + i))
        X, Y = np.meshgrid(0.2 + 0.4 * np.arange(15), 0.3 + 0.4 * np.arange(11))
        x0, y0 = X.ravel(), Y.ravel()
        probe = P.make_probe(min(amax, 20.0))
        refs.append(sim.scan(probe, x0, y0, DET, px=15, py=11).cpu().numpy())
        sims.append(sim)
        inputs.append((probe, x0, y0))
    assert len({s.info.n_beams for s in sims}) == len(sims)
    outs, errors = [None] * len(sims), []

    def worker(i):
        try:
            probe, x0, y0 = inputs[i]
            for _ in range(5):
                o = sims[i].scan(probe, x0, y0, DET, px=15, py=11)
                sims[i].sync()
            outs[i] = o.cpu().numpy()
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(sims))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for o, r in zip(outs, refs):
        assert np.array_equal(o, r)
    for s in sims:
        s.close()
