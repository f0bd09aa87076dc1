"""Batches of uneven cells run as one captured CUDA graph (prism_batch_*).

Every cell of a batch must give exactly (bitwise) what its own plan gives when run alone: the
graph replays the same kernels on the same inputs.  One small cell is also checked against the FP64
oracle directly."""
import numpy as np
import pytest
import torch

from oracle import prism_oracle as O
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
    return (amp * rng.random((H, n, n))).astype(np.float32)


def raster(px, py, step, x_start=0.0, y_start=0.0):
    X, Y = np.meshgrid(x_start + step * np.arange(px), y_start + step * np.arange(py))
    return X.ravel(), Y.ravel()


# uneven cells: sizes, slice counts (one with unequal slices), f, precision, probe shapes, an empty scan
SPECS = [
    dict(n=64, cell=8.0, H=3, f=2, prec=P.PRISM_PRECISION_FP32, px=7, py=5, c1=10.0),
    dict(n=128, cell=12.8, H=5, f=4, prec=P.PRISM_PRECISION_FP32, px=11, py=3, c1=0.0),
    dict(n=128, cell=12.8, H=2, f=2, prec=P.PRISM_PRECISION_FP16, px=9, py=9, c1=-20.0),
    dict(n=256, cell=16.0, H=4, f=4, prec=P.PRISM_PRECISION_BF16, px=8, py=4, c1=5.0),
    dict(n=64, cell=6.4, H=2, f=1, prec=P.PRISM_PRECISION_FP32, px=0, py=0, c1=0.0),
    dict(n=128, cell=16.0, H=3, f=4, prec=P.PRISM_PRECISION_FP32, px=4, py=4, c1=0.0, slice_dz=[1.0, 2.5, 0.5]),
]


def grid_of(sp):
    return P.make_grid(sp["n"], sp["n"], sp["H"], sp["cell"], sp["cell"], 2.0, 300.0, sp["f"], 2, 0.5, 20.0,
                       slice_dz=sp.get("slice_dz"), precision=sp["prec"])


def cells_of(specs, seed0):
    cells = []
    for i, sp in enumerate(specs):
        V = torch.from_numpy(rand_v(sp["H"], sp["n"], seed0 + i)).cuda()
        x0, y0 = raster(sp["px"], sp["py"], 0.3, 0.2 * i, 0.1)
        cells.append(dict(grid=grid_of(sp), V=V, probe=P.make_probe(20.0, c1=sp["c1"]), x0=x0, y0=y0,
                          px=sp["px"], py=sp["py"], det=DET))
    return cells


def alone(c):
    sim = PrismSimulation(c["grid"])
    sim.build(c["V"])
    out = sim.scan(c["probe"], c["x0"], c["y0"], c["det"], px=c["px"] or None, py=c["py"] or None)
    sim.sync()
    o = out.cpu().numpy()
    sim.close()
    return o


def test_batch_equals_cells_alone_and_replays():
    cells = cells_of(SPECS, 40)
    b = Batch(cells, n_branches=3)
    assert b.info.n_cells == len(SPECS) and b.info.n_branches == 3
    assert b.info.kernel_launches > 0 and b.info.graph_nodes >= b.info.kernel_launches
    b.run()
    b.sync()
    first = [o.cpu().numpy() for o in b.outs]
    for c, got in zip(cells, first):
        assert np.array_equal(got, alone(c))
    # a second run of the graph is bitwise identical
    for o in b.outs:
        o.fill_(-1.0)
    b.run()
    b.sync()
    for a, o in zip(first, b.outs):
        assert np.array_equal(a, o.cpu().numpy())
    # new potentials in the same buffers: the next run follows them
    for i, c in enumerate(cells):
        c["V"].copy_(torch.from_numpy(rand_v(c["grid"].n_slices, c["grid"].nx, 90 + i)))
    b.run()
    b.sync()
    for c, o in zip(cells, b.outs):
        assert np.array_equal(o.cpu().numpy(), alone(c))
    b.close()


def test_batch_cell_matches_oracle():
    sp = SPECS[0]
    cells = cells_of([sp, SPECS[1]], 70)
    b = Batch(cells, n_branches=2)
    b.run()
    b.sync()
    c = cells[0]
    g = dict(nx=sp["n"], ny=sp["n"], cell_x=sp["cell"], cell_y=sp["cell"], n_slices=sp["H"], dz=2.0, kv=300.0,
             f=sp["f"], downsample=2, aa_frac=0.5, alpha_mrad=20.0)
    S, m, n = O.smatrix_build(c["V"].cpu().numpy(), g)
    ref = O.prism_scan(S, m, n, g, dict(alpha_mrad=20.0, c1=sp["c1"]), dict(start_mrad=0.0, step_mrad=1.0, nbins=100),
                       c["x0"], c["y0"])
    got = b.outs[0].cpu().numpy().astype(np.float64)
    bright = ref.mean(0) >= 1e-7
    assert O.rel_l2_per_image(got[:, bright], ref[:, bright]).max() <= 1e-4
    assert np.max(np.abs(got[:, ~bright] - ref[:, ~bright])) <= 1e-9
    b.close()


def test_batch_errors():
    def code(fn):
        with pytest.raises(P.PrismError) as e:
            fn()
        return e.value.status, str(e.value)
    assert code(lambda: P.prism_batch_create([], 0, 0))[0] == P.PRISM_ERR_INVALID
    cells = cells_of(SPECS[:2], 80)
    assert code(lambda: Batch(cells, n_branches=17))[0] == P.PRISM_ERR_INVALID
    assert code(lambda: Batch(cells, hbm_budget_bytes=1 << 20))[0] == P.PRISM_ERR_BUDGET
    bad = cells_of([dict(SPECS[0], prec=P.PRISM_PRECISION_FP16, f=4)], 85)  # 8-pixel window: no 16-bit scan
    st, msg = code(lambda: Batch(cells + bad))
    assert st == P.PRISM_ERR_UNSUPPORTED and "cell 2" in msg


def test_uneven_workload_cells_in_one_graph_match_oracle():
    # five cells of the seeded 64-cell uneven workload spanning N = 256, 512, 1024 and f = 4, 8
    # (seeds 126, 112, 150, 132, 136: 10-17 slices, 49 to about 830 beams), run together in one graph
    # launch with their 16 x 16 raster scans; four probes of each against the oracle (one
    # multislice of each probe's d/f-periodic wave, Eq. PRISMfinal linearity)
    import oracle_pool
    from paper_1702_01904_gb300 import specimens
    seeds = (126, 112, 150, 132, 136)
    cells, work = [], []
    for s in seeds:
        w, V = specimens.batch_cell_potential(s)
        x0, y0 = w.scan_positions()
        cells.append(dict(grid=P.grid_from_workload(w), V=torch.from_numpy(V).cuda(), probe=P.make_probe(w.alpha_mrad),
                          x0=x0, y0=y0, px=w.scan_px, py=w.scan_py, det=DET))
        work.append((w, V, x0, y0))
    assert {w.nx for w, *_ in work} == {256, 512, 1024} and {w.f for w, *_ in work} == {4, 8}
    b = Batch(cells, n_branches=4)
    b.run()
    b.sync()
    det = dict(start_mrad=0.0, step_mrad=1.0, nbins=100)
    for (w, V, x0, y0), out in zip(work, b.outs):
        g = dict(nx=w.nx, ny=w.ny, cell_x=w.cell_x, cell_y=w.cell_y, n_slices=w.n_slices, dz=w.dz, kv=w.kv, f=w.f,
                 downsample=w.downsample, aa_frac=w.aa_frac, alpha_mrad=w.alpha_mrad)
        pick = [0, 17, 130, 255]
        ref = np.array(oracle_pool.evaluate("prism", V, g, [(dict(alpha_mrad=w.alpha_mrad), det, float(x0[k]), float(y0[k]))
                                                             for k in pick]))
        got = out.cpu().numpy().astype(np.float64)[pick]
        bright = ref.mean(0) >= 1e-7
        assert bright.sum() >= 10
        err = O.rel_l2_per_image(got[:, bright], ref[:, bright]).max()
        assert err <= 1e-4, (w.name, err)
        assert np.max(np.abs(got[:, ~bright] - ref[:, ~bright])) <= 1e-9
    b.close()
