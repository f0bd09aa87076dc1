"""GPU tests of the continuous-batching request engine: every result equals the same request run
alone (through a plan), requests on different cells overlap, resident S-matrices are reused by
key, admission respects the HBM budget, and impossible requests fail cleanly."""
import threading

import numpy as np
import pytest
import torch

from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300.runtime import PrismSimulation, Server

from test_gpu_parity import DET, c_grid, det_c, grid_dict, rand_v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()
    yield
    torch.cuda.synchronize()


def cells():
    """Uneven cells: grid, cell size, slices, f, seed."""
    out = []
    for i, (n, cell, H, f) in enumerate([(64, 8.0, 3, 2), (128, 12.8, 5, 4), (256, 16.0, 8, 4), (64, 6.4, 2, 1),
                                           (128, 16.0, 4, 2), (256, 32.0, 6, 8)]):
        g = grid_dict(n, n, cell, cell, H, 2.0, f)
        V = torch.from_numpy(rand_v(H, n, n, 40 + i)).pin_memory()
        out.append((g, V))
    return out


def requests_for(g, i):
    rng = np.random.Generator(np.random.PCG64(60 + i))
    n = 7 + 5 * i
    x0 = rng.uniform(0, g["cell_x"], n)
    y0 = rng.uniform(0, g["cell_y"], n)
    probe = P.make_probe(20.0 if i % 2 == 0 else 15.0, c1=10.0 * i)
    return probe, x0, y0


def alone(g, V, probe, x0, y0):
    sim = PrismSimulation(c_grid(g))
    sim.build(V.cuda())
    out = sim.scan(probe, x0, y0, det_c(DET)).cpu().numpy()
    sim.close()
    return out


def test_results_identical_alone_and_in_the_mix():
    cs = cells()
    refs = []
    for i, (g, V) in enumerate(cs):
        probe, x0, y0 = requests_for(g, i)
        refs.append(alone(g, V, probe, x0, y0))
    srv = Server(max_inflight=4)
    tickets = []
    for i, (g, V) in enumerate(cs):       # all submitted at once: they are admitted as slots free up
        probe, x0, y0 = requests_for(g, i)
        tickets.append(srv.submit(c_grid(g), V, probe, x0, y0, det_c(DET), key=0))
    for (t, out), ref in zip(tickets, refs):
        srv.wait(t)
        assert np.array_equal(out, ref)
    info = srv.stats()
    assert info.completed == len(cs) and info.running == 0 and info.pending == 0
    srv.close()


def test_resident_smatrix_is_reused_by_key():
    g = grid_dict(128, 128, 12.8, 12.8, 4, 2.0, 2)
    V = torch.from_numpy(rand_v(4, 128, 128, 70)).pin_memory()
    srv = Server(max_inflight=2)
    probes = [P.make_probe(20.0), P.make_probe(12.0, c1=50.0), P.make_probe(18.0, c3=1e4)]
    x0, y0 = np.linspace(0, 12.8, 9), np.linspace(3, 9, 9)
    first = srv.submit(c_grid(g), V, probes[0], x0, y0, det_c(DET), key=7)
    st = srv.wait(first[0])
    assert st.smatrix_reused == 0
    for pr in probes:
        t, out = srv.submit(c_grid(g), V, pr, x0, y0, det_c(DET), key=7)
        st = srv.wait(t)
        assert st.smatrix_reused == 1
        assert np.array_equal(out, alone(g, V, pr, x0, y0))
    assert srv.stats().resident == 1
    # the same key with another grid is refused
    g2 = grid_dict(64, 64, 12.8, 12.8, 4, 2.0, 2)
    t, _ = srv.submit(c_grid(g2), V, probes[0], x0, y0, det_c(DET), key=7)
    with pytest.raises(P.PrismError) as e:
        srv.wait(t)
    assert e.value.status == P.PRISM_ERR_INVALID
    srv.close()


def test_admission_under_a_tight_budget_and_concurrent_submitters():
    cs = cells()[:4]
    budget = 160 << 20  # fits about one 256^2 cell at a time
    srv = Server(hbm_budget_bytes=budget, max_inflight=4)
    results = {}

    def client(i):
        g, V = cs[i]
        probe, x0, y0 = requests_for(g, i)
        t, out = srv.submit(c_grid(g), V, probe, x0, y0, det_c(DET))
        srv.wait(t)
        results[i] = (out, alone(g, V, probe, x0, y0))

    threads = [threading.Thread(target=client, args=(i,)) for i in range(len(cs))]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert len(results) == len(cs)
    for out, ref in results.values():
        assert np.array_equal(out, ref)
    info = srv.stats()
    assert info.peak_bytes <= budget
    srv.close()


def test_request_larger_than_budget_fails_cleanly():
    g = grid_dict(256, 256, 16.0, 16.0, 8, 2.0, 4)
    V = torch.zeros((8, 256, 256)).pin_memory()
    srv = Server(hbm_budget_bytes=8 << 20, max_inflight=1)
    t, _ = srv.submit(c_grid(g), V, P.make_probe(20.0), [1.0], [1.0], det_c(DET))
    with pytest.raises(P.PrismError) as e:
        srv.wait(t)
    assert e.value.status == P.PRISM_ERR_BUDGET
    srv.close()


def test_requests_on_different_cells_overlap_on_the_device():
    # a long request (1024^2, 24 slices, 129 beams, 2000 probes) and a short one on another cell,
    # submitted together: both are in flight on the device at the same time (their device intervals,
    # taken by CUDA events on their own streams, intersect)
    from paper_1702_01904_gb300 import specimens
    big = specimens.workload_amorphous_carbon(n_slices=24)
    gb = P.grid_from_workload(big)
    Vb = torch.from_numpy(big.potential()).pin_memory()
    xb, yb = big.scan_positions()
    gs = grid_dict(256, 256, 16.0, 16.0, 8, 2.0, 4)
    Vs = torch.from_numpy(rand_v(8, 256, 256, 71)).pin_memory()
    probe = P.make_probe(20.0)
    srv = Server(max_inflight=4)
    warm, _ = srv.submit(c_grid(gs), Vs, probe, [1.0], [1.0], det_c(DET))  # code paths, not measured
    srv.wait(warm)
    t1, o1 = srv.submit(gb, Vb, probe, xb[:2000], yb[:2000], det_c(DET), key=11, px=200, py=10)
    t2, o2 = srv.submit(c_grid(gs), Vs, probe, np.linspace(0, 16, 64), np.linspace(2, 9, 64), det_c(DET), key=12)
    s1, s2 = srv.wait(t1), srv.wait(t2)
    srv.close()
    assert 0 <= s1.device_start_ms < s1.device_end_ms and 0 <= s2.device_start_ms < s2.device_end_ms
    assert max(s1.device_start_ms, s2.device_start_ms) < min(s1.device_end_ms, s2.device_end_ms), \
        (s1.device_start_ms, s1.device_end_ms, s2.device_start_ms, s2.device_end_ms)
    assert np.isfinite(o1).all() and np.isfinite(o2).all() and o1.sum() > 0 and o2.sum() > 0


def test_cancel_queued_and_running_requests():
    # one slot: a long request (1024^2, 24 slices, 129 beams) runs while a short one waits in the
    # queue; both are cancelled
    from paper_1702_01904_gb300 import specimens
    big = specimens.workload_amorphous_carbon(n_slices=24)
    Vb = torch.from_numpy(big.potential()).pin_memory()
    xb, yb = big.scan_positions()
    g = grid_dict(256, 256, 16.0, 16.0, 8, 2.0, 4)
    V = torch.from_numpy(rand_v(8, 256, 256, 72)).pin_memory()
    probe = P.make_probe(20.0)
    x0, y0 = np.linspace(0, 16, 50), np.linspace(1, 15, 50)
    srv = Server(max_inflight=1)
    t_run, o_run = srv.submit(P.grid_from_workload(big), Vb, probe, xb[:4000], yb[:4000], det_c(DET), key=22,
                              px=200, py=20)
    t_q, o_q = srv.submit(c_grid(g), V, probe, x0, y0, det_c(DET), key=21)
    o_run[:] = -1.0
    o_q[:] = -1.0
    srv.cancel(t_q)      # queued behind the first (one slot): leaves the queue
    srv.cancel(t_run)    # admitted or about to be: its result is discarded
    for t in (t_q, t_run):
        with pytest.raises(P.PrismError) as e:
            srv.wait(t)
        assert e.value.status == P.PRISM_ERR_CANCELLED
    assert np.all(o_q == -1.0) and np.all(o_run == -1.0)
    with pytest.raises(P.PrismError) as e:
        srv.cancel(t_q)  # already finished and waited for
    assert e.value.status == P.PRISM_ERR_INVALID
    # the server still serves afterwards
    t, out = srv.submit(c_grid(g), V, probe, x0, y0, det_c(DET), key=21)
    srv.wait(t)
    assert np.array_equal(out, alone(g, V, probe, x0, y0))
    srv.close()


def test_large_cell_in_a_mix_is_identical_alone():
    # a 2048^2 cell of the large serving workload (529 beams, 128-pixel windows; 6 slices) scanned at
    # two probe steps from one resident S-matrix, mixed with small cells on their own S-matrices:
    # every result equals the same request run alone through a plan
    from paper_1702_01904_gb300 import specimens
    w = specimens.workload_nanoparticle_on_carbon(n_slices=6, particle_diameter=8.0)
    Vl = torch.from_numpy(specimens.project_potential_vectorised(w.specimen, w.nx, w.ny, w.n_slices, w.dz)).pin_memory()
    gl = P.grid_from_workload(w)
    probe = P.make_probe(20.0)
    rois = []
    for k, step in enumerate((0.2, 0.5)):
        xs = 40.0 + 7.0 * k + step * np.arange(16)
        yy, xx = np.meshgrid(45.0 + step * np.arange(16), xs, indexing="ij")
        rois.append((xx.ravel(), yy.ravel()))
    sim = PrismSimulation(gl)
    sim.build(Vl.cuda())
    refs_l = [sim.scan(probe, x, y, det_c(DET), px=16, py=16).cpu().numpy() for x, y in rois]
    sim.close()
    torch.cuda.empty_cache()
    cs = cells()[:3]
    refs_s = [alone(g, V, *requests_for(g, i)) for i, (g, V) in enumerate(cs)]
    srv = Server(hbm_budget_bytes=60 << 30, max_inflight=4)
    tickets = []
    for i in range(3):
        g, V = cs[i]
        tickets.append(("s", i, srv.submit(c_grid(g), V, *requests_for(g, i), det_c(DET))))
        if i < 2:
            x, y = rois[i]
            tickets.append(("l", i, srv.submit(gl, Vl, probe, x, y, det_c(DET), key=31, px=16, py=16)))
    for kind, i, (t, out) in tickets:
        srv.wait(t)
        assert np.array_equal(out, refs_l[i] if kind == "l" else refs_s[i]), (kind, i)
    assert srv.stats().peak_bytes <= 60 << 30
    srv.close()
